"""Host logic of the paper's experiments (no GPU): the downward Mach scan of the
stability map (Sec. III A) returns the largest stable grid value, and the
parameter mapping of each run follows the section's definitions."""
import math

import pytest

from paper_2312_10318_gb300 import experiments as E
from paper_2312_10318_gb300 import params as P

N = 128


def _ma_of(case):
    u_c = case[0]
    return round(u_c / E.CS, 6)


def _re_of(case):
    u_c, tau1 = case[0], case[1]
    return u_c * N / P.nu_from_tau(tau1)


def test_dsl_run_length_is_two_convective_times():
    # t_c = L / (c_s Ma) with L = N nodes and c = 1: 2 t_c = 2 N / u_c steps
    assert E.dsl_steps(0.5, N) == math.ceil(2 * N / (0.5 / math.sqrt(3.0)))
    assert E.dsl_steps(0.62, N) == 716


def test_stability_scan_finds_the_largest_stable_grid_value():
    # a fake stability law: monotone for one pair, never stable for another,
    # and stable in two separate Ma bands for a third
    law = {
        (5e3, 1.6): lambda ma: ma <= 0.62 + 1e-9,
        (5e3, 0.1): lambda ma: False,
        (5e3, None): lambda ma: ma <= 0.20 + 1e-9 or 0.47 - 1e-9 <= ma <= 0.49 + 1e-9,
    }
    seen = []

    def survives(cases):
        out = []
        for c in cases:
            re = round(_re_of(c))
            inv = None if abs(c[2] - c[1]) < 1e-15 else round(1.0 / c[2], 6)
            seen.append((inv, _ma_of(c), c[3]))
            assert c[3] == E.dsl_steps(_ma_of(c), N)
            out.append(law[(re, inv)](_ma_of(c)))
        return out

    res = E.stability_map(re_list=(5e3,), inv_tau2=[1.6, 0.1], survives=survives)
    assert res["trt_rlb"][5e3] == {1.6: 0.62, 0.1: 0.0}
    assert res["rlb"][5e3] == 0.49
    # nothing above the reported value was left untried, nothing below it run
    tried = {}
    for inv, ma, _ in seen:
        tried.setdefault(inv, set()).add(round(ma, 2))
    assert tried[1.6] >= {round(0.01 * k, 2) for k in range(63, 101)}
    assert min(tried[1.6]) >= 0.57
    assert tried[0.1] == {round(0.01 * k, 2) for k in range(1, 101)}
    assert res["runs"] == len(seen)


def test_stability_runs_use_the_sections_parameters():
    cases = []

    def survives(cs):
        cases.extend(cs)
        return [True] * len(cs)

    E.stability_map(re_list=(1e4,), inv_tau2=[1.6], rlb=False, survives=survives)
    for c in cases:
        assert _re_of(c) == pytest.approx(1e4, rel=1e-12)
        assert 1.0 / c[2] == pytest.approx(1.6, rel=1e-12)


def test_sen_law_values():
    # C_d = 0.7496 + 10.5767 Re^-0.66 (Sec. III D), evaluated by hand
    assert E.sen_drag(1.0) == pytest.approx(11.3263, abs=1e-4)
    assert E.sen_drag(10.0) == pytest.approx(0.7496 + 10.5767 / 10 ** 0.66, rel=1e-12)
