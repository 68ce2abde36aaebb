"""The C-ABI library loads and exports every entry point include/trtrlb.h declares,
and the ctypes mirror of trtrlb_params matches the C layout.  No compute calls:
these run without a GPU."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2312_10318_gb300 import _build, _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "trtrlb.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(trtrlb_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return _lib.load()


def test_library_exports_every_declared_function(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(_lib.SIGNATURES)


def test_no_cuda_call_needed_for_error_strings(lib):
    assert lib.trtrlb_strerror(0) == b"ok"
    assert lib.trtrlb_strerror(_lib.EINVAL) == b"invalid argument"
    p = _lib.Params()
    lib.trtrlb_default_params(C.byref(p))
    assert (p.nx, p.ny, p.storage) == (64, 64, _lib.F32)


def test_create_rejects_invalid_parameters_before_touching_the_device(lib):
    p = _lib.Params()
    lib.trtrlb_default_params(C.byref(p))
    h = C.c_void_p()
    bad = [("tau_s", 0.5), ("nx", 0), ("storage", 9), ("g_mode", 7), ("rho0", -1.0),
           ("nx", (1 << 24) + 1), ("ny", 131071)]
    for field, val in bad:
        q = _lib.Params()
        C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
        setattr(q, field, val)
        assert lib.trtrlb_create(C.byref(q), None, None, C.byref(h)) == _lib.EINVAL, field
    q = _lib.Params()
    C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
    q.nx, q.ny = 1 << 24, 64                 # (nx + 63) * ny above 2^30
    assert lib.trtrlb_create(C.byref(q), None, None, C.byref(h)) == _lib.EINVAL
    q = _lib.Params()
    C.memmove(C.byref(q), C.byref(p), C.sizeof(p))
    q.tau_s2, q.magic = 0.4999, float("nan")     # tau_s2 = 1/2 is the smallest accepted
    assert lib.trtrlb_create(C.byref(q), None, None, C.byref(h)) == _lib.EINVAL
    assert b">= 1/2" in lib.trtrlb_last_error(None)
    q.tau_s2, q.magic = 1.0, 0.3     # disagree with tau_s = 0.8
    assert lib.trtrlb_create(C.byref(q), None, None, C.byref(h)) == _lib.EINVAL
    assert b"disagree" in lib.trtrlb_last_error(None)


def test_params_layout_matches_header():
    fields = [f for f, _ in _lib.Params._fields_]
    src = "#include <stdio.h>\n#include <stddef.h>\n#include \"trtrlb.h\"\nint main(void){\n"
    src += 'printf("%zu\\n", sizeof(trtrlb_params));\n'
    for f in fields:
        src += f'printf("%zu\\n", offsetof(trtrlb_params, {f}));\n'
    src += "return 0;}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "layout.c")
        exe = os.path.join(d, "layout")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals[0] == C.sizeof(_lib.Params)
    for f, off in zip(fields, vals[1:]):
        assert getattr(_lib.Params, f).offset == off, f
