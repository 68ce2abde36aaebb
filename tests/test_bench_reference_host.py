"""The benchmark's reference arm (the FP64 oracle on the host cores) prints the
same one-line JSON contract as the GPU arm: run here with a tiny step count."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--reference-seconds", "4"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["value"] > 0 and d["unit"] == "MLUPS" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"]


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                        "--warmup", "3", "--reference-seconds", "4"], cwd=ROOT, capture_output=True, text=True,
                       timeout=300, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.strip().startswith("{")]


def test_source_hash_ignores_comments_but_not_code(tmp_path):
    """The recorded DRAM traffic stays valid across comment edits and is
    dropped when the device code changes."""
    import shutil
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2312_10318_gb300", "csrc")
    dst = tmp_path / "csrc"
    shutil.copytree(src, dst)
    h0 = bench.kernel_source_hash(str(dst))
    assert h0 == bench.kernel_source_hash()
    p = dst / "lb_batch.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n\n" + text.replace("namespace trt {", "namespace trt {  /* note */", 1))
    assert bench.kernel_source_hash(str(dst)) == h0
    p.write_text(text.replace("BATCH_THREADS = 256", "BATCH_THREADS = 128", 1))
    assert bench.kernel_source_hash(str(dst)) != h0


def test_cpu_baseline_reports_all_cores_and_one_core():
    """The oracle baseline gives its all-threads rate, a one-core rate of the
    same lattice, the CPU model, and leaves the oracle's thread count as it was."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    from paper_2312_10318_gb300 import workloads as W
    before = O.num_threads()
    cb = bench.cpu_baseline([W.double_shear_layer(64, re=1e4)], seconds=0.3)
    assert O.num_threads() == before
    assert cb["kind"] == "oracle" and cb["cores"] == before and cb["value"] > 0
    assert cb["one_core"]["value"] > 0 and cb["cpu_model"]


def test_launch_count_and_label_follow_the_reported_kernels():
    """The roofline divides by the step-kernel launches per time step, counted
    from the kernels the library reports: in a batch the AA lattices share a
    launch, the small TMA-fed ones share one per 16, every other two-buffer
    lattice takes its own; outside a batch every lattice is a launch."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2312_10318_gb300 import _lib
    assert set(bench.KERNEL_NAMES) == set(_lib.STEP_KINDS)
    assert bench.step_launches("batch", ["aa"] * 3) == 1
    assert bench.step_launches("batch", ["aa_vector"] * 3) == 1
    assert bench.step_launches("single", ["aa"] * 3) == 3
    assert bench.step_launches("batch", ["ab_tma_shared"] * 3) == 1
    assert bench.step_launches("batch", ["ab_tma_shared"] * 18) == 2     # 16 + 2
    assert bench.step_launches("batch", ["ab_tma"] * 3) == 3             # 4096^2: a launch each
    assert bench.step_launches("batch", ["ab_column"] * 3 + ["ab"]) == 4
    assert bench.step_launches("single", ["ab_tma_shared"] * 3) == 3
    assert "up to 16 lattices in one launch" in bench.kernel_label("batch", ["ab_tma_shared"] * 3)
    assert "one launch per lattice" in bench.kernel_label("single", ["ab_tma_shared"])
    assert bench.kernel_label("batch", ["aa_vector"] * 3).startswith("trt::k_step_group_vec ")
    assert bench.kernel_label("single", ["aa"]).startswith("trt::k_step ")
    assert "k_step_ab_col" in bench.kernel_label("batch", ["ab_column"] * 3)
    assert bench.kernel_label("batch", ["ab_column", "ab"]).count("+") == 1


def test_reference_arm_follows_the_g_mode():
    """With --g-mode current the oracle runs its current-level Phi and the line
    names that mode in its workload."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3",
                        "--g-mode", "current", "--reference-seconds", "4"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([l for l in r.stdout.splitlines() if l.strip().startswith("{")][0])
    assert d["config"]["workload"].endswith("G current") and d["value"] > 0


def test_walled_and_masked_workloads():
    """The creeping-flow and channel workloads: their geometry, and the mask's
    byte in the algorithmic bytes per node."""
    sys.path.insert(0, ROOT)
    import bench
    import oracle as O
    probs, st, desc = bench.workload("creeping4096x2048", size=(256, 128))
    p = probs[0]
    assert st == "f32" and p.periodic == (False, True) and p.mask is not None
    assert (p.mask[:, 0] == O.INLET).all() and (p.mask[:, -1] == O.OUTLET).all()
    assert (p.mask == O.SOLID).sum() == 64 * 64
    probs, st, desc = bench.workload("channel4096", size=(64, 32))
    assert probs[0].periodic == (True, False) and probs[0].mask is None and probs[0].g[0] > 0
    assert bench.bytes_per_node("f32", "lagged", mask=True) == 89
    assert bench.bytes_per_node("f16", "current", mask=True) == 37
