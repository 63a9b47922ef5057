"""bench.py's reference arm (the FP64 oracle timed on the host cores) prints one JSON line
with the keys of the benchmark contract; it runs on the CPU alone."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def test_traffic_key_ignores_comments_but_not_code():
    """The key of bench.py's ncu traffic table hashes what the compiler acts on: a
    comment or re-indentation keeps it, a changed token does not, and the serving
    kernels (batch.cuh) are outside the step kernel's sources."""
    sys.path.insert(0, ROOT)
    import bench
    code = "int f(int a) {\n  return a * 2;  // twice\n}\n/* block\ncomment */ int g;\n"
    same = "int f(int a) { return a * 2; }\n\n// another note\nint   g;"
    changed = "int f(int a) {\n  return a * 3;  // twice\n}\nint g;\n"
    assert bench.source_code_text(code) == bench.source_code_text(same)
    assert bench.source_code_text(code) != bench.source_code_text(changed)
    assert "batch.cuh" not in bench.KERNEL_SOURCES
    for f in bench.KERNEL_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_1910_13515_gb300", "csrc", f)), f
    assert len(bench.kernel_source_hash()) == 16


def test_poly_reference_arm_line():
    """The comparison model's reference arm: its numpy oracle on a window of the same lattice."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "poly", "--poly-n", "64", "--steps", "1", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "MLUPS" and d["value"] > 0
    assert d["config"]["cells"] == 64 * 64 and "64x64x1" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_poly_helpers():
    sys.path.insert(0, ROOT)
    import argparse

    import numpy as np

    import bench
    from paper_1910_13515_gb300 import inputs
    s = inputs.subsonic_box(40, 30, 1, seed=1)
    c, desc = bench.poly_window(s, 16)
    assert (c.nx, c.ny, c.nz) == (16, 16, 1) and c.ncells == 256 and "16x16x1" in desc
    # the window is the lattice's first 16 x 16 block, x fastest
    np.testing.assert_array_equal(c.rho.reshape(16, 16), s.rho.reshape(30, 40)[:16, :16])
    np.testing.assert_array_equal(c.u[1].reshape(16, 16), s.u[1].reshape(30, 40)[:16, :16])
    for n, want in ((2048, "periodic 2048x2048x1 (the paper's comparison size)"),
                    (1024, "periodic 1024x1024x1,")):
        text = bench.workload_text(argparse.Namespace(workload="poly", poly_n=n, mach=0.8))
        assert want in text, text
