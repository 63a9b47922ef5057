"""The generated straight-line D3Q39 arithmetic in the CUDA sources is exactly what its
generator emits, and the generator's self-checks (every emitted sum against the direct sum over
the 39 velocities, the z-mirror variants on z-symmetric inputs) pass."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1910_13515_gb300", "csrc")


def test_generated_header_matches_its_generator():
    spec = importlib.util.spec_from_file_location("gen_d3q39", os.path.join(CSRC, "gen_d3q39.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    lines, nmono = gen.generate()  # runs the self-checks
    with open(os.path.join(CSRC, "d3q39_gen.cuh")) as fh:
        assert fh.read() == "\n".join(lines)
    assert nmono == 60
