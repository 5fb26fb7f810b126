"""The ncu figures bench.py reports beside its timings (DRAM traffic of the
headline kernel, FP64 instructions per interaction of the double-double
kernel) are tied to the sources they were captured on by sha256; bench.py
reports null for a figure whose sources changed.  This CPU check keeps the
committed figures current: a kernel change must come with a new capture."""
import hashlib
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _sha(path):
    with open(os.path.join(ROOT, path), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def test_recorded_counters_match_current_sources():
    b = _bench()
    for rec in (b.TRAFFIC, b.DD_INSTR):
        assert len(rec["files"]) == len(rec["sha256"])
        for f, h in zip(rec["files"], rec["sha256"]):
            assert _sha(f) == h, f
    assert b.TRAFFIC["bytes_per_launch"] > 0
    assert b.DD_INSTR["fp64_thread_instr_per_interaction"] > 0
