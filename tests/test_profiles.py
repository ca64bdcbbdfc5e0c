"""The committed trace profile belongs to the trace kernel's current code: the benchmark line takes
its DRAM traffic and instruction count from it, and reports them only while the recorded digest
matches (a changed kernel must be profiled again)."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_trace_profile_matches_the_kernel_source():
    bench = _bench()
    assert bench.profiled("dram_bytes_per_launch") is not None, (
        "profiles/trace_large_1080p_bench_poses.md was taken on other trace kernel code "
        f"(current digest {bench.kernel_digest()})")
    assert bench.profiled("warp_instructions_per_launch") > 1e8


def test_digest_ignores_comments(tmp_path):
    bench = _bench()
    d0 = bench.kernel_digest()
    for p in ("paper_2006_14726_b300/csrc/trace.cu", "paper_2006_14726_b300/csrc/common.cuh"):
        src = open(os.path.join(ROOT, p), encoding="utf-8").read()
        dst = tmp_path / p
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_text("// a comment\n" + src.replace("\n", "  \n", 3) + "\n/* another */\n")
    bench.ROOT = str(tmp_path)
    assert bench.kernel_digest() == d0
