"""Per-kernel launch statistics: the per-launch algorithmic bytes add up to the per-kernel
sums, and the counter sees every launch."""
import pytest

from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


def test_launch_bytes_match_kernel_sums():
    from paper_2409_05285_gb300.build import build
    build()
    ctx = binding.Context(6, 6, 4, 16, 256, precision=binding.PEPS_TF32, seed=7)
    ctx.mc_sweep(1, p=1)
    ctx.profile(True, gemm_only=True)
    n0 = ctx.launches()
    ctx.eval_chains()
    per = {k: ctx.profile_launch_bytes(k) for k in ("kb_gemm_tc", "kb_gemm")}
    sums = ctx.profile_read()
    ctx.profile(False)
    assert per["kb_gemm_tc"], "the TF32 path runs its contractions on the tensor cores"
    for k, v in per.items():
        launches, ms, nbytes, _ = sums.get(k, (0, 0.0, 0.0, 0.0))
        assert launches == len(v)
        assert nbytes == pytest.approx(sum(v), rel=1e-12)
        assert all(b > 0 for b in v) and ms > 0 or not v
    assert ctx.launches() - n0 >= sum(len(v) for v in per.values())
    assert ctx.profile_launch_bytes("kb_gemm_tc") == []   # folded by profile_read
    ctx.close()
