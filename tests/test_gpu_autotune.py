"""The launch-shape autotuner of the batched engine: its choice is one of the candidates,
it never changes a result, and later contexts of the same geometry start from it."""
import numpy as np
import pytest

from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


def test_autotune_keeps_results_and_is_shared_by_geometry():
    from paper_2409_05285_gb300.build import build
    build()
    L, D, chi, n = 6, 4, 16, 512
    ctx = binding.Context(L, L, D, chi, n, precision=binding.PEPS_TF32, seed=4)
    ctx.mc_sweep(2, p=1)
    S = ctx.get_configs()
    before = ctx.eval_batch(S)
    tune = ctx.autotune(reps=1)
    after = ctx.eval_batch(S)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    assert tune["grid_pct"] in (50, 100, 200)
    assert tune["db_bytes"] in (0, 12 * 1024, 48 * 1024)
    assert tune["ffma_g"] in (1, 16, 256)
    assert 0 < tune["ms_after"] <= tune["ms_before"]
    ctx.sr_step(0.02)   # the tuner left a valid evaluation of the chains behind
    ctx2 = binding.Context(L, L, D, chi, 64, precision=binding.PEPS_TF32, seed=5)
    t2 = ctx2.autotune(reps=0)
    assert (t2["grid_pct"], t2["db_bytes"], t2["ffma_g"]) == \
        (tune["grid_pct"], tune["db_bytes"], tune["ffma_g"])
    ctx.close()
    ctx2.close()
