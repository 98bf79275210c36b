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
    assert tune["kc_max"] in (16, 32, 64)
    assert tune["pipelined"] in (0, 1, 2)
    assert tune["stage_kb"] in (64, 96, 192)
    assert tune["trunc_threads"] in (32, 64, 256)
    assert 0 < tune["ms_after"] <= tune["ms_before"]
    ctx.sr_step(0.02)   # the tuner left a valid evaluation of the chains behind
    ctx2 = binding.Context(L, L, D, chi, 64, precision=binding.PEPS_TF32, seed=5)
    t2 = ctx2.autotune(reps=0)
    keys = ("grid_pct", "db_bytes", "ffma_g", "kc_max", "pipelined", "stage_kb", "trunc_threads")
    assert [t2[k] for k in keys] == [tune[k] for k in keys]
    ctx.close()
    ctx2.close()


def test_pinned_shapes_keep_results():
    from paper_2409_05285_gb300.build import build
    build()
    ctx = binding.Context(6, 6, 4, 16, 256, precision=binding.PEPS_TF32, seed=6)
    ctx.mc_sweep(1, p=1)
    S = ctx.get_configs()
    ctx.set_tune(100, 12 * 1024, 256, 64)
    ref = ctx.eval_batch(S)
    # both tensor-core kernel forms (register-staged, cp.async-pipelined for short or for all
    # vector contractions, with stage rings of 64-192 KB) and truncation blocks of 32-256
    # threads give the same bits
    for shapes in ((50, 0, 16, 16, 0, 96, 256), (200, 48 * 1024, 1, 32, 1, 64, 32),
                   (100, 12 * 1024, 256, 8, 0, 96, 128), (100, 12 * 1024, 256, 64, 1, 192, 64),
                   (100, 12 * 1024, 256, 64, 2, 96, 32), (100, 12 * 1024, 256, 32, 2, 192, 256)):
        ctx.set_tune(*shapes)
        got = ctx.autotune(reps=0)
        keys = ("grid_pct", "db_bytes", "ffma_g", "kc_max", "pipelined", "stage_kb", "trunc_threads")
        assert tuple(got[k] for k in keys) == shapes
        for a, b in zip(ref, ctx.eval_batch(S)):
            assert np.array_equal(a, b)
    for bad in ((0, 0, 16, 64), (100, 0, 0, 64), (100, 0, 16, 12), (100, 0, 16, 72), (100, 0, 16, 64, 3),
                (100, 0, 16, 64, 1, 16), (100, 0, 16, 64, 1, 256), (100, 0, 16, 64, 1, 96, 48)):
        with pytest.raises(RuntimeError):
            ctx.set_tune(*bad)
    ctx.close()


def test_truncation_block_size_keeps_fp64_bits():
    # the float64 engine's Jacobi truncation pairs columns as a 256-thread block would in any
    # block size, so its results do not depend on the size
    from paper_2409_05285_gb300.build import build
    build()
    ctx = binding.Context(6, 6, 4, 16, 64, precision=binding.PEPS_FP64, seed=7,
                          block_mode=binding.PEPS_BLOCKS_BATCHED)
    ctx.mc_sweep(1, p=1)
    S = ctx.get_configs()
    ctx.set_tune(100, 12 * 1024, 256, 64, 1, 96, 256)
    ref = ctx.eval_batch(S)
    for tt in (32, 64, 128):
        ctx.set_tune(100, 12 * 1024, 256, 64, 1, 96, tt)
        for a, b in zip(ref, ctx.eval_batch(S)):
            assert np.array_equal(a, b)
    ctx.close()
