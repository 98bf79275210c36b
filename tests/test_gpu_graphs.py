"""CUDA graphs of the batched engine (peps_set_graphs): replaying the captured launch sequences
of the Metropolis sweep and the evaluation gives the same bits as direct launches, over
several cooling steps with both sampling exponents, and counts the same launches."""
import ctypes

import numpy as np
import pytest

from paper_2409_05285_gb300 import binding

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


@pytest.mark.parametrize("prec,shape", [(binding.PEPS_FP64, (4, 4, 2, 4)),
                                        (binding.PEPS_TF32, (6, 6, 4, 16))])
def test_graph_replays_match_direct_launches(prec, shape):
    import torch
    L1, L2, D, chi = shape
    out = []
    side = torch.cuda.Stream()   # stream capture needs a stream other than the legacy default
    for graphs in (False, True):
        ctx = binding.Context(L1, L2, D, chi, 96, J1=1.0, J2=0.3, precision=prec, seed=9,
                              init_noise=1e-2, block_mode=binding.PEPS_BLOCKS_BATCHED,
                              stream=ctypes.c_void_p(side.cuda_stream))
        ctx.set_graphs(graphs)
        l0 = ctx.launches()
        stats = []
        for k in range(4):
            p = 1 if k < 2 else 2
            stats.append(ctx.step(n_sweeps=1, p=p, tau=0.05))
        S = ctx.get_configs()
        la, sg, es, ea, O = ctx.eval_batch(S)
        out.append((ctx.get_theta(), S, la, es, ea, O, stats, ctx.launches() - l0))
        assert (ctx.graphs_captured() > 0) == graphs
        ctx.close()
    a, b = out
    for x, y in zip(a[:6], b[:6]):
        assert np.array_equal(x, y)
    assert [s["E_site"] for s in a[6]] == [s["E_site"] for s in b[6]]
    assert [s["accept"] for s in a[6]] == [s["accept"] for s in b[6]]
    assert a[7] == b[7]


def test_graphs_need_the_batched_engine():
    ctx = binding.Context(3, 3, 2, 4, 8, precision=binding.PEPS_FP64,
                          block_mode=binding.PEPS_BLOCKS_NARROW)
    with pytest.raises(binding.PepsError):
        ctx.set_graphs(True)
    ctx.close()
