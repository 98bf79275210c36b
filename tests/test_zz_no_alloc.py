"""The allocation-free evaluation entry point (peps_eval_batch_noalloc) gives the same
results as the regular evaluation, through the C ABI, on two calls in a row.

Some callers cannot allocate GPU memory (a host framework that owns the device memory pool,
a plug-in called during CUDA-graph capture, a process with a fixed memory budget); this
entry point serves them from a fixed device array inside the library.  This file is named
so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def _noalloc(params, theta_d, S_d, outs, stream=None):
    lib = binding.load()
    la, sg, es, ea, O = outs
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    return lib.peps_eval_batch_noalloc(ctypes.byref(params), p(theta_d), p(S_d), int(S_d.shape[0]),
                                       p(la), p(sg), p(es), p(ea), p(O), stream)


@pytest.mark.parametrize("prec", [binding.PEPS_FP64, binding.PEPS_FP32])
def test_noalloc_matches_eval_batch_twice(prec):
    torch = pytest.importorskip("torch")
    from paper_2409_05285_gb300.build import build
    build()
    L1, L2, D, chi, J2, nb = 4, 5, 3, 5, 0.4, 23
    # the entry point runs the per-chain (narrow-block) engine: compare with the same engine
    ref = binding.Context(L1, L2, D, chi, 4, J1=1.0, J2=J2, precision=prec, seed=1,
                          block_mode=binding.PEPS_BLOCKS_NARROW)
    th = wl.random_theta(L1, L2, D, seed=3, scale=0.3, diag_bias=1.0)
    ref.set_theta(th)
    dev = torch.device("cuda:0")
    theta_d = torch.from_numpy(th).to(dev)
    odt = torch.float64 if prec == binding.PEPS_FP64 else torch.float32
    tol = 1e-10 if prec == binding.PEPS_FP64 else 2e-4
    for call, seed in enumerate((7, 8)):   # two calls in a row, different batches
        S = wl.random_configs(L1, L2, nb, seed=seed)
        la0, sg0, es0, ea0, O0 = ref.eval_batch(S)
        S_d = torch.from_numpy(S).to(dev)
        outs = (torch.empty(nb, dtype=torch.float64, device=dev),
                torch.empty(nb, dtype=torch.int8, device=dev),
                torch.empty(nb, dtype=torch.float64, device=dev),
                torch.empty(nb, dtype=torch.float64, device=dev),
                torch.empty((nb, ref.No), dtype=odt, device=dev))
        rc = _noalloc(ref.params, theta_d, S_d, outs)
        torch.cuda.synchronize()
        assert rc == binding.PEPS_OK, binding.load().peps_last_error(None)
        la, sg, es, ea, O = (t.cpu().numpy() for t in outs)
        assert np.array_equal(sg, sg0), call
        assert np.max(np.abs(la - la0)) <= tol, call
        scale = max(1.0, np.max(np.abs(es0)), np.max(np.abs(ea0)))
        assert np.max(np.abs(es - es0)) <= tol * scale and np.max(np.abs(ea - ea0)) <= tol * scale
        oscale = max(1.0, float(np.max(np.abs(O0))))
        assert np.max(np.abs(O.astype(np.float64) - O0.astype(np.float64))) <= tol * 10 * oscale
    ref.close()


def test_noalloc_rejects_problem_above_its_work_space():
    torch = pytest.importorskip("torch")
    lib = binding.load()
    big = binding.Params(L1=16, L2=16, model=0, J1=1.0, J2=0.0, D=8, chi=64, n_chains=1,
                         precision=binding.PEPS_FP64, init_noise=0.0, seed=0, n_blocks=0)
    dev = torch.device("cuda:0")
    th = torch.zeros(16, dtype=torch.float64, device=dev)
    S = torch.zeros((1, 256), dtype=torch.uint8, device=dev)
    rc = lib.peps_eval_batch_noalloc(ctypes.byref(big), ctypes.c_void_p(th.data_ptr()),
                                     ctypes.c_void_p(S.data_ptr()), 1, None, None, None, None,
                                     None, None)
    assert rc == binding.PEPS_EINVAL
    assert b"PEPS_NOALLOC_SCRATCH_BYTES" in lib.peps_last_error(None)


def _outs(torch, nb, No, odt, dev):
    return (torch.full((nb,), 7.0, dtype=torch.float64, device=dev),
            torch.full((nb,), 5, dtype=torch.int8, device=dev),
            torch.full((nb,), 7.0, dtype=torch.float64, device=dev),
            torch.full((nb,), 7.0, dtype=torch.float64, device=dev),
            torch.zeros((nb, No), dtype=odt, device=dev))


def test_noalloc_persistent_blocks_on_a_side_stream():
    # 8x8 D=4 chi=16 in float64 needs about 3.8 MB of work space per block, so the fixed
    # array holds about a dozen blocks and each block loops over several of the 40 samples;
    # the call is made on a non-default stream and compared with the regular evaluation
    torch = pytest.importorskip("torch")
    L, D, chi, nb = 8, 4, 16, 40
    ref = binding.Context(L, L, D, chi, 4, J1=1.0, precision=binding.PEPS_FP64, seed=1,
                          block_mode=binding.PEPS_BLOCKS_NARROW)
    th = wl.random_theta(L, L, D, seed=13, scale=0.2, diag_bias=1.0)
    ref.set_theta(th)
    S = wl.random_configs(L, L, nb, seed=14)
    la0, sg0, es0, ea0, O0 = ref.eval_batch(S)
    dev = torch.device("cuda:0")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        theta_d = torch.from_numpy(th).to(dev)
        S_d = torch.from_numpy(S).to(dev)
        outs = _outs(torch, nb, ref.No, torch.float64, dev)
        for call in range(2):
            rc = _noalloc(ref.params, theta_d, S_d, outs, ctypes.c_void_p(side.cuda_stream))
            assert rc == binding.PEPS_OK, binding.load().peps_last_error(None)
            side.synchronize()
            la, sg, es, ea, O = (t.cpu().numpy() for t in outs)
            assert np.array_equal(sg, sg0), call
            assert np.max(np.abs(la - la0)) <= 1e-10, call
            scale = max(1.0, np.max(np.abs(es0)), np.max(np.abs(ea0)))
            assert np.max(np.abs(es - es0)) <= 1e-10 * scale
            assert np.max(np.abs(ea - ea0)) <= 1e-10 * scale
            assert np.max(np.abs(O - O0)) <= 1e-9 * max(1.0, float(np.max(np.abs(O0))))
    ref.close()


def test_noalloc_skips_samples_with_invalid_entries():
    # an entry above 3 is caught by the kernel before it reads any parameter slice: that
    # sample's scalar outputs are NaN with sign 0, the other samples are evaluated as usual
    torch = pytest.importorskip("torch")
    L1, L2, D, chi, nb = 3, 4, 2, 4, 6
    ref = binding.Context(L1, L2, D, chi, 4, J1=1.0, precision=binding.PEPS_FP64, seed=1,
                          block_mode=binding.PEPS_BLOCKS_NARROW)
    th = wl.random_theta(L1, L2, D, seed=15, scale=0.3, diag_bias=1.0)
    ref.set_theta(th)
    S = wl.random_configs(L1, L2, nb, seed=16)
    la0, sg0, es0, ea0, _ = ref.eval_batch(S, with_O=False)
    bad = S.copy()
    bad[2, 5] = 4
    bad[4, 0] = 255
    dev = torch.device("cuda:0")
    outs = _outs(torch, nb, ref.No, torch.float64, dev)
    rc = _noalloc(ref.params, torch.from_numpy(th).to(dev), torch.from_numpy(bad).to(dev), outs)
    torch.cuda.synchronize()
    assert rc == binding.PEPS_OK
    la, sg, es, ea, _ = (t.cpu().numpy() for t in outs)
    for k in range(nb):
        if k in (2, 4):
            assert np.isnan(la[k]) and np.isnan(es[k]) and np.isnan(ea[k]) and sg[k] == 0
        else:
            assert abs(la[k] - la0[k]) <= 1e-10 and sg[k] == sg0[k]
    ref.close()
