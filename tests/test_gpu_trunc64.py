"""The float32 modes with a float64 truncation (peps_set_trunc_fp64): results against the
FP64 oracle within the float32 bounds, against the float64 engine on a cooled state of the
bench's shape (errors of both truncation arithmetics printed side by side), and the calls it
refuses."""
import time

import numpy as np
import pytest

from oracle import peps
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def _ctx(L1, L2, D, chi, n, prec, J2=0.0, seed=0):
    return binding.Context(L1, L2, D, chi, n, J1=1.0, J2=J2, precision=prec, seed=seed,
                           block_mode=binding.PEPS_BLOCKS_BATCHED)


@pytest.mark.parametrize("prec,tol", [(binding.PEPS_FP32, 2e-4), (binding.PEPS_TF32, 5e-2)])
def test_matches_oracle(prec, tol):
    # the oracle comparison of the float32 modes (4x4, D=3, chi=4 truncating, NNN bonds),
    # now with the float64 Jacobi; the tolerances of those modes
    L1, L2, D, chi, J2, n = 4, 4, 3, 4, 0.5, 6
    lat = Lattice(L1, L2, D, J1=1.0, J2=J2)
    th = wl.random_theta(L1, L2, D, seed=5, scale=0.1 if prec == binding.PEPS_TF32 else 0.3,
                         diag_bias=1.0)
    S = wl.random_configs(L1, L2, n, seed=6)
    ctx = _ctx(L1, L2, D, chi, n, prec, J2=J2)
    ctx.set_theta(th)
    ctx.set_trunc_fp64(True)
    la, sg, es, ea, O = ctx.eval_batch(S)
    for k in range(n):
        r = peps.eval_sample(lat, th, S[k], chi)
        assert sg[k] == r['sign']
        assert abs(la[k] - r['log_abs']) <= tol
        scale = max(1.0, abs(r['e_sys']), abs(r['e_anc']))
        assert abs(es[k] - r['e_sys']) <= tol * scale
        assert abs(ea[k] - r['e_anc']) <= tol * scale
        assert np.max(np.abs(O[k].astype(np.float64) - r['O'])) <= 10 * tol * max(1.0, np.max(np.abs(r['O'])))
    ctx.close()


def test_cooled_state_against_float64_engine():
    # 8x8, D=4, chi=16, a state cooled by four FP64 SR steps: amplitudes and local energies of
    # FP32 and TF32 with float32 and with float64 truncation against the FP64 engine, and the
    # cost of the float64 Jacobi in an evaluation of 2048 chains
    L, D, chi, n = 8, 4, 16, 256
    ref = _ctx(L, L, D, chi, n, binding.PEPS_FP64, seed=3)
    ref.mc_sweep(2, p=1)
    for _ in range(4):
        ref.step(n_sweeps=1, p=2, tau=0.1, eps=1e-4, max_cg=100, cg_tol=1e-10)
    th, S = ref.get_theta(), ref.get_configs()
    la64, sg64, es, ea, _ = ref.eval_batch(S, with_O=False)
    e64 = (es + ea) / (2 * L * L)
    ref.close()
    for prec in (binding.PEPS_FP32, binding.PEPS_TF32):
        errs = {}
        for t64 in (False, True):
            c = _ctx(L, L, D, chi, n, prec, seed=3)
            c.set_theta(th)
            c.set_trunc_fp64(t64)
            la, sg, es, ea, _ = c.eval_batch(S, with_O=False)
            e = (es + ea) / (2 * L * L)
            assert np.all(sg == sg64)
            errs[t64] = (np.median(np.abs(la - la64)), np.max(np.abs(la - la64)),
                         np.max(np.abs(e - e64)), abs(np.mean(e) - np.mean(e64)))
            assert errs[t64][3] <= 1e-3
            c.close()
        print(f"\nprec {prec}: |dlog rho| median/max, max |dE_loc|/2N, |dE/site| -- float32 Jacobi "
              f"{errs[False][0]:.2e}/{errs[False][1]:.2e}, {errs[False][2]:.2e}, {errs[False][3]:.2e}; "
              f"float64 Jacobi {errs[True][0]:.2e}/{errs[True][1]:.2e}, {errs[True][2]:.2e}, {errs[True][3]:.2e}")
    c = _ctx(L, L, D, chi, 2048, binding.PEPS_TF32, seed=4)
    c.mc_sweep(1, p=1)
    ms = {}
    for t64 in (False, True, False):
        c.set_trunc_fp64(t64)
        c.eval_chains()
        t0 = time.perf_counter()
        c.eval_chains()
        ms[t64] = (time.perf_counter() - t0) * 1e3
    print(f"TF32 evaluation of 2048 chains: float32 Jacobi {ms[False]:.1f} ms, float64 Jacobi {ms[True]:.1f} ms")
    c.close()


def test_refused_where_it_does_not_apply():
    a = _ctx(3, 3, 2, 4, 4, binding.PEPS_FP64)
    with pytest.raises(binding.PepsError) as e:
        a.set_trunc_fp64(True)
    assert e.value.code == binding.PEPS_ESTATE
    b = binding.Context(3, 3, 2, 4, 4, precision=binding.PEPS_FP32, block_mode=binding.PEPS_BLOCKS_NARROW)
    with pytest.raises(binding.PepsError) as e:
        b.set_trunc_fp64(True)
    assert e.value.code == binding.PEPS_ESTATE
    c = _ctx(3, 3, 2, 4, 4, binding.PEPS_TF32)
    assert c.lib.peps_set_trunc_fp64(c.ctx, 2) == binding.PEPS_EINVAL
    for x in (a, b, c):
        x.close()
