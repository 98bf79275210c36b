"""Evaluation of several lattices of different sizes in one launch (peps_group_*): every
context's results are the bits its own evaluation gives (amplitudes, energies, O rows, seen
through the SR update and the observables), in FP64 and FP32, and invalid groups are refused."""
import time

import numpy as np
import pytest

from paper_2409_05285_gb300 import binding
from paper_2409_05285_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


SHAPES = [  # (L1, L2, D, chi, J2, n): uneven lattices, bonds and chain counts
    (4, 4, 2, 4, 0.0, 7),
    (3, 5, 3, 5, 0.5, 13),
    (6, 6, 2, 8, 0.0, 40),
    (5, 4, 3, 6, 0.2, 3),
]


def _contexts(prec, shapes):
    out = []
    for k, (L1, L2, D, chi, J2, n) in enumerate(shapes):
        c = binding.Context(L1, L2, D, chi, n, J1=1.0, J2=J2, precision=prec, seed=k,
                            block_mode=binding.PEPS_BLOCKS_NARROW)
        th = wl.random_theta(L1, L2, D, seed=10 + k, scale=0.3, diag_bias=1.0)
        S = wl.random_configs(L1, L2, n, seed=20 + k)
        out.append((c, th, S))
    return out


def _step(c, p=2):
    obs = c.observables(p=p)
    st = c.sr_step(0.05, eps=1e-3, max_cg=200, cg_tol=1e-12, p=p)
    return obs, st, c.get_theta()


@pytest.mark.parametrize("prec", [binding.PEPS_FP64, binding.PEPS_FP32])
def test_group_gives_each_contexts_own_bits(prec):
    ctxs = _contexts(prec, SHAPES)
    for c, _, _ in ctxs:   # t > 0, so that C and chi carry their beta_obs factors
        c.eval_chains()
        c.sr_step(0.05, eps=1e-2, max_cg=5, cg_tol=1e-6, p=2)
    ref = []
    for c, th, S in ctxs:
        c.set_theta(th)
        c.set_configs(S)
        c.eval_chains()
        ref.append(_step(c))
    for c, th, S in ctxs:
        c.set_theta(th)
        c.set_configs(S)
    grp = binding.Group([c for c, _, _ in ctxs])
    grp.eval()
    for (c, _, _), (obs, st, th2) in zip(ctxs, ref):
        obs_g, st_g, th2_g = _step(c)
        for key in ("E_site", "E_err", "diag_frac"):
            assert obs_g[key] == obs[key], key
            assert st_g[key] == st[key], key
        # C and chi of the same samples at the later time t: their beta_obs factors scaled out
        b, bg = obs["beta_obs"], obs_g["beta_obs"]
        assert obs_g["C_site"] / bg ** 2 == pytest.approx(obs["C_site"] / b ** 2, rel=1e-12)
        assert obs_g["chi_sus"] / bg == pytest.approx(obs["chi_sus"] / b, rel=1e-12)
        assert st_g["cg_iters"] == st["cg_iters"]
        assert np.array_equal(th2_g, th2)
    # a second evaluation after the update sees the new parameters of every context
    for c, th, S in ctxs:
        c.set_configs(S)
    grp.eval()
    for c, _, _ in ctxs:
        assert np.isfinite(c.observables(p=2)["E_site"])
    grp.close()
    for c, _, _ in ctxs:
        c.close()


def test_invalid_groups_are_refused():
    a = binding.Context(4, 4, 2, 4, 8, precision=binding.PEPS_FP64, block_mode=binding.PEPS_BLOCKS_NARROW)
    b = binding.Context(3, 3, 2, 4, 8, precision=binding.PEPS_FP32, block_mode=binding.PEPS_BLOCKS_NARROW)
    c = binding.Context(3, 3, 2, 4, 8, precision=binding.PEPS_FP64, block_mode=binding.PEPS_BLOCKS_BATCHED)
    d = binding.Context(3, 3, 2, 4, 8, precision=binding.PEPS_FP64, block_mode=binding.PEPS_BLOCKS_WIDE)
    for bad in ([a, b], [a, c], [a, d], [a, a], []):
        with pytest.raises(binding.PepsError) as e:
            binding.Group(bad)
        assert e.value.code == binding.PEPS_EINVAL
    for x in (a, b, c, d):
        x.close()


def test_group_launch_against_separate_launches():
    # eight small lattices: one launch for all of them against one launch per lattice
    shapes = [(4, 4, 2, 4, 0.0, 64), (4, 5, 2, 4, 0.0, 64), (5, 5, 2, 4, 0.0, 64),
              (3, 6, 2, 4, 0.3, 64), (6, 4, 2, 4, 0.0, 64), (4, 4, 3, 6, 0.0, 64),
              (5, 3, 2, 4, 0.0, 64), (6, 6, 2, 4, 0.0, 64)]
    ctxs = _contexts(binding.PEPS_FP32, shapes)
    for c, th, S in ctxs:
        c.set_theta(th)
        c.set_configs(S)
    grp = binding.Group([c for c, _, _ in ctxs])
    grp.eval()
    for c, _, _ in ctxs:
        c.eval_chains()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        for c, _, _ in ctxs:
            c.eval_chains()
    t1 = time.perf_counter()
    for _ in range(reps):
        grp.eval()
    t2 = time.perf_counter()
    sep, one = (t1 - t0) / reps * 1e3, (t2 - t1) / reps * 1e3
    print(f"\n8 lattices x 64 chains, FP32: separate launches {sep:.2f} ms, one group launch {one:.2f} ms")
    assert one > 0 and sep > 0
    grp.close()
    for c, _, _ in ctxs:
        c.close()
