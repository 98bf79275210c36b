"""Pins of the oracle's SR step (Eqs. 5-7, 10) and CG solve."""
import numpy as np
import pytest

from oracle import ed, observables, peps, sr
from oracle.lattice import Lattice


def _random_problem(ns=40, npar=25, seed=31):
    rng = np.random.default_rng(seed)
    Of = rng.standard_normal((ns, npar))
    w = rng.random(ns)
    w /= w.sum()
    E = rng.standard_normal(ns)
    return Of, w, E


def test_two_pass_apply_is_eq6_matrix():
    Of, w, E = _random_problem()
    obar = w @ Of
    G6 = Of.T @ (w[:, None] * Of) - np.outer(obar, obar)        # <O_k O_k'> - <O_k><O_k'>
    v = np.random.default_rng(1).standard_normal(Of.shape[1])
    assert np.allclose(sr.apply_G(Of, w, obar, v, 0.0), G6 @ v, atol=1e-13)
    assert np.allclose(sr.apply_G(Of, w, obar, v, 0.3), G6 @ v + 0.3 * v, atol=1e-13)
    assert np.allclose(sr.dense_G(Of, w, obar, 0.0), G6, atol=1e-13)


def test_gradient_is_eq7():
    Of, w, E = _random_problem()
    obar, Ebar, g = sr.sr_quantities(Of, w, E)
    assert Ebar == pytest.approx(float(w @ E))
    g_centered = (Of - obar).T @ (w * (E - Ebar))
    assert np.allclose(g, g_centered, atol=1e-13)


def test_cg_matches_dense_solve():
    Of, w, E = _random_problem(ns=30, npar=60)     # rank-deficient G (N_s < N_p), as in the paper
    obar, _, g = sr.sr_quantities(Of, w, E)
    eps = 1e-3
    x, it, res = sr.cg(lambda v: sr.apply_G(Of, w, obar, v, eps), g, 1e-12, 500)
    xd = np.linalg.solve(sr.dense_G(Of, w, obar, eps), g)
    assert res <= 1e-12
    assert np.allclose(x, xd, rtol=1e-9, atol=1e-12 * np.abs(xd).max())


def test_cg_stops_at_maxit_and_zero_rhs():
    Of, w, E = _random_problem()
    obar, _, g = sr.sr_quantities(Of, w, E)
    x, it, res = sr.cg(lambda v: sr.apply_G(Of, w, obar, v, 1e-4), g, 1e-14, 3)
    assert it == 3 and res > 1e-14
    x0, it0, _ = sr.cg(lambda v: v, np.zeros(5), 1e-10, 10)
    assert it0 == 0 and not np.any(x0)


def test_weights():
    la = np.log(np.array([1.0, 2.0, 4.0, 1e-3]))
    assert np.allclose(sr.weights(la, 2), 0.25)
    w1 = sr.weights(la, 1)
    assert np.allclose(w1, np.array([1, 2, 4, 1e-3]) / 7.001)


def test_expand_O_layout():
    lat = Lattice(2, 3, 2)
    rng = np.random.default_rng(2)
    S = rng.integers(0, 4, (3, lat.N))
    O = rng.standard_normal((3, lat.No))
    Of = sr.expand_O(lat, S, O)
    assert np.count_nonzero(Of) == O.size
    for i in range(lat.N):
        for n in range(3):
            a = lat.theta_off[i] + S[n, i] * lat.sz[i]
            assert np.array_equal(Of[n, a:a + lat.sz[i]], O[n, lat.o_off[i]:lat.o_off[i + 1]])


def _sr_run(tau, t_end, noise=1e-3, eps=1e-4):
    """Deterministic SR with every configuration of 2x2 enumerated (weights |rho|^2), D = 4
    (exact representation); returns E/site - E_ED(4t) at the end."""
    lat = Lattice(2, 2, 4, J1=1.0)
    th = peps.init_theta(lat, 3, noise)
    cfgs = np.array([ed.config_of_index(k, 4) for k in range(256)])
    spec = ed.spectrum(lat)
    t = 0.0
    n = int(round(t_end / tau))
    for step in range(n + 1):
        res = [peps.eval_sample(lat, th, S, 64) for S in cfgs]
        la = np.array([r['log_abs'] for r in res])
        ok = np.isfinite(la)
        w = np.zeros(256)
        w[ok] = np.exp(2 * (la[ok] - la[ok].max()))
        w /= w.sum()
        es = np.array([r['e_sys'] if f else 0.0 for r, f in zip(res, ok)])
        ea = np.array([r['e_anc'] if f else 0.0 for r, f in zip(res, ok)])
        if step == n:
            obs = observables.observables(lat, t, w, es, ea, cfgs)
            return obs['E_site'] - ed.thermal(spec, lat.N, [4 * t])[0][0]
        O = np.array([r['O'] if f else np.zeros(lat.No) for r, f in zip(res, ok)])
        Of = sr.expand_O(lat, cfgs, O)
        obar, _, g = sr.sr_quantities(Of, w, es + ea)
        x, _, _ = sr.cg(lambda v: sr.apply_G(Of, w, obar, v, eps), g, 1e-10, 1000)
        th = th - tau * x
        t += tau


def test_sr_dynamics_follow_exact_evolution():
    # theta' = theta - tau G^-1 g approximates exp(-tau calH) (Eq. 5): against the exact
    # thermal energy at beta_obs = 4t the error is first order in tau.
    e2 = _sr_run(0.02, 0.12)
    e1 = _sr_run(0.01, 0.12)
    assert abs(e1) < 0.75 * abs(e2)
    assert abs(e2) < 0.02 and abs(e1) < 0.01
