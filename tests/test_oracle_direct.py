"""Pins of the oracle's direct (autoregressive) sampling and its reweighted form (App. A,
Eqs. A2-A7) against brute-force sums over every configuration, the chain rule of
probability, the beta = 0 closed form and a sampled histogram."""
import numpy as np
import pytest
from scipy import stats

from oracle import direct, ed, peps
from oracle.lattice import Lattice


def _all_configs(N):
    return np.array([ed.config_of_index(k, N) for k in range(4 ** N)])


def _p0(lat, th, cfgs):
    return np.array([peps.amplitude_exact(lat, th, S) ** 2 for S in cfgs])


def _theta(lat, seed):
    return np.random.default_rng(seed).standard_normal(lat.Np)


def test_fully_fixed_double_layer_is_rho_squared():
    # the double-layer contraction at a complete configuration is rho(S)^2 (single layer, Eq. 4)
    lat = Lattice(2, 3, 2)
    th = _theta(lat, 1)
    rng = np.random.default_rng(2)
    for _ in range(5):
        S = rng.integers(0, 4, lat.N)
        assert direct.marginal(lat, th, S) == pytest.approx(peps.amplitude_exact(lat, th, S) ** 2,
                                                            rel=1e-12)


def test_marginal_is_sum_over_completions():
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 3)
    cfgs = _all_configs(lat.N)
    p0 = _p0(lat, th, cfgs)
    rng = np.random.default_rng(4)
    for i in range(lat.N + 1):
        prefix = rng.integers(0, 4, i)
        fixed = -np.ones(lat.N, dtype=np.int64)
        fixed[:i] = prefix
        mask = np.all(cfgs[:, :i] == prefix, axis=1)
        assert direct.marginal(lat, th, fixed) == pytest.approx(p0[mask].sum(), rel=1e-12)


def test_plain_direct_sampling_is_p0():
    # exponent 1, b_d = 1: prod_i p_2c = p_0 / sum p_0 (Eq. A2, chain rule)
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 5)
    cfgs = _all_configs(lat.N)
    p0 = _p0(lat, th, cfgs)
    q = np.array([direct.sample_prob(lat, th, S, b_d=1.0, exponent=1.0) for S in cfgs])
    assert np.allclose(q, p0 / p0.sum(), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("b_d,exponent", [(1.0, 0.5), (0.3, 0.5), (0.05, 0.5), (1.0, 1.0)])
def test_sampling_distribution_is_normalised(b_d, exponent):
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 6)
    q = [direct.sample_prob(lat, th, S, b_d, exponent) for S in _all_configs(lat.N)]
    assert sum(q) == pytest.approx(1.0, abs=1e-12)


def test_reweighting_flattens_and_lowers_the_diagonal():
    # p_3c = sqrt(p_2c) moves weight toward rare configurations; b_d < 1 lowers the diagonal
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 7) * 0.3
    T = lat.tensors(th)
    for i in range(lat.N):       # a strongly diagonal state, as at high temperature
        T[i][0].reshape(-1)[0] += 3.0
        T[i][3].reshape(-1)[0] += 3.0
    cfgs = _all_configs(lat.N)
    diag = np.all(cfgs // 2 == cfgs % 2, axis=1)
    q2 = np.array([direct.sample_prob(lat, th, S, 1.0, 1.0) for S in cfgs])
    q3 = np.array([direct.sample_prob(lat, th, S, 1.0, 0.5) for S in cfgs])
    q4 = np.array([direct.sample_prob(lat, th, S, 0.2, 0.5) for S in cfgs])
    assert q2[diag].sum() > q3[diag].sum() > q4[diag].sum()


def test_beta0_closed_form():
    # rho = I: p_2c vanishes for s != s' and is 1/2 for both diagonal states, so every
    # diagonal configuration has q = 2^-N whatever b_d, and no other is drawn
    lat = Lattice(2, 2, 2)
    th = peps.init_theta(lat, 0, 0.0)
    for S in _all_configs(lat.N):
        is_diag = np.all(S // 2 == S % 2)
        for b_d in (1.0, 0.1):
            q = direct.sample_prob(lat, th, S, b_d, 0.5)
            assert q == pytest.approx(2.0 ** -lat.N if is_diag else 0.0, abs=1e-15)


def test_reweighted_estimate_matches_exact_average():
    # draws from q with b_d = 0.5: their histogram follows q (chi^2), and the Eq. A7
    # estimate with r_4 = p_0 / q reproduces the exact p_0 average of a diagonal indicator
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 8)
    cfgs = _all_configs(lat.N)
    p0 = _p0(lat, th, cfgs)
    b_d = 0.5
    q = np.array([direct.sample_prob(lat, th, S, b_d, 0.5) for S in cfgs])
    rng = np.random.default_rng(9)
    n = 1500
    idx, f, lq, lp = [], [], [], []
    for _ in range(n):
        S, logq, logp0 = direct.draw(lat, th, rng.random(lat.N), b_d, 0.5)
        k = 0
        for x in S:
            k = 4 * k + int(x)
        idx.append(k)
        assert logq == pytest.approx(np.log(q[k]), rel=1e-10, abs=1e-12)
        assert logp0 == pytest.approx(np.log(p0[k]), rel=1e-10, abs=1e-12)
        f.append(float(np.all(S // 2 == S % 2)))
        lq.append(logq)
        lp.append(logp0)
    counts = np.bincount(idx, minlength=len(cfgs))
    keep = q * n >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    exp = np.append(q[keep] * n, q[~keep].sum() * n)
    exp *= obs.sum() / exp.sum()
    assert stats.chisquare(obs, exp).pvalue > 1e-3
    diag = np.all(cfgs // 2 == cfgs % 2, axis=1)
    exact = p0[diag].sum() / p0.sum()
    r = p0 / np.where(q > 0, q, 1.0)
    sd = np.sqrt(np.sum(q * (r / np.sum(q * r)) ** 2 * (diag - exact) ** 2) / n)
    assert abs(direct.reweighted_mean(f, lq, lp) - exact) < 5 * sd + 1e-12


def test_literal_unnormalised_product_is_biased():
    # the reading of Eq. A6-A7: with r_4 = p_0 / prod p_4c (no per-site normalisation) the
    # ratio estimate over q differs from the exact average; with r_4 = p_0 / q it equals it
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 10)
    cfgs = _all_configs(lat.N)
    p0 = _p0(lat, th, cfgs)
    b_d = 0.4
    f = np.array([float(S[0] // 2) for S in cfgs])
    exact = np.sum(p0 * f) / p0.sum()
    q = np.array([direct.sample_prob(lat, th, S, b_d, 0.5) for S in cfgs])
    p4 = []
    for S in cfgs:
        w = 1.0
        for i in range(lat.N):
            w *= direct.site_weights(direct.conditional(lat, th, S[:i]), b_d, 0.5)[int(S[i])]
        p4.append(w)
    p4 = np.array(p4)
    ok = q > 0
    r_q = p0[ok] / q[ok]
    r_p4 = p0[ok] / p4[ok]
    assert np.sum(q[ok] * r_q * f[ok]) / np.sum(q[ok] * r_q) == pytest.approx(exact, rel=1e-12)
    assert abs(np.sum(q[ok] * r_p4 * f[ok]) / np.sum(q[ok] * r_p4) - exact) > 1e-3


def test_update_bd():
    N = 4
    diag = np.zeros((10, N), dtype=np.int64)                 # all diagonal (S = 0)
    mixed = np.vstack([diag[:5], np.ones((5, N), dtype=np.int64)])   # half diagonal
    assert direct.diagonal_fraction(diag) == 1.0
    assert direct.diagonal_fraction(mixed) == 0.5
    assert direct.update_bd(0.8, diag, N) == pytest.approx(0.8 * 0.5 ** 0.25)
    assert direct.update_bd(0.8, mixed, N) == 0.8
    assert direct.update_bd(1.0, mixed, N) == 1.0
    three_quarters = np.vstack([diag[:6], np.ones((2, N), dtype=np.int64)])
    assert direct.update_bd(1.0, three_quarters, N) == pytest.approx((0.5 / 0.75) ** 0.25)


@pytest.mark.parametrize("b_d,exponent", [(1.0, 1.0), (0.4, 0.5)])
def test_boundary_mps_form_equals_exact_at_large_chi(b_d, exponent):
    # the method's steps (summed down environments, up environments of the sampled rows,
    # one-row strips per candidate) at chi above every exact bond reproduce the exact draws
    lat = Lattice(3, 3, 2)
    th = _theta(lat, 11)
    rng = np.random.default_rng(12)
    down = direct.summed_down_envs(lat, th, 64)
    for _ in range(6):
        u = rng.random(lat.N)
        S, lq, _ = direct.draw(lat, th, u, b_d, exponent)
        Sb, lqb = direct.draw_bmps(lat, th, u, 64, b_d, exponent, down=down)
        assert np.array_equal(S, Sb)
        assert lqb == pytest.approx(lq, rel=1e-9, abs=1e-12)


def test_boundary_mps_truncation_changes_the_marginals():
    # at chi below the exact bond the truncated marginals differ (a check that chi is used)
    lat = Lattice(3, 3, 2)
    th = _theta(lat, 13)
    u = np.random.default_rng(14).random(lat.N)
    _, lq_exact, _ = direct.draw(lat, th, u, 1.0, 1.0)
    S2, lq2 = direct.draw_bmps(lat, th, u, 2, 1.0, 1.0)
    q_exact_S2 = np.log(direct.sample_prob(lat, th, S2, 1.0, 1.0))
    assert abs(lq2 - q_exact_S2) > 1e-8


def test_sr_weights_of_plain_direct_draws_are_uniform():
    # exponent 1, b_d = 1 draws p_0 exactly (q = p_0 / sum p_0): r_4 = p_0 / q is the same
    # for every sample, so the p = 0 weights of the SR step are 1/n
    from oracle import sr
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 11)
    rng = np.random.default_rng(12)
    lq, lp = [], []
    for _ in range(12):
        _, logq, logp0 = direct.draw(lat, th, rng.random(lat.N), 1.0, 1.0)
        lq.append(logq)
        lp.append(logp0)
    w = sr.weights(0.5 * np.array(lp), 0, np.array(lq))
    assert np.allclose(w, 1.0 / 12, rtol=1e-10)


def test_sr_weights_of_reweighted_draws_give_exact_average():
    # the p = 0 weights over every configuration, each counted with its probability q, give
    # the exact p_0 average of any function (Eq. A7); they differ from uniform weights
    from oracle import sr
    lat = Lattice(2, 2, 2)
    th = _theta(lat, 13)
    cfgs = _all_configs(lat.N)
    p0 = _p0(lat, th, cfgs)
    q = np.array([direct.sample_prob(lat, th, S, 0.3, 0.5) for S in cfgs])
    ok = q > 0
    f = np.array([float(S[1] % 2) - 0.3 * float(S[2] // 2) for S in cfgs])[ok]
    w = sr.weights(0.5 * np.log(p0[ok]), 0, np.log(q[ok]))
    exact = np.sum(p0 * np.array([float(S[1] % 2) - 0.3 * float(S[2] // 2) for S in cfgs])) / p0.sum()
    assert np.sum(q[ok] * w * f) / np.sum(q[ok] * w) == pytest.approx(exact, rel=1e-12)
    assert not np.allclose(w, w[0])
