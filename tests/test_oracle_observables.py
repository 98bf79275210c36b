"""Pins of the oracle's observables (Eq. 11, specific heat, Eq. 13): fed the exact
vectorised thermal state (all configurations, weights |rho|^2), they reproduce ED."""
import numpy as np
import pytest

from oracle import ed, observables
from oracle.lattice import Lattice


@pytest.mark.parametrize("J2", [0.0, 0.5])
def test_observables_on_exact_state(J2):
    lat = Lattice(2, 2, 1, J1=1.0, J2=J2)
    H = ed.full_hamiltonian(lat)
    I = np.eye(H.shape[0])
    perm = ed.pair_to_config_index(lat.N)
    Hsys = np.kron(H, I)[np.ix_(perm, perm)]        # H x I on configurations
    Hanc = np.kron(I, H.T)[np.ix_(perm, perm)]      # I x H^T
    cfgs = np.array([ed.config_of_index(k, lat.N) for k in range(4 ** lat.N)])
    spec = ed.spectrum(lat)
    for t in [0.05, 0.25, 1.0]:
        v = ed.evolve_identity(lat, t)
        nz = np.abs(v) > 1e-300
        es = np.where(nz, (Hsys @ v) / np.where(nz, v, 1), 0.0)
        ea = np.where(nz, (Hanc @ v) / np.where(nz, v, 1), 0.0)
        w = v * v / (v @ v)
        obs = observables.observables(lat, t, w, es, ea, cfgs)
        E, C, X = ed.thermal(spec, lat.N, [4 * t])[0]
        assert obs['beta_obs'] == 4 * t
        assert obs['E_site'] == pytest.approx(E, abs=1e-12)
        assert obs['C_site'] == pytest.approx(C, abs=1e-11)
        assert obs['chi'] == pytest.approx(X, abs=1e-12)


def test_beta0_values():
    # beta = 0: uniform over diagonal configurations; E = 0, <Mz^2> = N/4.
    lat = Lattice(2, 3, 1)
    N = lat.N
    cfgs = np.array([[3 * ((x >> k) & 1) for k in range(N)] for x in range(2 ** N)])
    w = np.full(len(cfgs), 1.0 / len(cfgs))
    zeros = np.zeros(len(cfgs))
    obs = observables.observables(lat, 0.0, w, zeros, zeros, cfgs)
    assert obs['Mz2'] == pytest.approx(N / 4)
    assert obs['diag_frac'] == 1.0 and obs['E_site'] == 0.0 and obs['chi'] == 0.0


def test_spline_cv_matches_fluctuation_formula():
    # Sec. III.A: C from the derivative of a B-spline through E(beta) equals the fluctuation
    # formula beta^2 (<H^2> - <H>^2)/N of exact diagonalisation (2x3 Heisenberg)
    lat = Lattice(2, 3, 1, J1=1.0)
    spec = ed.spectrum(lat)
    betas = np.linspace(0.05, 4.0, 80)
    th = ed.thermal(spec, lat.N, betas)
    cv = observables.cv_from_energy_curve(betas, th[:, 0])
    probe = np.linspace(0.3, 3.7, 15)
    assert np.allclose(cv(probe), ed.thermal(spec, lat.N, probe)[:, 1], atol=2e-4)


def test_spline_cv_two_level_closed_form_and_noise():
    # two levels at -+1: E = -tanh(beta), C = beta^2 / cosh(beta)^2; with noise of 1e-4 on
    # E a smoothing spline (smoothing factor n sigma^2) still gives C within 1e-2
    betas = np.linspace(0.0, 3.0, 121)
    cv = observables.cv_from_energy_curve(betas, -np.tanh(betas))
    probe = np.linspace(0.2, 2.8, 14)
    assert np.allclose(cv(probe), probe ** 2 / np.cosh(probe) ** 2, atol=1e-5)
    rng = np.random.default_rng(3)
    noisy = -np.tanh(betas) + 1e-4 * rng.standard_normal(betas.size)
    cvn = observables.cv_from_energy_curve(betas, noisy, smoothing=betas.size * 1e-8)
    assert np.allclose(cvn(probe), probe ** 2 / np.cosh(probe) ** 2, atol=1e-2)


def test_standard_error_iid_plain_weights():
    # p = 2 weights (1/n) on independent normal samples of variance sigma^2: the estimate
    # is sigma_hat / sqrt(n); over many repetitions its mean matches the observed spread of
    # the sample means and sigma / sqrt(n) (to the few per cent of 4000 repetitions)
    rng = np.random.default_rng(11)
    n, sigma, reps = 50, 1.7, 4000
    w = np.full(n, 1.0 / n)
    means, ses = [], []
    for _ in range(reps):
        h = 3.0 + sigma * rng.standard_normal(n)
        means.append(float(w @ h))
        ses.append(observables.standard_error(w, h))
    exact = sigma / np.sqrt(n)
    assert np.std(means) == pytest.approx(exact, rel=0.04)
    # the population-variance form is biased low by sqrt((n-1)/n) on average, plus the
    # Jensen gap of a square root: both under 2 % at n = 50
    assert np.mean(ses) == pytest.approx(exact, rel=0.03)


def test_standard_error_weighted_ratio_estimate():
    # p = 1 weights (Eq. A1): samples drawn from q, weights proportional to p/q, normalised.
    # Target p = N(1, 1), proposal q = N(0, 1.5^2), h(x) = x^2: the weighted mean estimates
    # E_p[x^2] = 2, and the delta-method error matches the observed spread of the estimates
    rng = np.random.default_rng(12)
    n, reps = 400, 3000
    est, ses = [], []
    for _ in range(reps):
        x = 1.5 * rng.standard_normal(n)
        logr = -0.5 * (x - 1.0) ** 2 + 0.5 * (x / 1.5) ** 2
        r = np.exp(logr - logr.max())
        w = r / r.sum()
        h = x * x
        est.append(float(w @ h))
        ses.append(observables.standard_error(w, h))
    assert np.mean(est) == pytest.approx(2.0, abs=0.02)
    assert np.mean(ses) == pytest.approx(np.std(est), rel=0.06)


def test_standard_error_special_cases():
    # one distinct value: zero error; two equally weighted values a, b: abs(a - b) / (2 sqrt 2)
    assert observables.standard_error([0.25] * 4, [2.0] * 4) == 0.0
    assert observables.standard_error([0.5, 0.5], [1.0, 3.0]) == pytest.approx(np.sqrt(2.0) / 2)
