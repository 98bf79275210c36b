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


def test_gpr_cv_matches_fluctuation_formula_and_closed_form():
    # Sec. III.B's Gaussian-process form of C = -beta^2 dE/dbeta: on the ED energy curve it
    # reproduces the fluctuation formula; on the two-level curve the closed form, also with
    # noise of 1e-4 on E (noise variance given as 1e-8)
    lat = Lattice(2, 3, 1, J1=1.0)
    spec = ed.spectrum(lat)
    betas = np.linspace(0.05, 4.0, 60)
    cv = observables.cv_from_energy_gpr(betas, ed.thermal(spec, lat.N, betas)[:, 0], noise=1e-12)
    probe = np.linspace(0.3, 3.7, 15)
    assert np.allclose(cv(probe), ed.thermal(spec, lat.N, probe)[:, 1], atol=1e-4)
    b2 = np.linspace(0.0, 3.0, 121)
    pr = np.linspace(0.2, 2.8, 14)
    exact = pr ** 2 / np.cosh(pr) ** 2
    assert np.allclose(observables.cv_from_energy_gpr(b2, -np.tanh(b2), noise=1e-12)(pr), exact,
                       atol=1e-4)
    noisy = -np.tanh(b2) + 1e-4 * np.random.default_rng(3).standard_normal(b2.size)
    assert np.allclose(observables.cv_from_energy_gpr(b2, noisy, noise=1e-8)(pr), exact, atol=3e-3)
