"""The library's specific heat from an energy curve (peps_cv_spline, Sec. III.A: C/N =
-beta^2 dE/dbeta of a spline through E against beta), on the CPU: against the exact
diagonalisation fluctuation formula, the two-level closed form with and without noise, and the
oracle's B-spline form of the same estimate."""
import numpy as np
import pytest

from oracle import ed, observables
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def test_matches_fluctuation_formula_and_oracle():
    lat = Lattice(2, 3, 1, J1=1.0)
    spec = ed.spectrum(lat)
    betas = np.linspace(0.05, 4.0, 80)
    E = ed.thermal(spec, lat.N, betas)[:, 0]
    probe = np.linspace(0.3, 3.7, 15)
    cv = binding.cv_spline(betas, E, probe)
    assert np.allclose(cv, ed.thermal(spec, lat.N, probe)[:, 1], atol=2e-4)
    assert np.allclose(cv, observables.cv_from_energy_curve(betas, E)(probe), atol=2e-4)


def test_two_level_closed_form_and_noise():
    # two levels at -+1: E = -tanh(beta), C = beta^2 / cosh(beta)^2
    betas = np.linspace(0.0, 3.0, 121)
    probe = np.linspace(0.2, 2.8, 14)
    exact = probe ** 2 / np.cosh(probe) ** 2
    assert np.allclose(binding.cv_spline(betas, -np.tanh(betas), probe), exact, atol=1e-5)
    rng = np.random.default_rng(3)
    noisy = -np.tanh(betas) + 1e-4 * rng.standard_normal(betas.size)
    got = binding.cv_spline(betas, noisy, probe, smoothing=betas.size * 1e-8)
    assert np.allclose(got, exact, atol=1e-2)
    # unordered input gives the same curve
    perm = rng.permutation(betas.size)
    assert np.allclose(binding.cv_spline(betas[perm], -np.tanh(betas)[perm], probe), exact, atol=1e-5)


def test_straight_line_and_arguments():
    # E linear in beta: dE/dbeta = slope everywhere, also with smoothing
    b = np.linspace(0.5, 2.0, 7)
    for s in (0.0, 1e-3):
        assert np.allclose(binding.cv_spline(b, 0.3 - 0.2 * b, [0.7, 1.9], smoothing=s),
                           [0.2 * 0.49, 0.2 * 3.61], atol=1e-12)
    with pytest.raises(binding.PepsError):
        binding.cv_spline([0.1, 0.2], [1.0, 2.0], [0.1])
    with pytest.raises(binding.PepsError):
        binding.cv_spline([0.1, 0.1, 0.3], [1.0, 2.0, 3.0], [0.1])
    with pytest.raises(binding.PepsError):
        binding.cv_spline([0.1, 0.2, 0.3], [1.0, 2.0, 3.0], [0.1], smoothing=-1.0)
