"""Pins of the oracle's Fermi-Hubbard exact diagonalisation (Sec. III.B, Eq. 14): the beta = 0
closed form, the two-site ground state, free fermions (U = 0) from the one-particle spectrum,
the atomic limit (t = 0), and the next-nearest-neighbour spin correlation of the large-U
plaquette (the four-site Heisenberg ring)."""
import numpy as np
import pytest

from oracle import hubbard_ed as h


@pytest.mark.parametrize("shape", [(2, 2), (2, 3)])
def test_beta0_closed_form(shape):
    # every mode occupied with probability 1/2: E/N = U/4 - mu, D = 1/4, no correlations
    U, mu = 8.0, 3.0
    E, D, F = h.thermal(*shape, 1.0, U, mu, [0.0])[0]
    assert E == pytest.approx(U / 4 - mu, abs=1e-12)
    assert D == pytest.approx(0.25, abs=1e-12) and abs(F) < 1e-12


@pytest.mark.parametrize("U", [0.0, 2.0, 8.0])
def test_two_site_ground_state(U):
    H, _ = h.sector_hamiltonian(1, 2, 1.0, U, 0.0, 1, 1)
    assert np.linalg.eigvalsh(H).min() == pytest.approx((U - np.sqrt(U * U + 16.0)) / 2, abs=1e-12)


def test_free_fermions():
    nrow, ncol, t, mu = 2, 3, 1.0, 0.3
    N = nrow * ncol
    T = np.zeros((N, N))
    for i, j in h._nn_bonds(nrow, ncol):
        T[i, j] = T[j, i] = -t
    eps, phi = np.linalg.eigh(T)
    for beta in (0.5, 2.0, 6.0):
        f = 1.0 / (np.exp(beta * (eps - mu)) + 1.0)
        E = 2.0 * np.sum((eps - mu) * f) / N
        n_site = (phi ** 2) @ f                    # <n_i sigma>
        D = np.sum(n_site ** 2) / N                # Wick: <n_iu n_id> = <n_iu><n_id>
        got = h.thermal(nrow, ncol, t, 0.0, mu, [beta])[0]
        assert got[0] == pytest.approx(E, abs=1e-11)
        assert got[1] == pytest.approx(D, abs=1e-11)


def test_atomic_limit():
    U, mu = 6.0, 2.0
    for beta in (0.3, 1.0, 4.0):
        z = 1.0 + 2.0 * np.exp(beta * mu) + np.exp(-beta * (U - 2 * mu))
        E = (-2.0 * mu * np.exp(beta * mu) + (U - 2 * mu) * np.exp(-beta * (U - 2 * mu))) / z
        D = np.exp(-beta * (U - 2 * mu)) / z
        got = h.thermal(2, 2, 0.0, U, mu, [beta])[0]
        assert got[0] == pytest.approx(E, abs=1e-12)
        assert got[1] == pytest.approx(D, abs=1e-12) and abs(got[2]) < 1e-12


def test_large_U_plaquette_spin_correlation():
    # half filling, U >> t: the 2x2 plaquette's low-energy sector is the Heisenberg ring with
    # J = 4t^2/U, whose ground state has S_i.S_j = +1/4 across each diagonal
    U = 40.0
    E, D, F = h.thermal(2, 2, 1.0, U, U / 2, [400.0])[0]
    assert F == pytest.approx(0.25, abs=0.02)
    assert D < 0.01


def test_sampled_energy_of_the_evolved_state_is_thermal():
    # Eq. 11 for fermions: <E_sys + E_anc>_{|rho|^2} / 2 of e^{-t calH}|I> is the thermal
    # energy at beta_obs = 4t, and at t = 0 the state is the identity with E_loc = 2 H_ss
    nrow, ncol, t_hop, U, mu = 2, 2, 1.0, 4.0, 1.5
    H = h.full_hamiltonian(nrow, ncol, t_hop, U, mu)
    rho0 = h.evolved_rho(H, 0.0)
    assert np.allclose(rho0, np.eye(H.shape[0]), atol=1e-12)
    es0, ea0 = h.local_energies(H, rho0)
    assert np.allclose(np.diag(es0) + np.diag(ea0), 2 * np.diag(H), atol=1e-12)
    for t in (0.05, 0.3):
        rho = h.evolved_rho(H, t)
        es, ea = h.local_energies(H, rho)
        w = rho ** 2
        ok = rho != 0
        E = np.sum(w[ok] * (es[ok] + ea[ok])) / (2 * np.sum(w)) / (nrow * ncol)
        assert E == pytest.approx(h.thermal(nrow, ncol, t_hop, U, mu, [4 * t])[0][0], abs=1e-10)
