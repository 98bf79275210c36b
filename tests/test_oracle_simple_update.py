"""Pins of the oracle's simple-update warm start (App. A; Eq. 3 applied bond by bond) against
the doubled Hamiltonian of exact diagonalisation, exact two-site evolution, the beta = 0
state, the system-ancilla symmetry of rho and the exact thermal energy at high temperature."""
import numpy as np
import pytest
from scipy.linalg import expm

from oracle import ed, peps, simple_update as su
from oracle.lattice import Lattice


def _vec(lat, th):
    return np.array([peps.amplitude_exact(lat, th, ed.config_of_index(k, lat.N))
                     for k in range(4 ** lat.N)])


def _evolved(lat, t, tau, D):
    st = su.SUState(lat)
    for _ in range(int(round(t / tau))):
        su.su_step(st, tau, D)
    return su.to_theta(st)


@pytest.mark.parametrize("J,tau", [(1.0, 0.05), (0.7, 0.3)])
def test_gate_is_the_doubled_bond_exponential(J, tau):
    # configuration index 4 S_0 + S_1 on a two-site lattice, calH from the ED code (Eq. 3)
    lat = Lattice(1, 2, 1, J1=J)
    Hd = ed.doubled_hamiltonian(lat)
    assert np.allclose(su.bond_gate(J, tau), expm(-tau * Hd), atol=1e-13)


def test_two_site_evolution_is_exact():
    # one bond: the Trotter step is exact, and D = 4 holds the full rank of the pair
    lat = Lattice(1, 2, 4)
    for t in (0.1, 0.5, 1.5):
        v = _vec(lat, _evolved(lat, t, 0.05, 4))
        w = ed.evolve_identity(lat, t)
        assert np.allclose(v / np.linalg.norm(v), w / np.linalg.norm(w), atol=1e-12)


def test_beta0_state_is_the_identity():
    lat = Lattice(2, 3, 3)
    v = _vec(lat, su.to_theta(su.SUState(lat)))
    w = ed.evolve_identity(lat, 0.0)
    assert np.allclose(v, w, rtol=0, atol=1e-12)


def test_rho_is_symmetric_in_system_and_ancilla():
    # H real symmetric: rho = e^{-2tH} = rho^T, i.e. rho(S) unchanged when s and s' swap at
    # every site (S = 2s + s' -> 2s' + s)
    lat = Lattice(2, 3, 4)
    v = _vec(lat, _evolved(lat, 0.3, 0.05, 4))
    idx = []
    for k in range(4 ** lat.N):
        S = ed.config_of_index(k, lat.N)
        St = (S % 2) * 2 + S // 2
        kk = 0
        for x in St:
            kk = 4 * kk + int(x)
        idx.append(kk)
    assert np.allclose(v, v[np.array(idx)], atol=1e-13 * np.abs(v).max())


@pytest.mark.parametrize("shape", [(2, 2), (2, 3)])
def test_high_temperature_energy_tracks_exact(shape):
    # at beta_obs = 4t <= 0.8 the SU state's energy (all configurations enumerated, Eq. 11)
    # is within 1e-3 per site of exact diagonalisation; the error grows with beta (the
    # environment of a bond is replaced by weights), which is why SR takes over later
    lat = Lattice(*shape, 4)
    Hd = ed.doubled_hamiltonian(lat)
    spec = ed.spectrum(lat)
    errs = []
    for t in (0.05, 0.2, 0.4):
        v = _vec(lat, _evolved(lat, t, 0.01, 4))
        e = v @ Hd @ v / (2 * (v @ v)) / lat.N
        errs.append(abs(e - ed.thermal(spec, lat.N, [4 * t])[0][0]))
    assert errs[0] < 1e-5 and errs[1] < 1e-3
    assert errs[0] < errs[1] < errs[2]


def test_swap_gate_exchanges_local_states():
    G = su.swap_gate()
    v = np.random.default_rng(3).standard_normal((4, 4))    # amplitudes over (S_i, S_j)
    assert np.array_equal((G @ v.reshape(-1)).reshape(4, 4), v.T)
    assert np.array_equal(G @ G, np.eye(16))


def test_next_nearest_neighbour_bonds_converge_to_exact():
    # J2 bonds routed through a plaquette site with exchange gates: with bonds large enough
    # for the exchanges (D = 32 on 2x2) the SU state tracks ED like the J1-only one; at D = 4
    # the exchanges are truncated and the error is three orders larger
    errs = {}
    for D in (4, 32):
        lat = Lattice(2, 2, D, J1=1.0, J2=0.5)
        Hd = ed.doubled_hamiltonian(lat)
        v = _vec(lat, _evolved(lat, 0.05, 0.01, D))
        e = v @ Hd @ v / (2 * (v @ v)) / lat.N
        errs[D] = abs(e - ed.thermal(ed.spectrum(lat), lat.N, [0.2])[0][0])
    assert errs[32] < 1e-6 and errs[4] > 1e-4
