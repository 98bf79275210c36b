"""Pins of the oracle's exact diagonalisation (Eq. 12) and of the vectorised evolution
(Eqs. 1-3, 11) against closed forms."""
import numpy as np
import pytest

from oracle import ed
from oracle.lattice import Lattice


def test_two_site_closed_form():
    # One bond: singlet -3/4 J (1 state), triplet +1/4 J (3 states).
    lat = Lattice(1, 2, 1, J1=1.0)
    betas = np.array([0.1, 0.5, 1.0, 3.0, 10.0])
    got = ed.thermal(ed.spectrum(lat), lat.N, betas)
    for b, (e, c, x) in zip(betas, got):
        z = np.exp(0.75 * b) + 3 * np.exp(-0.25 * b)
        E = (-0.75 * np.exp(0.75 * b) + 0.75 * np.exp(-0.25 * b)) / z
        E2 = (0.5625 * np.exp(0.75 * b) + 3 * 0.0625 * np.exp(-0.25 * b)) / z
        M2 = 2 * np.exp(-0.25 * b) / z            # triplet m = +-1
        assert e == pytest.approx(E / 2, abs=1e-13)
        assert c == pytest.approx(b * b * (E2 - E * E) / 2, abs=1e-12)
        assert x == pytest.approx(b * M2 / 2, abs=1e-13)


def test_four_site_ring_spectrum():
    # 2x2 open lattice = 4-site ring: H = J/2 [S_tot^2 - S_A^2 - S_B^2] with the two
    # diagonal pairs A, B -> eigenvalues -2 (x1), -1 (x3), 0 (x7), +1 (x5).
    lat = Lattice(2, 2, 1)
    ev = np.sort(np.concatenate([e for _, e in ed.spectrum(lat)]))
    expect = np.array([-2] + [-1] * 3 + [0] * 7 + [1] * 5, dtype=float)
    assert np.allclose(ev, expect, atol=1e-12)


def test_free_spins():
    lat = Lattice(2, 3, 1, J1=0.0)
    got = ed.thermal(ed.spectrum(lat), lat.N, [0.3, 2.0])
    for b, (e, c, x) in zip([0.3, 2.0], got):
        assert abs(e) < 1e-14 and abs(c) < 1e-13
        assert x == pytest.approx(b / 4, rel=1e-13)   # Curie law, <Mz^2> = N/4


def test_high_temperature_expansion():
    # <H> = -beta Tr(H^2)/2^N + O(beta^2), Tr(H^2)/2^N = (3/16) sum_b J_b^2 (Tr H = 0).
    lat = Lattice(3, 3, 1, J1=1.0, J2=0.5)
    b = 1e-4
    e, _, x = ed.thermal(ed.spectrum(lat), lat.N, [b])[0]
    sJ2 = sum(J * J for (_, _, J, _) in lat.bonds())
    assert e * lat.N == pytest.approx(-b * 3 / 16 * sJ2, rel=1e-3)
    assert x / b == pytest.approx(0.25, rel=1e-3)


def test_sector_blocks_match_full():
    lat = Lattice(2, 3, 1, J1=1.0, J2=0.7)
    H = ed.full_hamiltonian(lat)
    assert np.allclose(H, H.T)
    ev_full = np.linalg.eigvalsh(H)
    ev_sec = np.sort(np.concatenate([e for _, e in ed.spectrum(lat)]))
    assert np.allclose(ev_full, ev_sec, atol=1e-12)


def test_vectorised_evolution_is_thermal_at_4t():
    # |rho(t)> = exp(-t calH)|I> (Eq. 3) has <rho|calH|rho>/(2<rho|rho>) equal to the
    # thermal energy at inverse temperature 4t (Eq. 11 with beta = 2t).
    lat = Lattice(2, 2, 1, J1=1.0, J2=0.4)
    Hd = ed.doubled_hamiltonian(lat)
    spec = ed.spectrum(lat)
    for t in [0.0, 0.1, 0.5, 1.0]:
        v = ed.evolve_identity(lat, t)
        e = v @ Hd @ v / (2 * (v @ v))
        assert e / lat.N == pytest.approx(ed.thermal(spec, lat.N, [4 * t])[0][0], abs=1e-12)


def test_doubled_hamiltonian_on_identity():
    # calH |I> = vec(H + H^T) = 2 vec(H); <I|calH|I> = 2 Tr H = 0.
    lat = Lattice(2, 2, 1)
    Hd = ed.doubled_hamiltonian(lat)
    I = ed.evolve_identity(lat, 0.0)
    H = ed.full_hamiltonian(lat)
    perm = ed.pair_to_config_index(lat.N)
    assert np.allclose(Hd @ I, 2 * H.reshape(-1)[perm])
    assert abs(I @ Hd @ I) < 1e-12
