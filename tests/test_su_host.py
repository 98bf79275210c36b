"""The library's simple-update warm start (peps_su_theta, host-side, App. A) against the
oracle's simple update (tests/test_oracle_simple_update.py pins that one to ED): the same
state, compared through gauge-invariant amplitudes, wherever the truncation cuts between
distinct singular values (D = 4 here: the bond spectra are a singlet and a triplet)."""
import numpy as np
import pytest

from oracle import ed, peps, simple_update as su
from oracle.lattice import Lattice
from paper_2409_05285_gb300 import binding


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2409_05285_gb300.build import build
    build()


def test_coupling_enters_the_gate():
    lat = Lattice(2, 3, 4, J1=0.7)
    th = binding.su_theta(2, 3, 4, 0.7, 0.03, 6)
    tho = _oracle_theta(lat, 0.03, 6)
    cfgs = [ed.config_of_index(k, lat.N) for k in range(4 ** lat.N)]
    v = np.array([peps.amplitude_exact(lat, th, S) for S in cfgs])
    w = np.array([peps.amplitude_exact(lat, tho, S) for S in cfgs])
    assert np.allclose(_unit(v), _unit(w), atol=1e-12)
    th1 = binding.su_theta(2, 3, 4, 1.0, 0.03, 6)
    v1 = np.array([peps.amplitude_exact(lat, th1, S) for S in cfgs])
    assert np.max(np.abs(_unit(v1) - _unit(v))) > 1e-4


def _oracle_theta(lat, tau, n):
    st = su.SUState(lat)
    for _ in range(n):
        su.su_step(st, tau, lat.D)
    return su.to_theta(st)


def _unit(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("shape,n", [((2, 2), 10), ((2, 3), 12), ((3, 2), 7)])
def test_matches_oracle_on_every_configuration(shape, n):
    lat = Lattice(*shape, 4)
    th = binding.su_theta(lat.nrow, lat.ncol, 4, 1.0, 0.02, n)
    tho = _oracle_theta(lat, 0.02, n)
    cfgs = [ed.config_of_index(k, lat.N) for k in range(4 ** lat.N)]
    v = np.array([peps.amplitude_exact(lat, th, S) for S in cfgs])
    w = np.array([peps.amplitude_exact(lat, tho, S) for S in cfgs])
    assert np.allclose(_unit(v), _unit(w), atol=1e-12)


def test_matches_oracle_3x3_sampled():
    lat = Lattice(3, 3, 4)
    th = binding.su_theta(3, 3, 4, 1.0, 0.01, 6)
    tho = _oracle_theta(lat, 0.01, 6)
    rng = np.random.default_rng(5)
    S = rng.integers(0, 4, (200, lat.N))
    S[:50] = 3 * rng.integers(0, 2, (50, lat.N))
    v = np.array([peps.amplitude_exact(lat, th, s) for s in S])
    w = np.array([peps.amplitude_exact(lat, tho, s) for s in S])
    k = np.argmax(np.abs(w))
    assert np.allclose(v / v[k], w / w[k], atol=1e-11)


def test_zero_steps_is_the_beta0_state():
    lat = Lattice(3, 4, 3)
    assert np.array_equal(binding.su_theta(3, 4, 3, 1.0, 0.05, 0), peps.init_theta(lat, 0, 0.0))


def test_energy_tracks_exact_at_high_temperature():
    lat = Lattice(2, 3, 4)
    Hd = ed.doubled_hamiltonian(lat)
    t = 0.1
    th = binding.su_theta(2, 3, 4, 1.0, 0.01, 10)
    v = np.array([peps.amplitude_exact(lat, th, ed.config_of_index(k, lat.N))
                  for k in range(4 ** lat.N)])
    e = v @ Hd @ v / (2 * (v @ v)) / lat.N
    assert e == pytest.approx(ed.thermal(ed.spectrum(lat), lat.N, [4 * t])[0][0], abs=1e-4)


def test_rejects_bad_arguments():
    lib = binding.load()
    buf = np.zeros(16)
    ptr = buf.ctypes.data_as(binding.ctypes.POINTER(binding.ctypes.c_double))
    assert lib.peps_su_theta(2, 2, 1, 1.0, 0.01, 1, ptr, 16) == binding.PEPS_OK
    assert lib.peps_su_theta(2, 2, 1, 1.0, 0.01, 1, ptr, 15) == binding.PEPS_EINVAL
    assert lib.peps_su_theta(1, 2, 1, 1.0, 0.01, 1, ptr, 8) == binding.PEPS_EINVAL
    assert lib.peps_su_theta(2, 2, 1, 1.0, -0.01, 1, ptr, 16) == binding.PEPS_EINVAL
    assert lib.peps_su_theta(2, 2, 1, 1.0, 0.01, -1, ptr, 16) == binding.PEPS_EINVAL
