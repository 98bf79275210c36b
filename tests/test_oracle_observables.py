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
