"""Pins of the oracle's Metropolis sampler against the exact distribution |rho|^p on 2x2
(all 256 configurations enumerated), for p = 2 (Sec. II) and p = 1 with the reweighting
of Eq. A1.

The moves (both-flips, system-only and ancilla-only exchanges) keep M_z(s) - M_z(s') even;
the thermal state (Eq. 1) has rho(S) = 0 unless M_z(s) = M_z(s') because [H, M_z] = 0, so
chains started on the diagonal sample |rho|^p restricted to that class.  With random
tensors the target here is restricted the same way."""
import numpy as np
import pytest
from scipy import stats

from oracle import ed, peps, sampler, sr
from oracle.lattice import Lattice


def _exact(lat, th):
    """All configurations and their amplitudes, zeroed outside the reachable class."""
    cfgs = np.array([ed.config_of_index(k, lat.N) for k in range(4 ** lat.N)])
    amp = np.array([peps.amplitude_exact(lat, th, S) for S in cfgs])
    reach = (np.sum(cfgs // 2, axis=1) - np.sum(cfgs % 2, axis=1)) % 2 == 0
    return cfgs, np.where(reach, amp, 0.0)


def _index(S):
    k = 0
    for x in S:
        k = 4 * k + int(x)
    return k


@pytest.mark.parametrize("p", [2, 1])
def test_histogram_matches_exact(p):
    lat = Lattice(2, 2, 2, J1=1.0)
    rng = np.random.default_rng(21)
    th = rng.standard_normal(lat.Np)
    cfgs, amp = _exact(lat, th)
    target = np.abs(amp) ** p
    target /= target.sum()
    n_chains, n_sweeps = 600, 8
    S0 = peps.init_configs(lat, 5, n_chains)
    S, acc, prop = sampler.run_chains(lat, th, S0, 4, p, 5, 0, n_sweeps)
    counts = np.bincount([_index(s) for s in S], minlength=256)
    expect = target * n_chains
    big = expect >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(expect[big], expect[~big].sum())
    chi2 = np.sum((obs - exp) ** 2 / exp)
    pval = stats.chi2.sf(chi2, len(obs) - 1)
    assert pval > 1e-4, (chi2, len(obs))
    assert 0 < acc < prop


def test_reweighted_energy_estimate():
    # Eq. A1: sampling p1 = |rho| and weighting by r1 = |rho| estimates <E_loc> under
    # p0 = |rho|^2.
    lat = Lattice(2, 2, 2, J1=1.0, J2=0.3)
    rng = np.random.default_rng(22)
    th = rng.standard_normal(lat.Np)
    cfgs, amp = _exact(lat, th)
    e_all = np.array([sum(peps.eval_sample(lat, th, S, 4, with_O=False)[k] for k in ('e_sys', 'e_anc'))
                      for S in cfgs])
    exact = np.sum(amp ** 2 * e_all) / np.sum(amp ** 2)
    S0 = peps.init_configs(lat, 9, 800)
    S, _, _ = sampler.run_chains(lat, th, S0, 4, 1, 9, 0, 8)
    idx = np.array([_index(s) for s in S])
    assert np.all(amp[idx] != 0.0)
    w = sr.weights(np.log(np.abs(amp[idx])), p=1)
    est = float(w @ e_all[idx])
    # spread of the weighted estimator from the exact p1 distribution
    p1 = np.abs(amp) / np.abs(amp).sum()
    var = np.sum(p1 * np.abs(amp) ** 2 * (e_all - exact) ** 2) / np.sum(p1 * np.abs(amp)) ** 2
    assert abs(est - exact) < 5 * np.sqrt(var / len(idx))


def test_detailed_balance_of_one_move():
    # A single proposal S -> S' accepted with min(1, |rho'/rho|^p) satisfies detailed balance.
    for p in (1, 2):
        for ratio in (0.3, 1.0, 2.5, -0.7):
            a_fwd = min(1.0, abs(ratio) ** p)
            a_bwd = min(1.0, abs(1.0 / ratio) ** p)
            assert 1.0 * a_fwd == pytest.approx(abs(ratio) ** p * a_bwd)
            u = np.linspace(0, 1, 100001)[:-1]
            assert np.mean([sampler.accept(x, ratio, p) for x in u[::97]]) == pytest.approx(a_fwd, abs=2e-3)


def test_sweep_is_deterministic_given_seed():
    lat = Lattice(3, 3, 2)
    th = peps.init_theta(lat, 4, 1e-2)
    S0 = peps.init_configs(lat, 4, 3)
    a = sampler.run_chains(lat, th, S0, 4, 2, 4, 10, 2)[0]
    b = sampler.run_chains(lat, th, S0, 4, 2, 4, 10, 2)[0]
    c = sampler.run_chains(lat, th, S0, 4, 2, 5, 10, 2)[0]
    assert np.array_equal(a, b)
    assert a.shape == c.shape
