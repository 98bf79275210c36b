"""Pins of the oracle's PEPS contraction, amplitudes, E_loc (Eq. 9) and O_k (Eq. 8)."""
import string

import numpy as np
import pytest

from oracle import ed, peps, sr
from oracle.lattice import Lattice


def brute_force_amplitude(lat, theta, S):
    """Eq. 4 written out: one einsum over the whole network, a letter per leg."""
    T = lat.tensors(theta)
    letters = iter(string.ascii_letters)
    legs = {}
    subs, ops = [], []
    for r in range(lat.nrow):
        for c in range(lat.ncol):
            i = lat.site(r, c)
            names = []
            for key in [('h', r, c - 1), ('h', r, c), ('v', r - 1, c), ('v', r, c)]:
                inside = (key[0] == 'h' and 0 <= key[2] < lat.ncol - 1) or \
                         (key[0] == 'v' and 0 <= key[1] < lat.nrow - 1)
                if inside:
                    if key not in legs:
                        legs[key] = next(letters)
                    names.append(legs[key])
                else:
                    names.append(next(letters))
            subs.append(''.join(names))
            ops.append(T[i][int(S[i])])
    return float(np.einsum(','.join(subs) + '->', *ops, optimize='greedy'))


@pytest.mark.parametrize("shape,D", [((2, 2), 3), ((2, 3), 2), ((3, 3), 2)])
def test_row_vector_contraction_is_brute_force(shape, D):
    rng = np.random.default_rng(1)
    lat = Lattice(*shape, D)
    th = rng.standard_normal(lat.Np)
    for _ in range(4):
        S = rng.integers(0, 4, lat.N)
        assert peps.amplitude_exact(lat, th, S) == pytest.approx(brute_force_amplitude(lat, th, S),
                                                                 rel=1e-12)


@pytest.mark.parametrize("shape,D,chi", [((3, 3), 2, 4), ((4, 4), 2, 4), ((4, 3), 3, 9)])
def test_boundary_mps_exact_chi(shape, D, chi):
    # chi >= D^floor(ncol/2) is exact: boundary MPS equals the exact contraction, and every
    # row strip gives the same amplitude.
    rng = np.random.default_rng(2)
    lat = Lattice(*shape, D)
    th = rng.standard_normal(lat.Np)
    for _ in range(3):
        S = rng.integers(0, 4, lat.N)
        a = peps.amplitude_exact(lat, th, S)
        r = peps.eval_sample(lat, th, S, chi, with_O=False)
        assert r['sign'] == np.sign(a)
        assert r['log_abs'] == pytest.approx(np.log(abs(a)), abs=1e-11)
        rows = peps.row_amplitudes(lat, th, S, chi)
        assert np.allclose(rows, np.log(abs(a)), atol=1e-11)


def test_truncated_chi_converges():
    rng = np.random.default_rng(3)
    lat = Lattice(4, 4, 3)
    th = rng.standard_normal(lat.Np)
    S = rng.integers(0, 4, lat.N)
    a = peps.amplitude_exact(lat, th, S)
    errs = []
    for chi in [3, 6, 9]:
        r = peps.eval_sample(lat, th, S, chi, with_O=False)
        errs.append(abs(r['sign'] * np.exp(r['log_abs']) - a) / abs(a))
    assert errs[2] < 1e-12 and errs[1] < errs[0]


def _mps_vector(mps):
    v = np.ones((1, 1))
    for t in mps:
        v = np.einsum('xa,apb->xpb', v, t).reshape(-1, t.shape[2])
    return v.reshape(-1)


def test_compress_single_bond_is_eckart_young():
    # Only the middle bond exceeds chi, so SVD truncation in canonical form must give the
    # best rank-chi approximation of the state across that cut.
    rng = np.random.default_rng(4)
    mps = [rng.standard_normal(s) for s in [(1, 3, 3), (3, 3, 6), (6, 3, 3), (3, 3, 1)]]
    psi = _mps_vector(mps)
    got = _mps_vector(peps.compress(mps, 4))
    U, s, Vt = np.linalg.svd(psi.reshape(9, 9))
    best = (U[:, :4] * s[:4]) @ Vt[:4]
    assert np.allclose(got, best.reshape(-1), atol=1e-12 * np.abs(psi).max())


def test_compress_is_gauge_invariant():
    # Inserting X X^-1 on a bond changes no state, so the compressed state must not change.
    rng = np.random.default_rng(5)
    mps = [rng.standard_normal(s) for s in [(1, 2, 4), (4, 2, 8), (8, 2, 4), (4, 2, 2), (2, 2, 1)]]
    X = rng.standard_normal((8, 8)) + 4 * np.eye(8)
    g = [mps[0], np.einsum('apb,bc->apc', mps[1], X),
         np.einsum('cb,bpd->cpd', np.linalg.inv(X), mps[2]), mps[3], mps[4]]
    assert np.allclose(_mps_vector(peps.compress(mps, 3)), _mps_vector(peps.compress(g, 3)),
                       atol=1e-10)


def test_beta0_state_invariants():
    # noise 0: rho(S) = prod_i delta(s_i, s'_i) exactly (Eq. 1 at beta = 0, Eq. 2).
    lat = Lattice(3, 3, 2)
    th = peps.init_theta(lat, seed=1, noise=0.0)
    rng = np.random.default_rng(6)
    for _ in range(6):
        S = rng.integers(0, 4, lat.N)
        diag = np.all(S // 2 == S % 2)
        assert peps.amplitude_exact(lat, th, S) == (1.0 if diag else 0.0)
    # E_loc = sum_b J S^z_i S^z_j on diagonal S (off-diagonal neighbours have rho = 0);
    # averaged over the uniform diagonal ensemble this gives E = Tr H / 2^N = 0.
    lat = Lattice(2, 2, 2, J1=1.0, J2=0.5)
    th = peps.init_theta(lat, seed=1, noise=0.0)
    tot = 0.0
    for x in range(16):
        s = np.array([(x >> k) & 1 for k in range(4)])
        r = peps.eval_sample(lat, th, 3 * s, 4, with_O=False)
        tot += r['e_sys'] + r['e_anc']
    assert abs(tot / 16) < 1e-14


def test_init_theta_layout_and_noise():
    lat = Lattice(3, 4, 3)
    a = 1e-3
    th = peps.init_theta(lat, seed=11, noise=a)
    assert th.size == lat.Np
    for i in range(lat.N):
        T = lat.tensors(th)[i]
        z = (0,) * 4
        assert T[(0,) + z] == 1.0 and T[(3,) + z] == 1.0
        rest = T.copy()
        rest[(0,) + z] = rest[(3,) + z] = 0.0
        assert np.max(np.abs(rest)) <= a
    assert np.count_nonzero(th) == lat.Np
    assert lat.Np == 4 * sum(lat.sz)


def test_local_energy_matches_doubled_hamiltonian():
    # <rho|calH|rho>/<rho|rho> = sum_S |rho(S)|^2 E_loc(S) / sum_S |rho(S)|^2 (Eq. 9), with
    # calH = H x I + I x H^T built explicitly (Eq. 3), on all 256 configurations of 2x2.
    rng = np.random.default_rng(7)
    lat = Lattice(2, 2, 2, J1=1.0, J2=0.6)
    th = rng.standard_normal(lat.Np)
    Hd = ed.doubled_hamiltonian(lat)
    vec = np.array([peps.amplitude_exact(lat, th, ed.config_of_index(k, 4)) for k in range(256)])
    num = den = 0.0
    for k in range(256):
        r = peps.eval_sample(lat, th, ed.config_of_index(k, 4), 4, with_O=False)
        num += vec[k] ** 2 * (r['e_sys'] + r['e_anc'])
        den += vec[k] ** 2
    assert num / den == pytest.approx(vec @ Hd @ vec / (vec @ vec), rel=1e-12)


def test_local_energy_pointwise_3x3():
    # Pointwise: E_loc(S) = (calH rho)(S) / rho(S) on a 3x3 lattice (4^9 states; the
    # action of calH is applied to the amplitudes of the neighbours of S only).
    rng = np.random.default_rng(8)
    lat = Lattice(3, 3, 2, J1=1.0, J2=0.5)
    th = rng.standard_normal(lat.Np)
    for _ in range(3):
        S = rng.integers(0, 4, lat.N)
        rho = peps.amplitude_exact(lat, th, S)
        tot = 0.0
        for (i, j, J, _) in lat.bonds():
            for layer in (lambda x: x // 2, lambda x: x % 2):
                si, sj = layer(S[i]), layer(S[j])
                tot += J * (0.5 - si) * (0.5 - sj)
                if si != sj:
                    Sp = S.copy()
                    if layer(1) == 0:     # system layer (x // 2)
                        Sp[i], Sp[j] = 2 * sj + S[i] % 2, 2 * si + S[j] % 2
                    else:
                        Sp[i], Sp[j] = 2 * (S[i] // 2) + sj, 2 * (S[j] // 2) + si
                    tot += 0.5 * J * peps.amplitude_exact(lat, th, Sp) / rho
        r = peps.eval_sample(lat, th, S, 8, with_O=False)
        assert r['e_sys'] + r['e_anc'] == pytest.approx(tot, rel=1e-11, abs=1e-11)


def test_log_derivatives_finite_difference():
    rng = np.random.default_rng(9)
    lat = Lattice(3, 3, 2)
    th = rng.standard_normal(lat.Np)
    S = rng.integers(0, 4, lat.N)
    r = peps.eval_sample(lat, th, S, 8)
    Of = sr.expand_O(lat, S[None, :], r['O'][None, :])[0]
    h = 1e-6
    for k in rng.choice(lat.Np, 40, replace=False):
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (np.log(abs(peps.amplitude_exact(lat, tp, S)))
              - np.log(abs(peps.amplitude_exact(lat, tm, S)))) / (2 * h)
        assert Of[k] == pytest.approx(fd, abs=1e-8)


def test_log_derivatives_euler_identity():
    # rho is linear in each T_i, so sum_k O_{i,k} T_i^{S_i}[k] = 1 for every site, also at
    # truncated chi (the one-row strip value is linear in each tensor of the row).
    rng = np.random.default_rng(10)
    lat = Lattice(4, 4, 3)
    th = rng.standard_normal(lat.Np)
    S = rng.integers(0, 4, lat.N)
    r = peps.eval_sample(lat, th, S, 4)
    T = lat.tensors(th)
    for i in range(lat.N):
        o = r['O'][lat.o_off[i]:lat.o_off[i + 1]]
        assert float(o @ T[i][S[i]].ravel()) == pytest.approx(1.0, abs=1e-10)
