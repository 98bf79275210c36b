"""Pins of the fermionic sampler and SR step of the oracle (Sec. II MCMC and Eqs. 5-10 on the
fermionic PEPS of Fig. 1b): the move set against parity, symmetry and the support of the
exact thermal state; the sweep's exact transition matrix against |psi|^p; the sweep function
against that matrix; the estimators at infinite temperature in closed form; the SR dynamics
against exact imaginary-time evolution of the Hubbard dimer."""
from collections import deque

import numpy as np
import pytest

from oracle import fermion as fm
from oracle import fermion_vmc as fv
from oracle import philox
from oracle import sr


def _parity(S):
    return sum(bin(int(x)).count("1") for x in S) & 1


def _numbers(S):
    # (N_up(c), N_dn(c), N_up(d), N_dn(d))
    return tuple(sum((int(x) >> k) & 1 for x in S) for k in range(4))


def test_moves_are_even_involutions():
    nr, nc = 2, 3
    mv = fv.moves(nr, nc)
    assert len(mv) == 2 * nr * nc + 4 * len(fm.fpeps_bonds(nr, nc))
    rng = np.random.default_rng(0)
    for _ in range(50):
        S = [int(x) for x in rng.integers(0, 16, nr * nc)]
        for m in mv:
            S2 = fv.propose(S, m)
            if S2 is None:
                if m[0] == "hop":
                    assert ((S[m[1]] >> m[3]) & 1) == ((S[m[2]] >> m[3]) & 1)
                else:
                    assert ((S[m[1]] >> m[2]) & 1) != ((S[m[1]] >> (2 + m[2])) & 1)
                continue
            assert S2 != S and _parity(S2) == _parity(S)
            assert fv.propose(S2, m) == S
            n0, n1 = _numbers(S), _numbers(S2)
            if m[0] == "hop":
                assert n0 == n1
            else:
                s = m[2]
                assert n1[s] - n0[s] == n1[2 + s] - n0[2 + s] != 0
                assert n1[1 - s] == n0[1 - s] and n1[3 - s] == n0[3 - s]


def test_moves_connect_exactly_the_thermal_support():
    # from the empty lattice the moves reach every configuration with N_s(c) = N_s(d), and
    # that set holds the support of exp(-t calH)|I> (2x2)
    nr, nc = 2, 2
    N = nr * nc
    seen = {(0,) * N}
    todo = deque(seen)
    mv = fv.moves(nr, nc)
    while todo:
        S = todo.popleft()
        for m in mv:
            S2 = fv.propose(S, m)
            if S2 is not None and tuple(S2) not in seen:
                seen.add(tuple(S2))
                todo.append(tuple(S2))
    target = set()
    for st in range(1 << (4 * N)):
        S = tuple(fm.local_indices(st, N))
        n = _numbers(S)
        if n[0] == n[2] and n[1] == n[3]:
            target.add(S)
    assert seen == target
    assert len(target) == sum(__import__("math").comb(N, k) ** 2 for k in range(N + 1)) ** 2
    vec = fm.evolve(nr, nc, 1.0, 8.0, 4.0, 0.1)
    support = {tuple(fm.local_indices(int(st), N)) for st in np.nonzero(np.abs(vec) > 1e-14)[0]}
    assert support <= target
    assert len(support) > 0.9 * len(target)


@pytest.mark.parametrize("p", [1, 2])
def test_sweep_matrix_keeps_psi_to_the_p(p):
    # Metropolis with symmetric proposals: |psi|^p is stationary under every single move,
    # hence under the sweep; rows are stochastic (1x2, random even PEPS, all 128 even states)
    rng = np.random.default_rng(7)
    T = fm.random_even_fpeps(1, 2, 2, rng)
    psi = fm.fpeps_state(1, 2, T)
    states = [fm.local_indices(s, 2) for s in range(256) if bin(s).count("1") % 2 == 0]
    psi_of = lambda S: psi[fm.state_of(S)]
    P = fv.transition_matrix(1, 2, psi_of, states, p)
    pi = np.array([abs(psi_of(S)) ** p for S in states])
    pi /= pi.sum()
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-13)
    assert np.max(np.abs(pi @ P - pi)) < 1e-13
    assert np.count_nonzero(P > 1e-12) > 4 * len(states)     # the sweep does move


def test_sweep_function_draws_from_the_matrix():
    # from a fixed configuration, 20000 pairs of sweeps with independent uniforms: the
    # histogram of the final configurations against the exact row of the square of the
    # sweep's transition matrix
    rng = np.random.default_rng(11)
    T = fm.random_even_fpeps(1, 2, 2, rng)
    psi = fm.fpeps_state(1, 2, T)
    states = [fm.local_indices(s, 2) for s in range(256) if bin(s).count("1") % 2 == 0]
    psi_of = lambda S: psi[fm.state_of(S)]
    P = fv.transition_matrix(1, 2, psi_of, states, 2)
    index = {tuple(S): n for n, S in enumerate(states)}
    S0 = [5, 0]
    row = (P @ P)[index[tuple(S0)]]
    n_moves = len(fv.moves(1, 2))
    U = np.random.default_rng(12).random((20000, 2, n_moves))
    counts = np.zeros(len(states))
    for u in U:
        S, _, _ = fv.sweep(1, 2, T, S0, 2, u[0], amplitude=psi_of)
        S, _, _ = fv.sweep(1, 2, T, S, 2, u[1], amplitude=psi_of)
        counts[index[tuple(int(x) for x in S)]] += 1
    exp = row * len(U)
    big = exp >= 5
    chi2 = np.sum((counts[big] - exp[big]) ** 2 / exp[big])
    dof = int(big.sum()) - 1
    assert dof >= 10
    assert chi2 < dof + 5 * np.sqrt(2 * dof)
    assert counts[~big].sum() <= max(30, 3 * exp[~big].sum())


def test_sweep_special_uniforms():
    # u -> 0 accepts every proposal with psi' != 0; u -> 1 only those with |psi'| > |psi|
    rng = np.random.default_rng(3)
    T = fm.random_even_fpeps(2, 2, 2, rng)
    S0 = [1 | 4, 0, 2 | 8, 3 | 12]
    n = len(fv.moves(2, 2))
    S, acc, _ = fv.sweep(2, 2, T, S0, 2, np.full(n, 1e-300))
    # replay: every non-skipped proposal taken
    X = list(S0)
    taken = 0
    for m in fv.moves(2, 2):
        X2 = fv.propose(X, m)
        if X2 is not None and fm.fpeps_amplitude_bosonic(2, 2, T, X2) != 0.0:
            X = X2
            taken += 1
    assert acc == taken and list(S) == X
    S, acc, _ = fv.sweep(2, 2, T, S0, 2, np.full(n, 1.0 - 2.0 ** -53))
    a0 = abs(fm.fpeps_amplitude_bosonic(2, 2, T, S0))
    a1 = abs(fm.fpeps_amplitude_bosonic(2, 2, T, S))
    assert (acc == 0 and list(S) == S0) or a1 > a0


def test_uniform_stream_layout():
    u = fv.uniforms(99, 5, 7, 24)
    assert u.shape == (24,) and np.all((u >= 0) & (u < 1))
    assert u[3] == philox.uniform(99, 5, 7, 3, fv.TAG_FMC)
    assert len(set(np.round(u, 15))) == 24
    assert not np.array_equal(u, fv.uniforms(99, 6, 7, 24))


def test_estimators_at_infinite_temperature():
    # |I> (beta = 0): every configuration of its support has |psi| = 1 and E_sys = E_anc =
    # sum_i (U n_up n_dn - mu n) (no hop stays in the support), so with uniform weights over
    # the support E/N = U/4 - mu, double occupancy 1/4, density 1 (closed forms)
    nr, nc, U, mu = 2, 2, 8.0, 3.0
    T = fm.identity_fpeps(nr, nc)
    S_batch = [[a | (a << 2) for a in idx] for idx in np.ndindex(4, 4, 4, 4)]
    la, sg, es, ea, rows = fv.sample_quantities(nr, nc, T, S_batch, 1.0, U, mu)
    assert np.allclose(la, 0.0) and np.allclose(es, ea)
    w = sr.weights(la, 2)
    obs = fv.observables(nr * nc, S_batch, w, es, ea)
    assert obs["E_site"] == pytest.approx(U / 4 - mu, abs=1e-12)
    assert obs["docc"] == pytest.approx(0.25, abs=1e-12)
    assert obs["density"] == pytest.approx(1.0, abs=1e-12)


def test_expand_O_places_each_site_at_its_slice():
    rng = np.random.default_rng(4)
    T = fm.random_even_fpeps(2, 2, 2, rng)
    off, sz = fv.theta_offsets(T)
    S_batch = [[1, 5, 9, 12], [0, 3, 6, 15]]
    rows = rng.standard_normal((2, sum(sz)))
    Of = fv.expand_O(T, S_batch, rows)
    assert Of.shape == (2, off[-1]) and np.count_nonzero(Of) == rows.size
    o = 0
    for j in range(4):
        for n in range(2):
            a = off[j] + S_batch[n][j] * sz[j]
            assert np.array_equal(Of[n, a:a + sz[j]], rows[n, o:o + sz[j]])
        o += sz[j]
    assert np.array_equal(fv.unflatten(fv.flatten(T), T)[3], T[3])


def _padded_identity(D, noise, rng):
    # |I> on 1x2 in the first virtual slot of bond dimension D, uniform noise on the other
    # parity-even entries
    T = []
    for c in range(2):
        A = np.zeros((16, 1 if c == 0 else D, D if c == 0 else 1, 1, 1))
        for idx in np.ndindex(*A.shape):
            if (fm._pS(idx[0]) + sum(fm._pv(x) for x in idx[1:])) & 1 == 0:
                A[idx] = rng.uniform(-noise, noise)
        for a in range(4):
            A[(a | (a << 2), 0, 0, 0, 0)] = -1.0 if a == 3 else 1.0
        T.append(A)
    return T


def _dimer_run(tau, t_end, U=2.0, mu=1.0, t_hop=1.0, eps=1e-4):
    """Deterministic SR on the 1x2 Hubbard dimer with every even configuration enumerated
    (weights |psi|^2), D = 16 (eight even and eight odd virtual states: exact for two sites);
    returns E/site - E_exact(t) at the end."""
    T = _padded_identity(16, 1e-3, np.random.default_rng(3))
    cfgs = [fm.local_indices(s, 2) for s in range(256) if bin(s).count("1") % 2 == 0]
    n = int(round(t_end / tau))
    for step in range(n + 1):
        use = [S for S in cfgs if fm.fpeps_amplitude_bosonic(1, 2, T, S) != 0.0]
        lq = np.zeros(len(use))
        if step == n:
            la, _, es, ea, _ = fv.sample_quantities(1, 2, T, use, t_hop, U, mu)
            obs = fv.observables(2, use, sr.weights(la, 0, lq), es, ea)
            E, _ = fm.observables(1, 2, t_hop, U, mu, fm.evolve(1, 2, t_hop, U, mu, n * tau))
            return obs["E_site"] - E
        T, *_ = fv.sr_step(1, 2, T, use, t_hop, U, mu, 0, tau, eps, 1e-10, 1000, log_q=lq)


def test_sr_dynamics_follow_exact_evolution_of_the_dimer():
    # theta' = theta - tau G^-1 g approximates exp(-tau calH) (Eq. 5) for fermions too: against
    # the energy of exp(-t calH)|I> the error is first order in tau
    e2 = _dimer_run(0.02, 0.12)
    e1 = _dimer_run(0.01, 0.12)
    assert abs(e1) < 0.6 * abs(e2)
    assert abs(e2) < 0.06 and abs(e1) < 0.03


def test_vertical_hop_flips_reduce_to_one_right_leg_parity():
    # a vertical hop at column c flips the row-prefix bit b of every site right of c in both
    # rows; the plain contraction of the signed slices then equals the one with the old bits
    # and a parity operator on the right leg of the lower hop site, times the sign of the
    # lower row's physical parities right of c (the property a cached-strip sweep relies on)
    rng = np.random.default_rng(5)
    L1, L2, D = 3, 4, 2
    T = fm.random_even_fpeps(L1, L2, D, rng)
    Ts = fm.fpeps_signed_slices(T)

    def plain(S32, twist=None):
        t = []
        for i in range(L1 * L2):
            A = Ts[i][S32[i]].copy()
            if i == twist:
                A[:, 1::2, :, :] *= -1.0          # parity of the right leg (odd indices)
            t.append(A)
        return fm.plain_amplitude(L1, L2, t)

    n = 0
    while n < 40:
        S = [int(x) for x in rng.integers(0, 16, L1 * L2)]
        if sum(bin(x).count("1") for x in S) % 2:
            S[0] ^= 1
        r, c, k = int(rng.integers(0, L1 - 1)), int(rng.integers(0, L2)), int(rng.integers(0, 4))
        i, j = r * L2 + c, (r + 1) * L2 + c
        S2 = fv.propose(S, ("hop", i, j, k))
        if S2 is None:
            continue
        b_new = fm.fpeps_row_prefix_bits(L1, L2, S2)
        b_old = fm.fpeps_row_prefix_bits(L1, L2, S)
        true = plain([S2[q] + 16 * b_new[q] for q in range(L1 * L2)])
        alt = plain([S2[q] + 16 * b_old[q] for q in range(L1 * L2)], twist=j if c + 1 < L2 else None)
        sgn = (-1) ** sum(bin(S2[(r + 1) * L2 + cc]).count("1") for cc in range(c + 1, L2))
        assert true == pytest.approx(sgn * alt, rel=1e-10, abs=1e-14)
        n += 1
