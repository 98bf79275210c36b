"""Pins of the fermionic oracle (oracle/fermion.py).  Vectorisation: the identity's pairing
relations and closed form, the doubled Hamiltonian on it, the beta = 0 closed forms of
Eq. 14, the thermal energy and double occupancy against the sector-by-sector exact
diagonalisation, the local energies' average, and the amplitudes against the matrix
e^(-2tH) of the diagonalisation up to a fixed sign per configuration.  Fermionic PEPS: the
local form of the Grassmann sign against its definition, the row contraction against the
sum over virtual indices, and PEPS carrying hopping gates against the Jordan-Wigner state."""
import numpy as np
import pytest

from oracle import fermion as fm
from oracle import hubbard_ed as hed


def _fock_pairs(N):
    # doubled Fock state -> (s, s') in the diagonalisation's mode order (mode 2 i + spin)
    out = {}
    for st in range(1 << (4 * N)):
        S = fm.local_indices(st, N)
        s = sum(int(S[i] & 3) << (2 * i) for i in range(N))
        sp = sum(int(S[i] >> 2) << (2 * i) for i in range(N))
        out[st] = (s, sp)
    return out


def test_identity_pairs_system_with_ancilla():
    N = 2
    M = fm.n_modes(N)
    I = fm.identity_state(N)
    for i in range(N):
        for s in range(2):
            c = fm.create(M, fm.mode(i, s))
            d = fm.create(M, fm.mode(i, 2 + s))
            assert np.allclose(c.T @ I, d @ I)          # c|I> = d+|I>
            assert np.allclose(c @ I, -(d.T @ I))       # c+|I> = -d|I>
    # closed form: nonzero where system and ancilla occupations agree site by site, sign -1
    # per doubly occupied pair (c+_up d+_up c+_dn d+_dn brought into mode order)
    for st in range(1 << M):
        S = fm.local_indices(st, N)
        a, b = S & 3, S >> 2
        want = 0.0 if np.any(a != b) else float(np.prod([-1.0 if x == 3 else 1.0 for x in a]))
        assert I[st] == want


@pytest.mark.parametrize("shape", [(1, 2), (2, 2)])
def test_doubled_hamiltonian_on_identity(shape):
    # Eq. 3 read for fermions: H on the ancilla acts on |I> as H on the system
    nrow, ncol = shape
    I = fm.identity_state(nrow * ncol)
    Hc = fm.hubbard_terms(nrow, ncol, 0.7, 3.1, 1.3, 0)
    Hd = fm.hubbard_terms(nrow, ncol, 0.7, 3.1, 1.3, 1)
    assert np.allclose(Hc @ I, Hd @ I, atol=1e-12)
    assert np.allclose(fm.calH(nrow, ncol, 0.7, 3.1, 1.3) @ I, 2 * (Hc @ I), atol=1e-12)


def test_beta0_closed_forms():
    # infinite temperature: E/N = Tr H / 4^N / N = U/4 - mu, double occupancy 1/4
    for U, mu in ((8.0, 4.0), (3.0, 0.5)):
        E, D = fm.observables(2, 2, 1.0, U, mu, fm.identity_state(4))
        assert E == pytest.approx(U / 4 - mu, abs=1e-12)
        assert D == pytest.approx(0.25, abs=1e-12)


@pytest.mark.parametrize("shape,U,mu", [((2, 2), 8.0, 4.0), ((1, 3), 4.0, 1.0)])
def test_thermal_state_matches_exact_diagonalisation(shape, U, mu):
    # e^(-tau calH)|I> sampled with |rho|^2 is the thermal state at beta = 4 tau (Eq. 11)
    nrow, ncol = shape
    taus = [0.05, 0.2, 0.5]
    ref = hed.thermal(nrow, ncol, 1.0, U, mu, [4 * t for t in taus])
    for k, tau in enumerate(taus):
        v = fm.evolve(nrow, ncol, 1.0, U, mu, tau)
        E, D = fm.observables(nrow, ncol, 1.0, U, mu, v)
        assert E == pytest.approx(ref[k, 0], rel=1e-9, abs=1e-12)
        assert D == pytest.approx(ref[k, 1], rel=1e-9, abs=1e-12)
        # the estimator of Eq. 9-11: <(E_sys + E_anc)/2>_{|rho|^2} is the same energy
        es, ea = fm.local_energies(nrow, ncol, 1.0, U, mu, v)
        w = v ** 2
        nz = v != 0
        assert np.sum(w[nz] * 0.5 * (es[nz] + ea[nz])) / np.sum(w) / (nrow * ncol) == pytest.approx(
            ref[k, 0], rel=1e-9, abs=1e-12)


def test_amplitudes_are_the_matrix_up_to_a_fixed_sign():
    # <S|e^(-tau calH)|I> against e^(-2 tau H)(s, s') of the diagonalisation: equal in size,
    # with a sign that depends on the configuration alone (the same at every tau)
    nrow, ncol, U, mu = 1, 2, 3.0, 1.0
    N = nrow * ncol
    H = hed.full_hamiltonian(nrow, ncol, 1.0, U, mu)
    pairs = _fock_pairs(N)
    signs = None
    for tau in (0.1, 0.4):
        v = fm.evolve(nrow, ncol, 1.0, U, mu, tau)
        rho = hed.evolved_rho(H, tau)
        m = np.array([rho[pairs[st]] for st in range(len(v))])
        scale = np.linalg.norm(m)
        nz = np.abs(m) > 1e-12 * scale
        assert np.all(np.abs(v[~nz]) <= 1e-12)
        ratio = v[nz] / (m[nz] / scale)
        assert np.allclose(np.abs(ratio), 1.0, atol=1e-10)
        sg = np.sign(ratio)
        if signs is None:
            signs = sg
        else:
            assert np.array_equal(sg, signs)


# ---------------------------------------------------------------- fermionic PEPS amplitudes

def _consistent_assignment(nr, nc, rng):
    bonds = fm.fpeps_bonds(nr, nc)
    vb = rng.integers(0, 4, len(bonds))
    S = []
    for i in range(nr * nc):
        par = 0
        for b, (a, c, _) in enumerate(bonds):
            if i in (a, c):
                par ^= int(vb[b]) & 1
        choices = [s for s in range(16) if (bin(s).count("1") & 1) == par]
        S.append(int(rng.choice(choices)))
    return S, vb


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 3), (3, 4), (4, 3)])
def test_fpeps_sign_local_form_equals_its_definition(shape):
    # the permutation parity of the odd Grassmann letters against its local factors (the
    # physical strings, each site's parity against its incoming legs, crossings of vertical
    # bonds within a cut and with the next cut to the left)
    nr, nc = shape
    rng = np.random.default_rng(nr * 10 + nc)
    for _ in range(200):
        S, vb = _consistent_assignment(nr, nc, rng)
        assert fm.fpeps_sign(nr, nc, S, vb) == fm.fpeps_sign_local(nr, nc, S, vb)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_fpeps_row_contraction_equals_definition(shape):
    # the contraction a sampler would run (signs on the cut indices) against the sum over
    # every virtual assignment; odd-parity configurations vanish in both
    nr, nc = shape
    rng = np.random.default_rng(7 + nr + nc)
    T = fm.random_even_fpeps(nr, nc, 2, rng)
    nonzero = 0
    for _ in range(8):
        S = rng.integers(0, 16, nr * nc)
        a = fm.fpeps_amplitude_brute(nr, nc, T, S)
        b = fm.fpeps_amplitude_rows(nr, nc, T, S)
        assert b == pytest.approx(a, rel=1e-12, abs=1e-14)
        if sum(bin(int(s)).count("1") for s in S) % 2:
            assert a == 0.0
        else:
            nonzero += a != 0.0
    assert nonzero > 0


def test_identity_fpeps():
    assert np.array_equal(fm.fpeps_state(2, 2, fm.identity_fpeps(2, 2)), fm.identity_state(4))


@pytest.mark.parametrize("shape,gates", [
    ((1, 2), [(0, 1, "h")]),
    ((2, 1), [(0, 1, "v")]),
    ((2, 2), [(0, 2, "v")]),
    ((2, 2), [(0, 1, "h"), (2, 3, "h")]),
    ((2, 2), [(0, 2, "v"), (1, 3, "v")]),
])
def test_fpeps_of_gated_identity_is_the_fermionic_state(shape, gates):
    # hopping gates of Eq. 14 applied to |I> on the state vector (Jordan-Wigner operators)
    # against the fermionic PEPS that carries each gate on one bond: the same amplitudes,
    # signs included, also where two vertical bonds cross in the Grassmann order
    from scipy.sparse.linalg import expm_multiply
    nr, nc = shape
    tau, t_hop = 0.3, 1.0
    f = fm.hopping_gate_factors(t_hop, tau)
    assert sorted({q for q, _, _ in f}) == [0, 1]
    N = nr * nc
    M = fm.n_modes(N)
    T = fm.identity_fpeps(nr, nc)
    v = fm.identity_state(N)
    for (i, j, kind) in gates:
        T = fm.apply_gate_to_product(T, i, j, kind, f)
        h = None
        for s in range(2):
            hop = fm.create(M, fm.mode(i, s)) @ fm.create(M, fm.mode(j, s)).T
            h = (hop + hop.T) if h is None else h + hop + hop.T
        v = expm_multiply(tau * t_hop * h, v)
    psi = fm.fpeps_state(nr, nc, T)
    assert np.max(np.abs(psi - v)) <= 1e-12 * np.max(np.abs(v))
    # and its thermal content: the same energy as the state vector
    E1, _ = fm.observables(nr, nc, t_hop, 8.0, 4.0, psi)
    E2, _ = fm.observables(nr, nc, t_hop, 8.0, 4.0, v)
    assert E1 == pytest.approx(E2, rel=1e-12)


def test_fpeps_local_energy_and_log_derivative():
    # a fermionic PEPS with hopping gates on two crossing vertical bonds (2x2): its local
    # energies (Eq. 9, terms of Eq. 14, Jordan-Wigner signs, amplitudes of the row contraction)
    # against the state vector's, and O (Eq. 8) against finite differences of the amplitude
    nr, nc, t_hop, U, mu = 2, 2, 1.0, 8.0, 4.0
    f = fm.hopping_gate_factors(t_hop, 0.3)
    T = fm.identity_fpeps(nr, nc)
    for (i, j, kind) in [(0, 2, "v"), (1, 3, "v")]:
        T = fm.apply_gate_to_product(T, i, j, kind, f)
    psi = fm.fpeps_state(nr, nc, T)
    es, ea = fm.local_energies(nr, nc, t_hop, U, mu, psi)
    rng = np.random.default_rng(3)
    support = np.nonzero(np.abs(psi) > 1e-8 * np.max(np.abs(psi)))[0]
    for st in rng.choice(support, 12, replace=False):
        S = fm.local_indices(int(st), nr * nc)
        e1, e2 = fm.fpeps_local_energy(nr, nc, T, S, t_hop, U, mu)
        assert e1 == pytest.approx(es[st], rel=1e-10, abs=1e-10)
        assert e2 == pytest.approx(ea[st], rel=1e-10, abs=1e-10)
    # O against central differences of the amplitude on a random even PEPS
    T = fm.random_even_fpeps(nr, nc, 2, rng)
    S = [1, 3, 0, 2]   # even total parity
    O, amp = fm.fpeps_log_derivative(nr, nc, T, S)
    assert amp == pytest.approx(fm.fpeps_amplitude_rows(nr, nc, T, S), rel=1e-12)
    h = 1e-6
    for i in range(nr * nc):
        for idx in list(np.ndindex(*T[i].shape[1:]))[:6]:
            Tp = [x.copy() for x in T]
            Tm = [x.copy() for x in T]
            Tp[i][(S[i],) + idx] += h
            Tm[i][(S[i],) + idx] -= h
            d = (fm.fpeps_amplitude_rows(nr, nc, Tp, S) - fm.fpeps_amplitude_rows(nr, nc, Tm, S)) / (2 * h)
            assert O[i][idx] == pytest.approx(d / amp, rel=1e-6, abs=1e-8)


@pytest.mark.parametrize("shape", [(2, 2), (2, 3), (3, 2), (3, 3)])
def test_fpeps_bosonic_form(shape):
    # the fully local form: a configuration sign times a plain contraction of 32 signed
    # slices per site, against the sum over every virtual assignment (the definition)
    nr, nc = shape
    rng = np.random.default_rng(17 + nr * nc)
    T = fm.random_even_fpeps(nr, nc, 2, rng)
    for _ in range(8):
        S = rng.integers(0, 16, nr * nc)
        a = fm.fpeps_amplitude_brute(nr, nc, T, S)
        assert fm.fpeps_amplitude_bosonic(nr, nc, T, S) == pytest.approx(a, rel=1e-12, abs=1e-14)
