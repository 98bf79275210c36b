"""Vectorised thermal state of the Fermi-Hubbard model (Sec. II, fermionic vectorisation and
Fig. 1b; Sec. III.B, Eq. 14) in the doubled Fock space, and the amplitudes of a fermionic PEPS
of it (Fermi arrows as an ordering of Grassmann-graded tensors).

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.  Small lattices only (dense vectors of
2^(4N) amplitudes).

Readings (the paper gives the vectorisation as a figure and a sentence):
  * Modes.  Every site carries four modes: system c_up, c_dn and ancilla d_up, d_dn, in that
    order; sites are row-major, so mode m = 4 i + k (k = 0 c_up, 1 c_dn, 2 d_up, 3 d_dn).  A
    Fock state is a bit string (bit m set: mode m occupied); operators act in increasing mode
    order, c+_m carrying the Jordan-Wigner sign (-1)^(occupied modes below m).  The local
    index of site i is S_i = bits 4i..4i+3 of the state: a = S_i & 3 the system occupation
    (bit 0 up, bit 1 down), b = S_i >> 2 the ancilla's; sixteen local states (d^2 = 16).
  * Identity.  Reversing the Fermi arrow of the ancilla leg pairs every system mode with its
    ancilla mode in an even state: |I> = prod_(i,s) (1 + c+_is d+_is)|0>.  On it a system
    operator equals an ancilla one: c_a|I> = d+_a|I> and c+_a|I> = -d_a|I>, so c+_a c_b|I> =
    d+_b d_a|I>: the hopping term, the interaction and the chemical potential of Eq. 14 on the
    system modes act on |I> as the same terms on the ancilla modes.  calH = H(c) + H(d) is the
    fermionic form of Eq. 3 (H^T with the arrows reversed is H on the ancilla).
  * Thermal state.  e^(-t calH)|I> = e^(-2t H(c))|I>, so weights |rho(S)|^2 give the
    e^(-4tH) averages: beta_obs = 4 t (Eq. 11), as for spins.
"""
import numpy as np
from scipy.sparse import csr_matrix
from scipy.sparse.linalg import expm_multiply

from .hubbard_ed import _nn_bonds


def n_modes(N):
    return 4 * N


def mode(i, k):
    """Mode index of site i, k = 0 c_up, 1 c_dn, 2 d_up, 3 d_dn."""
    return 4 * i + k


def create(M, m):
    """c+_m on the Fock space of M modes (Jordan-Wigner sign of the modes below m)."""
    dim = 1 << M
    rows, cols, vals = [], [], []
    for s in range(dim):
        if (s >> m) & 1:
            continue
        sign = -1.0 if bin(s & ((1 << m) - 1)).count("1") % 2 else 1.0
        rows.append(s | (1 << m))
        cols.append(s)
        vals.append(sign)
    return csr_matrix((vals, (rows, cols)), shape=(dim, dim))


def identity_state(N):
    """|I> = prod_(i,s) (1 + c+_is d+_is)|0> as a dense vector of 2^(4N) amplitudes."""
    M = n_modes(N)
    v = np.zeros(1 << M)
    v[0] = 1.0
    for i in range(N):
        for s in range(2):
            cd = create(M, mode(i, s)) @ create(M, mode(i, 2 + s))
            v = v + cd @ v
    return v


def hubbard_terms(nrow, ncol, t, U, mu, layer):
    """H of Eq. 14 on the system (layer 0: modes c) or the ancilla (layer 1: modes d) of the
    doubled lattice, sparse."""
    N = nrow * ncol
    M = n_modes(N)
    cr = {(i, s): create(M, mode(i, 2 * layer + s)) for i in range(N) for s in range(2)}
    H = csr_matrix((1 << M, 1 << M))
    for i, j in _nn_bonds(nrow, ncol):
        for s in range(2):
            hop = cr[(i, s)] @ cr[(j, s)].T
            H = H - t * (hop + hop.T)
    for i in range(N):
        nu = cr[(i, 0)] @ cr[(i, 0)].T
        nd = cr[(i, 1)] @ cr[(i, 1)].T
        H = H + U * (nu @ nd) - mu * (nu + nd)
    return H.tocsr()


def calH(nrow, ncol, t, U, mu):
    """The doubled operator calH = H(c) + H(d) (Eq. 3 for fermions, see the readings)."""
    return (hubbard_terms(nrow, ncol, t, U, mu, 0) + hubbard_terms(nrow, ncol, t, U, mu, 1)).tocsr()


def evolve(nrow, ncol, t_hop, U, mu, tau_total):
    """e^(-tau calH)|I>, normalised."""
    N = nrow * ncol
    v = expm_multiply(-tau_total * calH(nrow, ncol, t_hop, U, mu), identity_state(N))
    return v / np.linalg.norm(v)


def double_occupancy_op(N, layer=0):
    M = n_modes(N)
    out = csr_matrix((1 << M, 1 << M))
    for i in range(N):
        nu = create(M, mode(i, 2 * layer)) @ create(M, mode(i, 2 * layer)).T
        nd = create(M, mode(i, 2 * layer + 1)) @ create(M, mode(i, 2 * layer + 1)).T
        out = out + nu @ nd
    return out.tocsr()


def observables(nrow, ncol, t_hop, U, mu, vec):
    """E/N = <H(c)>/N and the double occupancy per site in the state vec (weights |vec|^2)."""
    N = nrow * ncol
    Hc = hubbard_terms(nrow, ncol, t_hop, U, mu, 0)
    nrm = vec @ vec
    return float(vec @ (Hc @ vec)) / nrm / N, float(vec @ (double_occupancy_op(N) @ vec)) / nrm / N


def local_energies(nrow, ncol, t_hop, U, mu, vec):
    """E_sys(S) = (H(c) vec)(S) / vec(S) and E_anc(S) = (H(d) vec)(S) / vec(S) on the
    configurations with vec(S) != 0 (Eq. 9: the local energy of calH is their sum)."""
    Hc = hubbard_terms(nrow, ncol, t_hop, U, mu, 0)
    Hd = hubbard_terms(nrow, ncol, t_hop, U, mu, 1)
    nz = vec != 0
    es = np.full(vec.shape, np.nan)
    ea = np.full(vec.shape, np.nan)
    es[nz] = (Hc @ vec)[nz] / vec[nz]
    ea[nz] = (Hd @ vec)[nz] / vec[nz]
    return es, ea


def local_indices(state, N):
    """The sixteen-valued local indices S_i of a Fock state of the doubled lattice."""
    return np.array([(state >> (4 * i)) & 15 for i in range(N)], dtype=np.int64)


def state_of(S):
    """The Fock state (bit string) of local indices S."""
    out = 0
    for i, v in enumerate(S):
        out |= int(v) << (4 * i)
    return out


# ----------------------------------------------------------------- fermionic PEPS amplitudes
#
# Reading of the Fermi arrows (the paper names the scheme, PRB 99, 195153, and gives no
# formula): every tensor is parity even, T_i[S, l, r, u, d] = 0 unless p(S) + p(l) + p(r) +
# p(u) + p(d) is even, with p(S) = popcount(S) mod 2 for a local index and p(v) = v mod 2 for
# a virtual index (index 0 even; the open edges have one even index).  The state is
#     |psi> = sum_S psi(S)|S>,  psi(S) = sum_v prod_i T_i[S_i, v_i] sigma(S, v),
# the Grassmann-ordered product of the site tensors: site i contributes, in site order, the
# letters l_i, u_i, P_i, d_i, r_i (incoming legs, its physical creation string, outgoing legs),
# odd letters anticommute, and sigma is the sign of the permutation of the odd letters that
# brings every physical string to the front in site order (the Fock state |S>, modes in
# increasing order) and every bond's two letters next to each other, the earlier site's
# first (where the bond is integrated out).  A gate sum_k A_k B_k on sites i < j, A_k and B_k
# of parity p_k on the sites' modes, acts on a state of even letters by attaching one virtual
# index k to an outgoing leg of i and an incoming leg of j (tests/test_oracle_fermion.py).

def _pv(v):
    return int(v) & 1


def _pS(s):
    return bin(int(s)).count("1") & 1


def fpeps_bonds(nrow, ncol):
    """Bonds (i, j, 'h' or 'v'), i < j, horizontal (r of i, l of j) and vertical (d of i, u
    of j), in a fixed order."""
    out = []
    for r in range(nrow):
        for c in range(ncol):
            i = r * ncol + c
            if c + 1 < ncol:
                out.append((i, i + 1, "h"))
            if r + 1 < nrow:
                out.append((i, i + ncol, "v"))
    return out


def fpeps_sign(nrow, ncol, S, vb):
    """sigma(S, v) by its definition: the parity of the permutation of the odd letters.
    vb[b] is the index of bond b of fpeps_bonds."""
    N = nrow * ncol
    bonds = fpeps_bonds(nrow, ncol)
    legs = {}   # (site, leg) -> bond position
    for b, (i, j, kind) in enumerate(bonds):
        legs[(i, "r" if kind == "h" else "d")] = b
        legs[(j, "l" if kind == "h" else "u")] = b
    # target position of each letter: physical strings first, then the bonds' letter pairs
    seq = []
    for i in range(N):
        for leg in ("l", "u", "P", "d", "r"):
            if leg == "P":
                if _pS(S[i]):
                    seq.append(i)
            elif (i, leg) in legs:
                b = legs[(i, leg)]
                if _pv(vb[b]):
                    first = leg in ("r", "d")          # the earlier site's letter
                    seq.append(N + 2 * b + (0 if first else 1))
    inv = sum(1 for a in range(len(seq)) for c in range(a + 1, len(seq)) if seq[a] > seq[c])
    return -1.0 if inv & 1 else 1.0


def fpeps_sign_local(nrow, ncol, S, vb):
    """sigma(S, v) from local factors: the physical strings among themselves, each site's
    physical parity against its incoming legs, and every crossing of two vertical bonds
    (the bond below (r, c) crosses those below (r, c') for c' > c and those below (r+1, c')
    for c' < c)."""
    N = nrow * ncol
    bonds = fpeps_bonds(nrow, ncol)
    idx = {(i, kind): b for b, (i, j, kind) in enumerate(bonds)}
    inc = {}
    for b, (i, j, kind) in enumerate(bonds):
        inc[(j, kind)] = b
    e = 0
    pre = 0
    for j in range(N):
        pj = _pS(S[j])
        pin = sum(_pv(vb[inc[(j, k)]]) for k in ("h", "v") if (j, k) in inc)
        e += pj * (pre + pin)
        pre += pj
    def pvert(r, c):
        b = idx.get((r * ncol + c, "v"))
        return 0 if b is None else _pv(vb[b])
    for r in range(nrow - 1):
        for c in range(ncol):
            pa = pvert(r, c)
            if not pa:
                continue
            for c2 in range(c + 1, ncol):
                e += pa * pvert(r, c2)
            if r + 2 <= nrow - 1:
                for c2 in range(c):
                    e += pa * pvert(r + 1, c2)
    return -1.0 if e & 1 else 1.0


def fpeps_state(nrow, ncol, T):
    """The whole state vector (2^(4N) amplitudes) of a fermionic PEPS by its definition:
    every assignment of the virtual indices, every nonzero tensor entry.  T[i] has shape
    (16, dl, dr, du, dd)."""
    N = nrow * ncol
    bonds = fpeps_bonds(nrow, ncol)
    dims = []
    for (i, j, kind) in bonds:
        dims.append(T[i].shape[2] if kind == "h" else T[i].shape[4])
    psi = np.zeros(1 << (4 * N))
    legpos = {}
    for b, (i, j, kind) in enumerate(bonds):
        legpos[(i, 2 if kind == "h" else 4)] = b
        legpos[(j, 1 if kind == "h" else 3)] = b
    for vb in np.ndindex(*dims) if dims else [()]:
        # per site: the vector over its sixteen local states at these virtual indices
        slices = []
        for i in range(N):
            ix = [slice(None)] + [vb[legpos[(i, a)]] if (i, a) in legpos else 0 for a in (1, 2, 3, 4)]
            slices.append(T[i][tuple(ix)])
        nz = [np.nonzero(s)[0] for s in slices]
        for S in np.ndindex(*[len(x) for x in nz]):
            Sv = [int(nz[i][S[i]]) for i in range(N)]
            amp = np.prod([slices[i][Sv[i]] for i in range(N)])
            if amp == 0.0:
                continue
            psi[state_of(Sv)] += amp * fpeps_sign(nrow, ncol, Sv, vb)
    return psi


def random_even_fpeps(nrow, ncol, D, rng, scale=1.0):
    """Seeded random parity-even tensors (16 local states, virtual dimension D inside, 1 on
    the open edges)."""
    T = []
    for r in range(nrow):
        for c in range(ncol):
            dl, dr = (1 if c == 0 else D), (1 if c == ncol - 1 else D)
            du, dd = (1 if r == 0 else D), (1 if r == nrow - 1 else D)
            A = scale * rng.standard_normal((16, dl, dr, du, dd))
            for idx in np.ndindex(*A.shape):
                if (_pS(idx[0]) + sum(_pv(x) for x in idx[1:])) & 1:
                    A[idx] = 0.0
            T.append(A)
    return T


def fpeps_amplitude_brute(nrow, ncol, T, S):
    """psi(S) by its definition: every assignment of the virtual indices."""
    bonds = fpeps_bonds(nrow, ncol)
    dims = [T[i].shape[2] if kind == "h" else T[i].shape[4] for (i, j, kind) in bonds]
    legpos = {}
    for b, (i, j, kind) in enumerate(bonds):
        legpos[(i, 2 if kind == "h" else 4)] = b
        legpos[(j, 1 if kind == "h" else 3)] = b
    out = 0.0
    for vb in np.ndindex(*dims) if dims else [()]:
        amp = 1.0
        for i in range(nrow * ncol):
            ix = [int(S[i])] + [vb[legpos[(i, a)]] if (i, a) in legpos else 0 for a in (1, 2, 3, 4)]
            amp *= T[i][tuple(ix)]
            if amp == 0.0:
                break
        if amp != 0.0:
            out += amp * fpeps_sign(nrow, ncol, S, vb)
    return out


def fpeps_amplitude_rows(nrow, ncol, T, S):
    """psi(S) contracted row by row with the signs in local form (fpeps_sign_local): each
    site's physical parity against its incoming legs folded into its tensor, the physical
    strings' sign as one factor, and the crossings of vertical bonds applied to the indices
    of the cuts (the bonds below one row among themselves, and those below row r against
    those below row r+1 further left).  The contraction keeps the full index vector of a cut
    (small lattices)."""
    N = nrow * ncol
    p = [_pS(s) for s in S]
    gsign = 1.0
    pre = 0
    for j in range(N):
        if p[j] and pre:
            gsign = -gsign
        pre ^= p[j]
    # site tensors at S, with (-1)^(p(S) (p(l) + p(u)))
    t = []
    for i in range(N):
        A = T[i][int(S[i])].copy()                    # (l, r, u, d)
        if p[i]:
            for idx in np.ndindex(*A.shape):
                if (_pv(idx[0]) + _pv(idx[2])) & 1:
                    A[idx] = -A[idx]
        t.append(A)

    def cut_sign(dims, other=None, other_dims=None):
        # (-1)^(sum_{c<c'} p_c p_c') over one cut; with `other`, the cross term
        # (-1)^(sum_{c'<c} p(this_c) p(next_c')) as an array over (this, next)
        if other is None:
            sg = np.ones(dims)
            for idx in np.ndindex(*dims):
                e = sum(_pv(idx[a]) * _pv(idx[b]) for a in range(len(idx)) for b in range(a + 1, len(idx)))
                sg[idx] = -1.0 if e & 1 else 1.0
            return sg
        sg = np.ones(tuple(dims) + tuple(other_dims))
        for idx in np.ndindex(*sg.shape):
            a, b = idx[:len(dims)], idx[len(dims):]
            e = sum(_pv(a[c]) * _pv(b[c2]) for c in range(len(a)) for c2 in range(c))
            sg[idx] = -1.0 if e & 1 else 1.0
        return sg

    vec = np.ones([1] * ncol)                          # over the up legs of row 0
    prev_dims = None
    for r in range(nrow):
        # row tensor over (up legs, down legs), horizontal bonds summed
        R = t[r * ncol][0]                             # (h, u_0, d_0): left edge l = 0
        for c in range(1, ncol):
            k = c                                      # ups (and downs) gathered so far
            R = np.tensordot(R, t[r * ncol + c], axes=([0], [0]))   # (u.., d.., h, u_c, d_c)
            perm = [2 * k] + list(range(k)) + [2 * k + 1] + list(range(k, 2 * k)) + [2 * k + 2]
            R = np.transpose(R, perm)                  # (h, u_0..u_c, d_0..d_c)
        R = R[0]                                       # right edge: h of dimension 1
        ups = R.shape[:ncol]
        downs = R.shape[ncol:]
        if r > 0:
            # crossings of the bonds above this row (cut r-1) with the bonds below it (cut r)
            R = R * cut_sign(ups, True, downs)
        vec = np.tensordot(vec * cut_sign(ups), R, axes=(list(range(ncol)), list(range(ncol))))
    return gsign * float(vec.reshape(()))


def identity_fpeps(nrow, ncol):
    """|I> as a fermionic PEPS of bond dimension 1: T_i[S] = <S_i|prod_s (1 + c+_s d+_s)|0>."""
    T = []
    for _ in range(nrow * ncol):
        A = np.zeros((16, 1, 1, 1, 1))
        for a in range(4):
            A[a | (a << 2), 0, 0, 0, 0] = -1.0 if a == 3 else 1.0
        T.append(A)
    return T


def hopping_gate_factors(t_hop, tau, spins=(0, 1)):
    """exp(tau t sum_s (c+_is c_js + c+_js c_is)) over the given spins, the gate of the hopping
    term of Eq. 14 on the system modes of two sites i < j, as sum_k A_k B_k: A_k, B_k 16 x 16
    matrices on the
    sites' local states (acting on their c modes), of parity p_k.  Obtained from the gate on
    the two sites' eight modes (site i's first) by undoing the sign (-1)^(p_k p(a)) that
    moving B_k past site i's string gives, then an SVD per parity."""
    M = 8
    cr = [create(M, m) for m in range(M)]
    h = csr_matrix((1 << M, 1 << M))
    for s in spins:
        hop = cr[s] @ cr[4 + s].T
        h = h + (hop + hop.T)
    from scipy.linalg import expm
    G = expm(tau * t_hop * h.toarray())
    par = np.array([_pS(x) for x in range(16)])
    Gt = np.zeros((16, 16, 16, 16))                   # [a', a, b', b]
    for a2 in range(16):
        for a in range(16):
            for b2 in range(16):
                for b in range(16):
                    v = G[a2 + 16 * b2, a + 16 * b]
                    if v != 0.0 and (par[b2] ^ par[b]) & par[a]:
                        v = -v
                    Gt[a2, a, b2, b] = v
    out = []
    for q in (0, 1):
        rows = [(a2, a) for a2 in range(16) for a in range(16) if par[a2] ^ par[a] == q]
        cols = [(b2, b) for b2 in range(16) for b in range(16) if par[b2] ^ par[b] == q]
        Mq = np.array([[Gt[a2, a, b2, b] for (b2, b) in cols] for (a2, a) in rows])
        U, sv, Vt = np.linalg.svd(Mq)
        for k in range(len(sv)):
            if sv[k] <= 1e-13 * sv[0]:
                break
            A = np.zeros((16, 16))
            B = np.zeros((16, 16))
            for r_, (a2, a) in enumerate(rows):
                A[a2, a] = U[r_, k] * np.sqrt(sv[k])
            for c_, (b2, b) in enumerate(cols):
                B[b2, b] = Vt[k, c_] * np.sqrt(sv[k])
            out.append((q, A, B))
    return out


def apply_gate_to_product(T, i, j, kind, factors):
    """Attaches a two-site gate sum_k A_k B_k (hopping_gate_factors) to the bond-dimension-1
    tensors of sites i < j of a fermionic PEPS whose other legs at i and j are of dimension 1:
    the virtual index of factor k (parity p_k; even factors on even indices, odd on odd) on
    the outgoing leg of i (r for 'h', d for 'v') and the incoming leg of j (l or u)."""
    ev = [f for f in factors if f[0] == 0]
    od = [f for f in factors if f[0] == 1]
    Dn = 2 * max(len(ev), len(od))
    A_new = np.zeros((16, 1, Dn, 1, 1) if kind == "h" else (16, 1, 1, 1, Dn))
    B_new = np.zeros((16, Dn, 1, 1, 1) if kind == "h" else (16, 1, 1, Dn, 1))
    ti = T[i][:, 0, 0, 0, 0]
    tj = T[j][:, 0, 0, 0, 0]
    for q, lst in ((0, ev), (1, od)):
        for n, (_, A, B) in enumerate(lst):
            k = 2 * n + q
            if kind == "h":
                A_new[:, 0, k, 0, 0] = A @ ti
                B_new[:, k, 0, 0, 0] = B @ tj
            else:
                A_new[:, 0, 0, 0, k] = A @ ti
                B_new[:, 0, 0, k, 0] = B @ tj
    T = list(T)
    T[i], T[j] = A_new, B_new
    return T


def _hop_sign(state, m_from, m_to):
    """c+_{m_to} c_{m_from}|state>: (sign, new state) or None (Jordan-Wigner signs)."""
    if not (state >> m_from) & 1:
        return None
    s1 = state & ~(1 << m_from)
    sign = -1.0 if bin(state & ((1 << m_from) - 1)).count("1") % 2 else 1.0
    if (s1 >> m_to) & 1:
        return None
    sign *= -1.0 if bin(s1 & ((1 << m_to) - 1)).count("1") % 2 else 1.0
    return sign, s1 | (1 << m_to)


def fpeps_local_energy(nrow, ncol, T, S, t_hop, U, mu):
    """E_sys(S) and E_anc(S) of a fermionic PEPS (Eq. 9 with the terms of Eq. 14 on the system
    and on the ancilla modes): the diagonal terms at S, plus every hop of one electron along a
    nearest-neighbour bond with its Jordan-Wigner sign times psi(S') / psi(S), each amplitude
    from the row contraction."""
    N = nrow * ncol
    st = state_of(S)
    psi = fpeps_amplitude_rows(nrow, ncol, T, S)
    out = []
    for layer in (0, 1):
        e = 0.0
        for i in range(N):
            nu = (st >> mode(i, 2 * layer)) & 1
            nd = (st >> mode(i, 2 * layer + 1)) & 1
            e += U * nu * nd - mu * (nu + nd)
        for i, j in _nn_bonds(nrow, ncol):
            for s in range(2):
                for a, b in ((i, j), (j, i)):
                    res = _hop_sign(st, mode(b, 2 * layer + s), mode(a, 2 * layer + s))
                    if res is None:
                        continue
                    sign, st2 = res
                    e += -t_hop * sign * fpeps_amplitude_rows(nrow, ncol, T, local_indices(st2, N)) / psi
        out.append(e)
    return out[0], out[1]


def fpeps_log_derivative(nrow, ncol, T, S):
    """O for configuration S (Eq. 8): d log psi(S) / d T_i[S_i, l, r, u, d] for every site, by
    the definition (every virtual assignment; the entries of T_i at S_i)."""
    N = nrow * ncol
    bonds = fpeps_bonds(nrow, ncol)
    dims = [T[i].shape[2] if kind == "h" else T[i].shape[4] for (i, j, kind) in bonds]
    legpos = {}
    for b, (i, j, kind) in enumerate(bonds):
        legpos[(i, 2 if kind == "h" else 4)] = b
        legpos[(j, 1 if kind == "h" else 3)] = b
    grads = [np.zeros(T[i].shape[1:]) for i in range(N)]
    psi = 0.0
    for vb in np.ndindex(*dims) if dims else [()]:
        ix = []
        vals = []
        for i in range(N):
            leg = tuple(vb[legpos[(i, a)]] if (i, a) in legpos else 0 for a in (1, 2, 3, 4))
            ix.append(leg)
            vals.append(T[i][(int(S[i]),) + leg])
        if sum(v != 0.0 for v in vals) < N - 1:
            continue
        sg = fpeps_sign(nrow, ncol, S, vb)
        full = np.prod(vals)
        psi += sg * full
        for i in range(N):
            rest = np.prod([vals[k] for k in range(N) if k != i])
            grads[i][ix[i]] += sg * rest
    return [g / psi for g in grads], psi


# The Grassmann sign in fully local form (tests/test_oracle_fermion.py pins it against the
# definition): with P_R the parity of the physical indices of rows 0..R (by parity evenness,
# the parity of the vertical bonds below row R) and b_i the parity of the physical indices to
# the left of site i in its row,
#     sigma(S, v) = (-1)^(sum_(i<j) p_i p_j + sum_R P_(R-1) P_R)
#                   * prod_i (-1)^((p(S_i) + p(d_i)) (p(l_i) + p(u_i)) + p(d_i) b_i),
# a configuration sign times a sign per site that depends on its own legs, its local index
# and one bit of the configuration.  So psi(S) is that configuration sign times the plain
# contraction of the tensors T_i[S_i] with the per-site signs folded in: a PEPS of 32 slices
# per site (S_i + 16 b_i) contracted as a bosonic one.

def fpeps_config_sign(nrow, ncol, S):
    """(-1)^(sum_(i<j) p_i p_j + sum_R P_(R-1) P_R)."""
    p = [_pS(s) for s in S]
    e = 0
    pre = 0
    for j in range(nrow * ncol):
        e += p[j] * pre
        pre ^= p[j]
    prev = 0
    acc = 0
    for R in range(nrow):
        acc ^= sum(p[R * ncol:(R + 1) * ncol]) & 1
        e += prev * acc
        prev = acc
    return -1.0 if e & 1 else 1.0


def fpeps_row_prefix_bits(nrow, ncol, S):
    """b_i: the parity of the physical indices left of site i in its row."""
    out = []
    for r in range(nrow):
        b = 0
        for c in range(ncol):
            out.append(b)
            b ^= _pS(S[r * ncol + c])
    return out


def fpeps_signed_slices(T):
    """The 32 signed slices per site: slice S + 16 b is T[S] times
    (-1)^((p(S) + p(d)) (p(l) + p(u)) + p(d) b), shape (32, dl, dr, du, dd)."""
    out = []
    for A in T:
        B = np.zeros((32,) + A.shape[1:])
        for b in range(2):
            for S in range(16):
                for idx in np.ndindex(*A.shape[1:]):
                    l, r, u, d = idx
                    e = (_pS(S) + _pv(d)) * (_pv(l) + _pv(u)) + _pv(d) * b
                    B[S + 16 * b][idx] = -A[S][idx] if e & 1 else A[S][idx]
        out.append(B)
    return out


def plain_amplitude(nrow, ncol, tensors):
    """Contraction of a plain (bosonic) PEPS whose site tensors are given at a fixed
    configuration, each of shape (l, r, u, d): the row-vector method."""
    vec = np.ones([1] * ncol)
    for r in range(nrow):
        R = tensors[r * ncol][0]
        for c in range(1, ncol):
            k = c
            R = np.tensordot(R, tensors[r * ncol + c], axes=([0], [0]))
            perm = [2 * k] + list(range(k)) + [2 * k + 1] + list(range(k, 2 * k)) + [2 * k + 2]
            R = np.transpose(R, perm)
        R = R[0]
        vec = np.tensordot(vec, R, axes=(list(range(ncol)), list(range(ncol))))
    return float(vec.reshape(()))


def fpeps_amplitude_function(nrow, ncol, T):
    """S -> psi(S): the configuration sign times the plain contraction of the signed slices
    (made once for T)."""
    Ts = fpeps_signed_slices(T)

    def amp(S):
        b = fpeps_row_prefix_bits(nrow, ncol, S)
        t = [Ts[i][int(S[i]) + 16 * b[i]] for i in range(nrow * ncol)]
        return fpeps_config_sign(nrow, ncol, S) * plain_amplitude(nrow, ncol, t)
    return amp


def fpeps_amplitude_bosonic(nrow, ncol, T, S):
    """psi(S) as the configuration sign times the plain contraction of the signed slices."""
    return fpeps_amplitude_function(nrow, ncol, T)(S)
