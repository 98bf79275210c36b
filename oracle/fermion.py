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
from scipy.sparse import csr_matrix, identity
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
