"""Exact diagonalisation of the Fermi-Hubbard model (Sec. III.B, Eq. 14) in the grand-canonical
ensemble, for the checks of a fermionic PEPS: energy, double occupancy and next-nearest-
neighbour spin correlation per site against beta.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

  H = -t sum_<ij>,s (c+_is c_js + h.c.) + U sum_i n_iu n_id - mu sum_i,s n_is   (Eq. 14)

on the open nrow x ncol lattice.  Modes: m = 2 i + s (site i row-major, s = 0 up, 1 down);
a Fock state is a bit string with bit m set when mode m is occupied, and operators act in
the order of increasing mode index (Jordan-Wigner sign (-1)^(occupied modes before m)).
H conserves N_up and N_down, so it is diagonalised sector by sector.

Observables at inverse temperature beta (grand canonical):
  E/N = <H>/N, D = sum_i <n_iu n_id> / N (double occupancy), and
  F = sum_<<ij>> <S_i . S_j> / M over the M next-nearest-neighbour pairs (the diagonals of
  every plaquette), S_i the spin-1/2 operator of the electron at site i.
"""
from itertools import combinations

import numpy as np


def _nn_bonds(nrow, ncol):
    out = []
    for r in range(nrow):
        for c in range(ncol - 1):
            out.append((r * ncol + c, r * ncol + c + 1))
    for r in range(nrow - 1):
        for c in range(ncol):
            out.append((r * ncol + c, (r + 1) * ncol + c))
    return out


def _nnn_pairs(nrow, ncol):
    out = []
    for r in range(nrow - 1):
        for c in range(ncol - 1):
            out.append((r * ncol + c, (r + 1) * ncol + c + 1))
            out.append((r * ncol + c + 1, (r + 1) * ncol + c))
    return out


def _hop(state, m_from, m_to):
    """c+_{m_to} c_{m_from} |state>: (sign, new state) or None."""
    if not (state >> m_from) & 1:
        return None
    s1 = state & ~(1 << m_from)
    sign = -1 if bin(state & ((1 << m_from) - 1)).count("1") % 2 else 1
    if (s1 >> m_to) & 1:
        return None
    sign *= -1 if bin(s1 & ((1 << m_to) - 1)).count("1") % 2 else 1
    return sign, s1 | (1 << m_to)


def sector_basis(N, n_up, n_dn):
    """Fock states with n_up up and n_dn down electrons on N sites."""
    states = []
    for ups in combinations(range(N), n_up):
        for dns in combinations(range(N), n_dn):
            s = 0
            for i in ups:
                s |= 1 << (2 * i)
            for i in dns:
                s |= 1 << (2 * i + 1)
            states.append(s)
    return sorted(states)


def sector_hamiltonian(nrow, ncol, t, U, mu, n_up, n_dn):
    """Dense H in one (N_up, N_down) sector; returns (H, basis)."""
    N = nrow * ncol
    basis = sector_basis(N, n_up, n_dn)
    index = {s: k for k, s in enumerate(basis)}
    H = np.zeros((len(basis), len(basis)))
    bonds = _nn_bonds(nrow, ncol)
    for k, s in enumerate(basis):
        d = sum(((s >> (2 * i)) & 1) * ((s >> (2 * i + 1)) & 1) for i in range(N))
        H[k, k] = U * d - mu * (n_up + n_dn)
        for i, j in bonds:
            for sp in (0, 1):
                for a, b in ((i, j), (j, i)):
                    res = _hop(s, 2 * b + sp, 2 * a + sp)     # c+_a c_b
                    if res is not None:
                        sign, s2 = res
                        H[index[s2], k] += -t * sign
    return H, basis


def _diag_occ(s, N):
    return sum(((s >> (2 * i)) & 1) * ((s >> (2 * i + 1)) & 1) for i in range(N))


def _nnn_szsz(s, pairs):
    """Diagonal part sum_<<ij>> S^z_i S^z_j of a Fock state."""
    v = 0.0
    for i, j in pairs:
        zi = 0.5 * (((s >> (2 * i)) & 1) - ((s >> (2 * i + 1)) & 1))
        zj = 0.5 * (((s >> (2 * j)) & 1) - ((s >> (2 * j + 1)) & 1))
        v += zi * zj
    return v


def spin_exchange_matrix(nrow, ncol, basis):
    """sum_<<ij>> (S+_i S-_j + S-_i S+_j)/2 in a sector (S+_i = c+_iu c_id)."""
    index = {s: k for k, s in enumerate(basis)}
    M = np.zeros((len(basis), len(basis)))
    for k, s in enumerate(basis):
        for i, j in _nnn_pairs(nrow, ncol):
            for a, b in ((i, j), (j, i)):
                # S+_a S-_b = c+_au c_ad c+_bd c_bu
                r1 = _hop(s, 2 * b, 2 * b + 1)          # c+_bd c_bu
                if r1 is None:
                    continue
                r2 = _hop(r1[1], 2 * a + 1, 2 * a)      # c+_au c_ad
                if r2 is None:
                    continue
                M[index[r2[1]], k] += 0.5 * r1[0] * r2[0]
    return M


def thermal(nrow, ncol, t, U, mu, betas):
    """E/N, double occupancy D and NNN spin correlation F at each beta."""
    N = nrow * ncol
    pairs = _nnn_pairs(nrow, ncol)
    Mp = max(len(pairs), 1)
    sectors = []
    for n_up in range(N + 1):
        for n_dn in range(N + 1):
            H, basis = sector_hamiltonian(nrow, ncol, t, U, mu, n_up, n_dn)
            ev, V = np.linalg.eigh(H)
            dvec = np.array([_diag_occ(s, N) for s in basis], dtype=np.float64)
            zz = np.array([_nnn_szsz(s, pairs) for s in basis])
            F = np.diag(zz) + spin_exchange_matrix(nrow, ncol, basis)
            sectors.append((ev, np.einsum('ik,i,ik->k', V, dvec, V), np.einsum('ik,ij,jk->k', V, F, V)))
    e0 = min(s[0].min() for s in sectors)
    out = []
    for b in np.atleast_1d(betas):
        Z = E = Dn = Fn = 0.0
        for ev, dk, fk in sectors:
            w = np.exp(-b * (ev - e0))
            Z += w.sum()
            E += (w * ev).sum()
            Dn += (w * dk).sum()
            Fn += (w * fk).sum()
        out.append((E / Z / N, Dn / Z / N, Fn / Z / Mp))
    return np.array(out)


# ----------------------------------------------------------- the doubled (vectorised) state
#
# Eqs. 2-3 for fermions: rho(t) = e^{-t calH}|I> with calH = H x I + I x H^T is the Fock-basis
# matrix e^{-2tH} (up to normalisation), its entries rho(s, s') the amplitudes the method
# samples; the local energy of configuration S = (s, s') is
#     E_loc(S) = [(H rho)(s, s') + (rho H)(s, s')] / rho(s, s')  (E_sys + E_anc, Eq. 9)
# and Eq. 11 gives E = <E_loc>_{|rho|^2} / 2 at beta_obs = 4t.

def full_hamiltonian(nrow, ncol, t, U, mu):
    """Dense H on the whole Fock space (4^N states), Fock state = basis index."""
    N = nrow * ncol
    H = np.zeros((4 ** N, 4 ** N))
    for n_up in range(N + 1):
        for n_dn in range(N + 1):
            Hs, basis = sector_hamiltonian(nrow, ncol, t, U, mu, n_up, n_dn)
            idx = np.array(basis)
            H[np.ix_(idx, idx)] = Hs
    return H


def evolved_rho(H, t):
    """e^{-2tH} (shifted by the ground energy), the amplitudes of e^{-t calH}|I>."""
    ev, V = np.linalg.eigh(H)
    return (V * np.exp(-2.0 * t * (ev - ev.min()))) @ V.T


def local_energies(H, rho):
    """E_sys(s, s') = (H rho)(s, s') / rho(s, s'), E_anc = (rho H)(s, s') / rho(s, s'), where
    rho(s, s') != 0 (NaN elsewhere)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        nz = rho != 0
        es = np.where(nz, (H @ rho) / np.where(nz, rho, 1.0), np.nan)
        ea = np.where(nz, (rho @ H) / np.where(nz, rho, 1.0), np.nan)
    return es, ea
