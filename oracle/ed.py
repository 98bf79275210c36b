"""Exact diagonalisation and full-state imaginary-time evolution (Sec. II Eqs. 1-3, Eq. 12).

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

  H = J1 sum_<ij> S_i.S_j + J2 sum_<<ij>> S_i.S_j on the open nrow x ncol lattice (Eq. 12).
  Spin basis: bit i of the state index (site 0 most significant) is s_i (0 = up).
  S_i.S_j = S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j)/2: diagonal J s^z s^z, and J/2
  between states that differ by exchanging antiparallel spins i and j.

  Thermal values at inverse temperature beta from the spectrum, sector by sector in
  M_z (H conserves M_z):  E = <H>, C = beta^2 (<H^2> - <H>^2), chi = beta <M_z^2> (Eq. 13
  with <M_z> = 0), each divided by N.

  Vectorisation (Eq. 2): rho_{s s'} -> rho(S_1..S_N) with S_i = 2 s_i + s'_i; Eq. 3's
  calH = H x I + I x H^T as a matrix on that space, for the full-state checks.
"""
from itertools import combinations

import numpy as np


def _bond_list(lat):
    return [(i, j, J) for (i, j, J, _) in lat.bonds()]


def hamiltonian_sector(lat, n_down):
    """Dense H restricted to states with n_down down spins; returns (H, basis states)."""
    N = lat.N
    states = []
    for downs in combinations(range(N), n_down):
        x = 0
        for i in downs:
            x |= 1 << (N - 1 - i)
        states.append(x)
    states = sorted(states)
    index = {x: k for k, x in enumerate(states)}
    H = np.zeros((len(states), len(states)))
    bonds = _bond_list(lat)
    for k, x in enumerate(states):
        for (i, j, J) in bonds:
            si = (x >> (N - 1 - i)) & 1
            sj = (x >> (N - 1 - j)) & 1
            H[k, k] += J * (0.5 - si) * (0.5 - sj)
            if si != sj:
                y = x ^ (1 << (N - 1 - i)) ^ (1 << (N - 1 - j))
                H[index[y], k] += 0.5 * J
    return H, states


def spectrum(lat):
    """All eigenvalues with their M_z: list of (M_z, eigenvalues)."""
    out = []
    for nd in range(lat.N + 1):
        H, _ = hamiltonian_sector(lat, nd)
        out.append((0.5 * lat.N - nd, np.linalg.eigvalsh(H)))
    return out


def thermal(spec, N, betas):
    """E/N, C/N, chi/N at each beta from the sector spectra (shifted by the ground energy)."""
    betas = np.atleast_1d(np.asarray(betas, dtype=np.float64))
    e0 = min(ev.min() for _, ev in spec)
    out = []
    for b in betas:
        Z = E1 = E2 = M2 = 0.0
        for mz, ev in spec:
            wts = np.exp(-b * (ev - e0))
            Z += wts.sum()
            E1 += (wts * ev).sum()
            E2 += (wts * ev * ev).sum()
            M2 += wts.sum() * mz * mz
        E1, E2, M2 = E1 / Z, E2 / Z, M2 / Z
        out.append((E1 / N, b * b * (E2 - E1 * E1) / N, b * M2 / N))
    return np.array(out)


def full_hamiltonian(lat):
    """Dense H on all 2^N spin states."""
    N = lat.N
    dim = 1 << N
    H = np.zeros((dim, dim))
    for nd in range(N + 1):
        Hs, states = hamiltonian_sector(lat, nd)
        idx = np.array(states)
        H[np.ix_(idx, idx)] = Hs
    return H


def doubled_hamiltonian(lat):
    """calH = H x I + I x H^T (Eq. 3) on the vectorised space, as a matrix over the
    configuration index sum_i S_i 4^(N-1-i)."""
    H = full_hamiltonian(lat)
    I = np.eye(H.shape[0])
    Hd = np.kron(H, I) + np.kron(I, H.T)      # index s * 2^N + s'
    perm = pair_to_config_index(lat.N)
    return Hd[np.ix_(perm, perm)]


def pair_to_config_index(N):
    """perm[cfg] = s * 2^N + s' for configuration index cfg = sum_i S_i 4^(N-1-i)."""
    perm = np.zeros(4 ** N, dtype=np.int64)
    for cfg in range(4 ** N):
        s = sp = 0
        for i in range(N):
            Si = (cfg >> (2 * (N - 1 - i))) & 3
            s = (s << 1) | (Si >> 1)
            sp = (sp << 1) | (Si & 1)
        perm[cfg] = (s << N) | sp
    return perm


def config_of_index(cfg, N):
    """Local indices S_i of configuration index cfg."""
    return np.array([(cfg >> (2 * (N - 1 - i))) & 3 for i in range(N)], dtype=np.int64)


def evolve_identity(lat, t):
    """|rho(t)> = exp(-t calH)|I> = vec(exp(-2tH)) (Eqs. 1-3), as a vector over configurations."""
    H = full_hamiltonian(lat)
    ev, V = np.linalg.eigh(H)
    rho = (V * np.exp(-2.0 * t * (ev - ev.min()))) @ V.T
    perm = pair_to_config_index(lat.N)
    return rho.reshape(-1)[perm]
