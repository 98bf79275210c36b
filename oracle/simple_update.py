"""Simple-update (SU) evolution of the doubled-lattice PEPS at high temperature.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

Definitions followed (arXiv:2409.05285):
  * Eq. 3: |rho_beta> = e^{-tau calH} ... e^{-tau calH} |I>, calH = H x I + I x H^T, and H is
    a sum of bond terms (Eq. 12).  For one bond the doubled term is h_ij x I + I x h_ij^T on
    the system and ancilla spins of the two sites; the two parts commute, so
    e^{-tau calH_ij} = e^{-tau h_ij} (system) x e^{-tau h_ij^T} (ancilla).
  * App. A: at very high temperature the state is close to the product state |I>, so the
    environment of a bond can be replaced by bond weights (the SU scheme of Jiang, Weng and
    Xiang, PRL 101, 090603); tens to hundreds of SU steps, then SR.

Scheme (the paper gives no details; the standard SU written out here):
  * State: site tensors G_i[S][l][r][u][d] and a weight vector lam on every bond.  At beta = 0
    every bond has dimension 1 and weight 1, and G_i^S = delta_{s s'}.
  * One SU step of length tau: the gate e^{-tau calH_ij} on every bond, horizontal bonds row
    by row and then vertical bonds (first-order Trotter order).  For a bond (A, B): multiply
    the weights of A's and B's other bonds into their legs, contract A - lam_AB - B, apply the
    gate on (S_A, S_B), split by SVD, keep the D largest singular values (those above 1e-14 of
    the largest), store them divided by their largest as the new lam_AB, and divide the outer
    weights back out of the two new tensors.
  * Next-nearest-neighbour bonds (J2) through a site of their plaquette with exchange gates
    (su_step).
  * to_theta: sqrt(lam) of each bond multiplied into both of its tensors, legs zero-padded to
    the lattice's bond dimension D (trimmed open boundaries keep dimension 1), in the layout
    of oracle.lattice.  The overall scale of the state is arbitrary (ratios, O and the
    normalised estimators do not depend on it).
"""
import numpy as np
from scipy.linalg import expm

# spin-1/2 S_i . S_j on (s_i, s_j), s = 0 up, 1 down, index 2 s_i + s_j
_SS = np.array([[0.25, 0.0, 0.0, 0.0],
                [0.0, -0.25, 0.5, 0.0],
                [0.0, 0.5, -0.25, 0.0],
                [0.0, 0.0, 0.0, 0.25]])


def bond_gate(J, tau):
    """e^{-tau calH_ij} as a 16 x 16 matrix on (S_i, S_j), index 4 S_i + S_j, S = 2 s + s'."""
    g = expm(-tau * J * _SS)                       # on (s_i, s_j); h real symmetric: h^T = h
    G = np.einsum('ac,bd->abcd', g, g)            # [(s_i' s_j'), (s'_i' s'_j'), (s_i s_j), (s'_i s'_j)]
    G = G.reshape(2, 2, 2, 2, 2, 2, 2, 2)          # s_i' s_j' a_i' a_j' s_i s_j a_i a_j
    G = G.transpose(0, 2, 1, 3, 4, 6, 5, 7)        # (s_i' a_i') (s_j' a_j') (s_i a_i) (s_j a_j)
    return G.reshape(16, 16)


class SUState:
    """Site tensors G[i] (4, dl, dr, du, dd) and bond weights: lh[(r, c)] between (r, c) and
    (r, c+1), lv[(r, c)] between (r, c) and (r+1, c)."""

    def __init__(self, lat):
        self.lat = lat
        self.G = []
        for _ in range(lat.N):
            t = np.zeros((4, 1, 1, 1, 1))
            t[0, 0, 0, 0, 0] = 1.0                 # s = s' = up
            t[3, 0, 0, 0, 0] = 1.0                 # s = s' = down
            self.G.append(t)
        self.lh = {(r, c): np.ones(1) for r in range(lat.nrow) for c in range(lat.ncol - 1)}
        self.lv = {(r, c): np.ones(1) for r in range(lat.nrow - 1) for c in range(lat.ncol)}

    def weights(self, r, c):
        """Weights of the four legs (l, r, u, d) of site (r, c); ones on open boundaries."""
        lat = self.lat
        one = np.ones(1)
        return (self.lh[(r, c - 1)] if c > 0 else one,
                self.lh[(r, c)] if c < lat.ncol - 1 else one,
                self.lv[(r - 1, c)] if r > 0 else one,
                self.lv[(r, c)] if r < lat.nrow - 1 else one)


def _scale(t, w, leg, power):
    """Multiply leg `leg` (1..4 of a (4, l, r, u, d) tensor) by w**power."""
    shape = [1] * 5
    shape[leg] = len(w)
    return t * (w ** power).reshape(shape)


def _inv(w):
    return np.where(w > 0, 1.0 / np.where(w > 0, w, 1.0), 0.0)


def swap_gate():
    """Exchange of the whole local states of two sites, 16 x 16 on (S_i, S_j)."""
    G = np.zeros((16, 16))
    for a in range(4):
        for b in range(4):
            G[4 * b + a, 4 * a + b] = 1.0
    return G


def apply_bond(st, r, c, horizontal, J, tau, D, gate=None):
    """Gate on the bond from (r, c) to its right (horizontal) or lower neighbour
    (e^{-tau calH_ij} with coupling J, or the 16 x 16 `gate` when given)."""
    lat = st.lat
    ia = lat.site(r, c)
    rb, cb = (r, c + 1) if horizontal else (r + 1, c)
    ib = lat.site(rb, cb)
    wa, wb = st.weights(r, c), st.weights(rb, cb)
    la, lb = (2, 1) if horizontal else (4, 3)      # shared leg: A's right / down, B's left / up
    A, B = st.G[ia], st.G[ib]
    outer_a = [k for k in (1, 2, 3, 4) if k != la]
    outer_b = [k for k in (1, 2, 3, 4) if k != lb]
    for k in outer_a:
        A = _scale(A, wa[k - 1], k, 1.0)
    for k in outer_b:
        B = _scale(B, wb[k - 1], k, 1.0)
    lam = st.lh[(r, c)] if horizontal else st.lv[(r, c)]
    A = _scale(A, lam, la, 1.0)
    # move the shared leg last in A, first (after S) in B
    pa = [0] + outer_a + [la]
    pb = [0, lb] + outer_b
    A2 = A.transpose(pa)                           # S_A, o1, o2, o3, k
    B2 = B.transpose(pb)                           # S_B, k, o1, o2, o3
    sa, sb = A2.shape[1:4], B2.shape[2:5]
    theta = np.tensordot(A2, B2, axes=([4], [1]))  # S_A, oa..., S_B, ob...
    theta = np.moveaxis(theta, 4, 1)               # S_A, S_B, oa..., ob...
    th = theta.reshape(16, -1)
    th = ((bond_gate(J, tau) if gate is None else gate) @ th).reshape((4, 4) + sa + sb)
    th = np.moveaxis(th, 1, 4)                     # S_A, oa..., S_B, ob...
    M = th.reshape(4 * int(np.prod(sa)), 4 * int(np.prod(sb)))
    U, s, Vt = np.linalg.svd(M, full_matrices=False)
    keep = int(np.sum(s > 1e-14 * s[0])) if s[0] > 0 else 1
    k = max(1, min(D, keep))
    U, s, Vt = U[:, :k], s[:k], Vt[:k]
    lam_new = s / s[0]
    An = U.reshape((4,) + sa + (k,))               # S_A, oa..., k
    Bn = Vt.reshape((k, 4) + sb)                    # k, S_B, ob...
    Bn = np.moveaxis(Bn, 0, 1)                      # S_B, k, ob...
    An = An.transpose(np.argsort(pa))
    Bn = Bn.transpose(np.argsort(pb))
    for kk in outer_a:
        An = _scale(An, _inv(wa[kk - 1]), kk, 1.0)
    for kk in outer_b:
        Bn = _scale(Bn, _inv(wb[kk - 1]), kk, 1.0)
    st.G[ia], st.G[ib] = An, Bn
    if horizontal:
        st.lh[(r, c)] = lam_new
    else:
        st.lv[(r, c)] = lam_new


def su_step(st, tau, D):
    """One first-order Trotter step of length tau: every bond of Eq. 12 once.  Nearest-
    neighbour bonds directly; a next-nearest-neighbour bond of plaquette (r, c) through the
    plaquette's top-right site (r, c+1) for the diagonal (r,c)-(r+1,c+1), or top-left site
    (r, c) for the anti-diagonal (r,c+1)-(r+1,c): exchange the local states across the top
    bond, apply the gate on the vertical bond that then joins the two sites' states, and
    exchange back (each exchange a bond update with truncation to D)."""
    lat = st.lat
    for r in range(lat.nrow):
        for c in range(lat.ncol - 1):
            apply_bond(st, r, c, True, lat.J1, tau, D)
    for r in range(lat.nrow - 1):
        for c in range(lat.ncol):
            apply_bond(st, r, c, False, lat.J1, tau, D)
    if lat.J2 != 0.0:
        sw, g2 = swap_gate(), bond_gate(lat.J2, tau)
        for r in range(lat.nrow - 1):
            for c in range(lat.ncol - 1):
                for via in (c + 1, c):            # diagonal, then anti-diagonal
                    apply_bond(st, r, c, True, 0.0, 0.0, D, gate=sw)
                    apply_bond(st, r, via, False, 0.0, 0.0, D, gate=g2)
                    apply_bond(st, r, c, True, 0.0, 0.0, D, gate=sw)


def to_theta(st):
    """Plain PEPS parameters: sqrt of each bond weight into both tensors, legs zero-padded to
    the lattice's dimensions."""
    lat = st.lat
    theta = np.zeros(lat.Np)
    for r in range(lat.nrow):
        for c in range(lat.ncol):
            i = lat.site(r, c)
            t = st.G[i]
            for k, w in enumerate(st.weights(r, c)):
                t = _scale(t, w, k + 1, 0.5)
            full = np.zeros((4,) + lat.dims[i])
            full[:, :t.shape[1], :t.shape[2], :t.shape[3], :t.shape[4]] = t
            off = int(lat.theta_off[i])
            theta[off:off + full.size] = full.reshape(-1)
    return theta
