"""PEPS of the vectorised density matrix and its single-layer contraction at fixed S.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

Definitions followed (arXiv:2409.05285, Sec. II):
  * Eq. 4: rho_theta(S) = full contraction of T_1^{S_1} ... T_N^{S_N} (open boundaries).
  * Eq. 8: O_k(S) = d rho_theta(S)/d theta_k / rho_theta(S).
  * Eq. 9: E_loc(S) = sum_S' rho(S')/rho(S) * calH_{S S'}, calH = H x I + I x H^T (Eq. 3).
  * App. A: beta = 0 state with its zero entries perturbed.
  * Sec. III.A: the single-layer network is contracted by boundary MPS of bond dimension
    D_c = chi (the boundary-MPS method of PRB 103, 235155).

Boundary-MPS conventions used here (the paper gives no truncation scheme):
  * An environment is an MPS over the ncol columns, tensors E_c[a, p, b] (left bond, the
    open vertical leg, right bond), plus a float64 log-scale.  up[r] is the contraction of
    rows 0..r-1 (open legs = up legs of row r); down[r] is rows r..nrow-1 (open legs = down
    legs of row r-1).  up[0] and down[nrow] are trivial (all dims 1, value 1).
  * Absorbing a row multiplies its tensors into the MPS, fusing bond (a, l) -> a*dl + l.
  * compress(C, chi): if every bond of C is <= chi, C is kept as is.  Otherwise
      (i)  right-to-left: factors L_c with C_{>=c} = L_c Q_{>=c}, Q_{>=c} row-orthonormal,
           from the LQ decomposition of C_c . L_{c+1};
      (ii) left-to-right: X_c = (carry . C_c) . L_{c+1}, reshaped (b'*p) x k; its SVD keeps
           the chi largest singular values; the site tensor becomes U_chi and the carry
           U_chi^T (carry . C_c).  This is SVD truncation of the MPS in canonical form.
  * Every environment tensor is divided by its max-abs entry, the logarithm added to the
    log-scale (any normalisation gives the same ratios, O and log|rho|).
  * Multi-operand contractions are written as a sequence of pairwise tensordot calls.
  * rho(S) reported as the amplitude is the row-0 strip value (up[0], row 0, down[1]).
  * One-row strip of row r: up[r], row r, down[r+1].  Horizontal-bond ratios and O for the
    sites of row r use it.  Two-row strip of rows (r, r+1): up[r], rows r and r+1,
    down[r+2]; vertical and next-nearest-neighbour ratios use it.  Each ratio is the strip
    value at S' over the strip value at S, both with the same environments.
"""
import numpy as np

from . import philox
from .lattice import Lattice, spin_sys, spin_anc, sz_of


# ----------------------------------------------------------------------------- init

def init_theta(lat: Lattice, seed: int, noise: float) -> np.ndarray:
    """beta = 0 state (Eq. 1 at beta = 0 is rho = I, vectorised |I> has
    rho(S) = prod_i delta_{s_i s'_i}): the D = 1 tensors T_i^{S}[0,0,0,0] = delta_{s s'},
    padded to bond D; every zero entry perturbed by noise * (2u - 1), u uniform from
    Philox(seed; counter = (index lo, index hi, 0, TAG_INIT)) (App. A)."""
    idx = np.arange(lat.Np, dtype=np.uint64)
    u = philox.uniform(seed, idx & np.uint64(0xFFFFFFFF), idx >> np.uint64(32), np.zeros_like(idx),
                       philox.TAG_INIT)
    theta = noise * (2.0 * u - 1.0)
    for i in range(lat.N):
        off, sz = int(lat.theta_off[i]), lat.sz[i]
        theta[off + 0 * sz] = 1.0   # S = 0: s = s' = up
        theta[off + 3 * sz] = 1.0   # S = 3: s = s' = down
    return theta


def init_configs(lat: Lattice, seed: int, n_chains: int) -> np.ndarray:
    """Initial chain configurations: diagonal (s = s', the support of rho at beta = 0),
    s_i = low bit of Philox(seed; counter = (chain, site, 0, TAG_CFG)).  uint8 [n][N]."""
    ch = np.repeat(np.arange(n_chains, dtype=np.uint64), lat.N)
    st = np.tile(np.arange(lat.N, dtype=np.uint64), n_chains)
    b = philox.bits(seed, ch, st, np.zeros_like(ch), philox.TAG_CFG) & np.uint64(1)
    return (3 * b).astype(np.uint8).reshape(n_chains, lat.N)


# ------------------------------------------------------------- exact contraction (Eq. 4)

def row_tensors(lat, T, S, r):
    """Tensors T_{r,c}^{S_{r,c}}[l, r, u, d] of row r at configuration S."""
    return [T[lat.site(r, c)][int(S[lat.site(r, c)])] for c in range(lat.ncol)]


def amplitude_exact(lat: Lattice, theta, S) -> float:
    """rho_theta(S) of Eq. 4 by exact contraction, one tensor at a time (row-vector method).

    The running tensor v carries the down legs of the sites already absorbed in the
    current row, the open horizontal bond, and the up legs of the remaining sites."""
    T = lat.tensors(theta)
    n = lat.ncol
    v = np.ones([1] * n)                       # up legs of row 0 (dimension 1)
    for r in range(lat.nrow):
        v = v[np.newaxis]                      # open horizontal bond at the left edge (dim 1)
        # v legs: (h, u_0, ..., u_{n-1}); after site c: (d_0..d_c, h, u_{c+1}..u_{n-1})
        for c in range(n):
            A = T[lat.site(r, c)][int(S[lat.site(r, c)])]          # (l, r, u, d)
            v = np.tensordot(v, A, axes=([c, c + 1], [0, 2]))      # (d_<c, u_>c, r, d)
            v = np.moveaxis(v, [v.ndim - 1, v.ndim - 2], [c, c + 1])
        v = v.reshape(v.shape[:n])             # drop the right-edge bond (dimension 1)
    return float(v.reshape(()))


# ------------------------------------------------------------------- boundary MPS

def trivial_env(ncol):
    return [np.ones((1, 1, 1)) for _ in range(ncol)], 0.0


def absorb_down(env_tensors, row):
    """Row above a down environment: C_c[(a,l), u, (b,r)] = sum_d A[l,r,u,d] E[a,d,b]."""
    out = []
    for E, A in zip(env_tensors, row):
        C = np.einsum('lrud,adb->alubr', A, E)
        a, l, u, b, r = C.shape
        out.append(C.reshape(a * l, u, b * r))
    return out


def absorb_up(env_tensors, row):
    """Row below an up environment: C_c[(a,l), d, (b,r)] = sum_u E[a,u,b] A[l,r,u,d]."""
    out = []
    for E, A in zip(env_tensors, row):
        C = np.einsum('aub,lrud->aldbr', E, A)
        a, l, d, b, r = C.shape
        out.append(C.reshape(a * l, d, b * r))
    return out


def compress(mps, chi):
    """SVD truncation of an open MPS to bond chi in canonical form (see module docstring)."""
    n = len(mps)
    if max(t.shape[2] for t in mps) <= chi:
        return [t.copy() for t in mps]
    # (i) right-to-left: C_{>=c} = L_c Q_{>=c}
    Lf = [None] * (n + 1)
    Lf[n] = np.ones((1, 1))
    for c in range(n - 1, 0, -1):
        M = np.einsum('apb,bk->apk', mps[c], Lf[c + 1])
        M = M.reshape(M.shape[0], -1)
        _, rr = np.linalg.qr(M.T)            # M^T = q rr  ->  M = rr^T q^T  (LQ of M)
        Lf[c] = rr.T
    # (ii) left-to-right SVD truncation
    out = []
    carry = np.ones((1, 1))
    for c in range(n - 1):
        A = np.einsum('xa,apb->xpb', carry, mps[c])
        bp, p, bn = A.shape
        A2 = A.reshape(bp * p, bn)
        U, s, _ = np.linalg.svd(A2 @ Lf[c + 1], full_matrices=False)
        k = min(chi, len(s))
        out.append(U[:, :k].reshape(bp, p, k))
        carry = U[:, :k].T @ A2
    out.append(np.einsum('xa,apb->xpb', carry, mps[n - 1]))
    return out


def normalize(mps, logscale):
    """Divide each tensor by its max-abs entry, adding the logarithms to the log-scale."""
    out = []
    for t in mps:
        m = float(np.max(np.abs(t)))
        if m > 0.0:
            out.append(t / m)
            logscale += np.log(m)
        else:
            out.append(t.copy())
    return out, logscale


def down_envs(lat, T, S, chi):
    """down[r] for r = 1..nrow (down[nrow] trivial); each entry (tensors, logscale)."""
    envs = [None] * (lat.nrow + 1)
    envs[lat.nrow] = trivial_env(lat.ncol)
    for r in range(lat.nrow - 1, 0, -1):
        t, ls = envs[r + 1]
        C = compress(absorb_down(t, row_tensors(lat, T, S, r)), chi)
        envs[r] = normalize(C, ls)
    return envs


def up_envs(lat, T, S, chi):
    """up[r] for r = 0..nrow-1 (up[0] trivial); each entry (tensors, logscale)."""
    envs = [None] * lat.nrow
    envs[0] = trivial_env(lat.ncol)
    for r in range(1, lat.nrow):
        t, ls = envs[r - 1]
        C = compress(absorb_up(t, row_tensors(lat, T, S, r - 1)), chi)
        envs[r] = normalize(C, ls)
    return envs


# ------------------------------------------------------------------------- strips

def strip1_step(L, U, A, Dn):
    """L'[x,r,y] = sum L[a,l,b] U[a,u,x] A[l,r,u,d] Dn[b,d,y] (one column of a one-row strip)."""
    t = np.tensordot(L, U, axes=([0], [0]))                     # [l,b,u,x]
    t = np.tensordot(t, A, axes=([0, 2], [0, 2]))               # [b,x,r,d]
    return np.tensordot(t, Dn, axes=([0, 3], [0, 1]))           # [x,r,y]


def strip1_value(Ut, row, Dt):
    """One-row strip: sum over all bonds of up-env x row x down-env (no log-scales)."""
    L = np.ones((1, 1, 1))
    for U, A, Dn in zip(Ut, row, Dt):
        L = strip1_step(L, U, A, Dn)
    return float(L.reshape(()))


def strip1_partials(Ut, row, Dt):
    """Left partials L[c] (columns < c) and right partials R[c] (columns >= c)."""
    n = len(row)
    L = [np.ones((1, 1, 1))]
    for c in range(n):
        L.append(strip1_step(L[c], Ut[c], row[c], Dt[c]))
    R = [None] * (n + 1)
    R[n] = np.ones((1, 1, 1))
    for c in range(n - 1, -1, -1):
        # R[c][a,l,b] = sum U[a,u,x] A[l,r,u,d] Dn[b,d,y] R[c+1][x,r,y]
        t = np.tensordot(Dt[c], R[c + 1], axes=([2], [2]))          # [b,d,x,r]
        t = np.tensordot(row[c], t, axes=([1, 3], [3, 1]))          # [l,u,b,x]
        R[c] = np.tensordot(Ut[c], t, axes=([1, 2], [1, 3]))        # [a,l,b]
    return L, R


def strip2_value(Ut, row1, row2, Dt):
    """Two-row strip: up-env x row r x row r+1 x down-env."""
    L = np.ones((1, 1, 1, 1))
    for U, A1, A2, Dn in zip(Ut, row1, row2, Dt):
        # L'[x,r,s,y] = sum L[a,i,j,b] U[a,u,x] A1[i,r,u,m] A2[j,s,m,d] Dn[b,d,y]
        t = np.tensordot(L, U, axes=([0], [0]))                 # [i,j,b,u,x]
        t = np.tensordot(t, A1, axes=([0, 3], [0, 2]))          # [j,b,x,r,m]
        t = np.tensordot(t, A2, axes=([0, 4], [0, 2]))          # [b,x,r,s,d]
        L = np.tensordot(t, Dn, axes=([0, 4], [0, 1]))          # [x,r,s,y]
    return float(L.reshape(()))


# ------------------------------------------------------------- per-sample evaluation

def swap_sys(S, i, j):
    """S with the system spins of sites i and j exchanged (ancilla unchanged)."""
    Sp = np.array(S, dtype=np.int64)
    si, sj = Sp[i] // 2, Sp[j] // 2
    Sp[i] = 2 * sj + Sp[i] % 2
    Sp[j] = 2 * si + Sp[j] % 2
    return Sp


def swap_anc(S, i, j):
    """S with the ancilla spins of sites i and j exchanged (system unchanged)."""
    Sp = np.array(S, dtype=np.int64)
    ai, aj = Sp[i] % 2, Sp[j] % 2
    Sp[i] = 2 * (Sp[i] // 2) + aj
    Sp[j] = 2 * (Sp[j] // 2) + ai
    return Sp


def bond_ratio(lat, T, S, Sp, kind, i, up, down):
    """rho(S')/rho(S) for a change on a bond whose first site i lies in the upper row, from the strip
    the bond lies in: one-row strip of its row ('h'), else the two-row strip of its rows."""
    r = i // lat.ncol
    if kind == 'h':
        Ut, Dt = up[r][0], down[r + 1][0]
        num = strip1_value(Ut, row_tensors(lat, T, Sp, r), Dt)
        den = strip1_value(Ut, row_tensors(lat, T, S, r), Dt)
    else:
        Ut, Dt = up[r][0], down[r + 2][0]
        num = strip2_value(Ut, row_tensors(lat, T, Sp, r), row_tensors(lat, T, Sp, r + 1), Dt)
        den = strip2_value(Ut, row_tensors(lat, T, S, r), row_tensors(lat, T, S, r + 1), Dt)
    return num / den


def local_energy(lat, T, S, up, down):
    """E_loc of Eq. 9 split as E_sys + E_anc.  With H real symmetric (Eq. 12), H^T = H, so
    calH = H x I + I x H acts on the system spins s and the ancilla spins s' alike:
      E_sys(S) = sum_bonds J [S^z_i S^z_j + 1/2 * [s_i != s_j] * rho(S_sys-swap)/rho(S)]
    and E_anc the same on s'."""
    e_sys = e_anc = 0.0
    s, a = spin_sys(S), spin_anc(S)
    for (i, j, J, kind) in lat.bonds():
        e_sys += J * sz_of(s[i]) * sz_of(s[j])
        e_anc += J * sz_of(a[i]) * sz_of(a[j])
        if s[i] != s[j]:
            e_sys += 0.5 * J * bond_ratio(lat, T, S, swap_sys(S, i, j), kind, i, up, down)
        if a[i] != a[j]:
            e_anc += 0.5 * J * bond_ratio(lat, T, S, swap_anc(S, i, j), kind, i, up, down)
    return float(e_sys), float(e_anc)


def log_derivatives(lat, T, S, up, down):
    """Compressed O row (Eq. 8): for each site i of row r, the environment of T_i in the
    one-row strip of row r divided by that strip's value, i.e. d log rho / d T_i^{S_i}."""
    O = np.zeros(lat.No)
    for r in range(lat.nrow):
        Ut, Dt = up[r][0], down[r + 1][0]
        row = row_tensors(lat, T, S, r)
        L, R = strip1_partials(Ut, row, Dt)
        val = float(L[lat.ncol].reshape(()))
        for c in range(lat.ncol):
            # env[l,r,u,d] = sum L[a,l,b] U[a,u,x] Dn[b,d,y] R[x,r,y]
            t = np.tensordot(L[c], Ut[c], axes=([0], [0]))          # [l,b,u,x]
            t = np.tensordot(t, R[c + 1], axes=([3], [0]))          # [l,b,u,r,y]
            t = np.tensordot(t, Dt[c], axes=([1, 4], [0, 2]))       # [l,u,r,d]
            env = t.transpose(0, 2, 1, 3)
            i = lat.site(r, c)
            O[lat.o_off[i]:lat.o_off[i + 1]] = env.ravel() / val
    return O


def eval_sample(lat, theta, S, chi, with_O=True):
    """Amplitude (log|rho|, sign), E_sys, E_anc and the compressed O row of one sample."""
    T = lat.tensors(theta)
    S = np.asarray(S, dtype=np.int64)
    down = down_envs(lat, T, S, chi)
    up = up_envs(lat, T, S, chi)
    val = strip1_value(up[0][0], row_tensors(lat, T, S, 0), down[1][0])
    log_abs = (np.log(abs(val)) if val != 0.0 else -np.inf) + down[1][1]
    e_sys, e_anc = local_energy(lat, T, S, up, down)
    O = log_derivatives(lat, T, S, up, down) if with_O else None
    return dict(log_abs=float(log_abs), sign=int(np.sign(val)), e_sys=e_sys, e_anc=e_anc, O=O)


def row_amplitudes(lat, theta, S, chi):
    """log|rho_r| of every one-row strip (all equal when chi is exact)."""
    T = lat.tensors(theta)
    down = down_envs(lat, T, S, chi)
    up = up_envs(lat, T, S, chi)
    out = []
    for r in range(lat.nrow):
        v = strip1_value(up[r][0], row_tensors(lat, T, S, r), down[r + 1][0])
        out.append(np.log(abs(v)) + up[r][1] + down[r + 1][1])
    return np.array(out)
