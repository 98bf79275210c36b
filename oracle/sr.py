"""Stochastic reconfiguration step (Sec. II, Eqs. 5-7 and 10) on a fixed set of samples.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

  weights   p = 2 (samples of |rho|^2): w_i = 1/N_s.
            p = 1 (samples of |rho|, Eq. A1): w_i = r_1(S_i) / sum_j r_1(S_j), r_1 = |rho|.
            p = 0 (direct draws of probability q, App. A Eq. A7): w_i = r_4(S_i) / sum_j
            r_4(S_j), r_4 = p_0 / q = |rho|^2 / q (oracle/direct.py, first reading).
  metric    G_kk' = <O_k O_k'> - <O_k><O_k'> (Eq. 6), written for samples as Eq. 10.
  gradient  g_k = <O_k E_loc> - <O_k><E_loc> (Eq. 7), E_loc the full calH local energy.
  solve     (G + eps I) x = g by conjugate gradient, x_0 = 0; G is applied as two passes
            over the samples, (O_i - o_bar).v then sum_i w_i t_i (O_i - o_bar) (Sec. II,
            normal-equation CG).  eps is an absolute shift (the paper states none).
  update    theta' = theta - tau x (Eq. 5).
All vectors here live in the full parameter space (the compressed O rows are expanded).
"""
import numpy as np


def weights(log_abs, p, log_q=None):
    log_abs = np.asarray(log_abs, dtype=np.float64)
    n = log_abs.shape[0]
    if p == 2:
        return np.full(n, 1.0 / n)
    if p == 0:
        lr = 2.0 * log_abs - np.asarray(log_q, dtype=np.float64)
        r4 = np.exp(lr - np.max(lr))
        return r4 / np.sum(r4)
    r1 = np.exp(log_abs - np.max(log_abs))
    return r1 / np.sum(r1)


def expand_O(lat, S_batch, O_rows):
    """Dense O (N_s x N_p): O_i[theta_off_j + S_ij * sz_j + k] = O_rows[i, o_off_j + k]."""
    ns = O_rows.shape[0]
    Of = np.zeros((ns, lat.Np))
    for j in range(lat.N):
        sz = lat.sz[j]
        for i in range(ns):
            t0 = lat.theta_off[j] + int(S_batch[i, j]) * sz
            Of[i, t0:t0 + sz] = O_rows[i, lat.o_off[j]:lat.o_off[j + 1]]
    return Of


def sr_quantities(Of, w, E):
    """o_bar = <O>, E_bar = <E>, g of Eq. 7."""
    obar = w @ Of
    Ebar = float(w @ E)
    g = w @ (Of * E[:, None]) - obar * Ebar
    return obar, Ebar, g


def apply_G(Of, w, obar, v, eps):
    """(G + eps I) v with G = sum_i w_i (O_i - o_bar)(O_i - o_bar)^T, two passes (Eq. 10)."""
    t = (Of - obar) @ v
    return (Of - obar).T @ (w * t) + eps * v


def dense_G(Of, w, obar, eps):
    C = Of - obar
    return C.T @ (w[:, None] * C) + eps * np.eye(Of.shape[1])


def cg(apply, b, tol, maxit):
    """Textbook conjugate gradient from x_0 = 0.  Before each iteration the relative
    residual |r|/|b| is tested against tol.  Returns (x, iterations, relative residual)."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(r @ r)
    bnorm = np.sqrt(float(b @ b))
    it = 0
    while it < maxit and np.sqrt(rr) > tol * bnorm:
        q = apply(p)
        alpha = rr / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        rr_new = float(r @ r)
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it, (np.sqrt(rr) / bnorm if bnorm > 0 else 0.0)


def sr_step(lat, theta, S_batch, log_abs, e_sys, e_anc, O_rows, p, tau, eps, tol, maxit,
            log_q=None):
    """One SR update (p = 0: direct draws with log q given).  Returns (theta', x, g, cg
    iterations, relative residual)."""
    w = weights(log_abs, p, log_q)
    E = np.asarray(e_sys) + np.asarray(e_anc)
    Of = expand_O(lat, S_batch, O_rows)
    obar, _, g = sr_quantities(Of, w, E)
    x, it, res = cg(lambda v: apply_G(Of, w, obar, v, eps), g, tol, maxit)
    return np.asarray(theta) - tau * x, x, g, it, res
