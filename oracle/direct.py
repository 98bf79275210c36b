"""Direct (autoregressive) sampling of the doubled-lattice PEPS and its reweighted form.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

Definitions followed (arXiv:2409.05285, App. A, after Eq. A1):
  * p_0(S) = |rho(S)|^2 is the weight of the standard estimator.
  * Direct sampling draws the sites one after another: p_2(S) = prod_i p_2c(S_i | S_<i)
    (Eq. A2), where p_2c(S_i | S_<i) is the sum of p_0 over the unsampled sites S_>i
    divided by its sum over S_>=i (Eq. A3).  Then p_2 = p_0 / sum_S p_0.
  * Reweighted: p_3c = sqrt(p_2c) (Eq. A4) and p_4c = b(S_i) p_3c (Eq. A5) with
    b(s s') = 1 for s != s' and a value b_d for s = s' that is adjusted every gradient
    step so that diagonal samples stay at most half of the batch; p_4 = prod_i p_4c
    (Eq. A6); <f>_{p_0} = <f r_4>_{p_4} / <r_4>_{p_4} with r_4 = p_0 / p_4 (Eq. A7).

Readings (the appendix leaves these open):
  * Site order: row-major, site i = r * ncol + c (the order of the boundary-MPS rows).
  * p_3c and p_4c do not sum to one over S_i.  A site is drawn from p_4c normalised over its
    four values, so the distribution actually sampled is
        q(S) = prod_i p_4c(S_i | S_<i) / sum_s p_4c(s | S_<i),
    and the weight of Eq. A7 is r_4 = p_0 / q.  (Eq. A7 is a ratio estimator, so constant
    factors cancel; with q the estimate is exact in expectation.)  For b_d = 1 and the
    exponent 1 instead of 1/2 this is plain direct sampling, q = p_2.
  * The sum of p_0 over unsampled sites is the double-layer network: site j carries
    T_j^{S_j} (x) T_j^{S_j} when sampled and sum_S T_j^S (x) T_j^S otherwise (real tensors:
    rho^2 = rho rho), with bonds of dimension D^2.  Here it is contracted exactly by the
    row-vector method (small lattices only).
  * A "diagonal term" is a sample with s = s' on every site (a diagonal entry of rho).
    After a step whose samples hold a fraction f_d > 1/2 of diagonal terms, b_d is
    multiplied by (1/2 / f_d)^(1/N): the diagonal fraction scales like b_d^N, so this aims
    it at one half; otherwise b_d is left unchanged.  b_d never exceeds 1.
  * Uniform numbers are inputs (one per site and sample), drawn by the caller.
"""
import numpy as np

from .peps import (absorb_down, absorb_up, amplitude_exact, compress, normalize, strip1_partials,
                   strip1_step, trivial_env)


def double_layer(lat, theta, fixed):
    """Site tensors of the double-layer network, shape (dl^2, dr^2, du^2, dd^2): the
    product T^S (x) T^S at a site with fixed[i] = S, the sum over S where fixed[i] < 0."""
    T = lat.tensors(theta)
    out = []
    for i in range(lat.N):
        dl, dr, du, dd = lat.dims[i]
        if fixed[i] >= 0:
            A = T[i][int(fixed[i])]
            E = np.einsum('lrud,LRUD->lLrRuUdD', A, A)
        else:
            E = np.einsum('slrud,sLRUD->lLrRuUdD', T[i], T[i])
        out.append(E.reshape(dl * dl, dr * dr, du * du, dd * dd))
    return out


def marginal(lat, theta, fixed):
    """Sum of rho(S)^2 over the sites with fixed[i] < 0, the others held at fixed[i]:
    exact contraction of the double-layer network (row-vector method, as for Eq. 4)."""
    E = double_layer(lat, theta, fixed)
    n = lat.ncol
    v = np.ones([1] * n)
    for r in range(lat.nrow):
        v = v[np.newaxis]
        for c in range(n):
            A = E[lat.site(r, c)]                                  # (l, r, u, d)
            v = np.tensordot(v, A, axes=([c, c + 1], [0, 2]))
            v = np.moveaxis(v, [v.ndim - 1, v.ndim - 2], [c, c + 1])
        v = v.reshape(v.shape[:n])
    return float(v.reshape(()))


def conditional(lat, theta, prefix):
    """p_2c(s | S_<i) for s = 0..3 at site i = len(prefix) (Eq. A3); zeros when the prefix
    has zero weight."""
    i = len(prefix)
    fixed = -np.ones(lat.N, dtype=np.int64)
    fixed[:i] = prefix
    m = np.empty(4)
    for s in range(4):
        fixed[i] = s
        m[s] = marginal(lat, theta, fixed)
    tot = m.sum()
    return m / tot if tot > 0 else np.zeros(4)


def site_weights(p2c, b_d, exponent):
    """p_4c(s) = b(s) p_2c(s)^exponent (Eqs. A4-A5 with exponent 1/2; exponent 1 and b_d = 1
    give plain direct sampling), b(s) = b_d for the diagonal local states s = s' (S = 0, 3)."""
    b = np.array([b_d, 1.0, 1.0, b_d])
    return b * p2c ** exponent


def draw(lat, theta, u, b_d=1.0, exponent=0.5):
    """One sample: sites in row-major order, site i drawn from p_4c normalised over its four
    values by inverse CDF with u[i].  Returns (S, log q(S), log p_0(S))."""
    S = np.zeros(lat.N, dtype=np.int64)
    logq = 0.0
    for i in range(lat.N):
        w = site_weights(conditional(lat, theta, S[:i]), b_d, exponent)
        w = w / w.sum()
        cdf = np.cumsum(w)
        s = int(np.searchsorted(cdf, u[i] * cdf[-1], side='right'))
        s = min(s, 3)
        while w[s] == 0.0:       # u at the top edge of the CDF: the last state of weight > 0
            s -= 1
        S[i] = s
        logq += np.log(w[s])
    amp = amplitude_exact(lat, theta, S)
    return S, logq, 2.0 * np.log(abs(amp))


def sample_prob(lat, theta, S, b_d=1.0, exponent=0.5):
    """q(S): the probability that draw() returns S."""
    q = 1.0
    for i in range(lat.N):
        w = site_weights(conditional(lat, theta, S[:i]), b_d, exponent)
        tot = w.sum()
        if tot == 0.0:
            return 0.0
        q *= w[int(S[i])] / tot
    return q


def reweighted_mean(f, logq, logp0):
    """<f>_{p_0} from samples of q (Eq. A7 with r_4 = p_0 / q)."""
    lr = np.asarray(logp0) - np.asarray(logq)
    r = np.exp(lr - lr.max())
    return float(np.sum(r * np.asarray(f)) / np.sum(r))


def diagonal_fraction(S_batch):
    """Fraction of samples with s = s' on every site."""
    S_batch = np.asarray(S_batch)
    diag = np.all((S_batch // 2) == (S_batch % 2), axis=1)
    return float(diag.mean())


def update_bd(b_d, S_batch, N):
    """b_d after a step whose samples are S_batch (see the module docstring)."""
    f = diagonal_fraction(S_batch)
    if f > 0.5:
        b_d = b_d * (0.5 / f) ** (1.0 / N)
    return min(b_d, 1.0)


# ------------------------------------------------- boundary-MPS form (the method's steps)
#
# The sums over unsampled sites are double-layer contractions, so the boundary-MPS scheme of
# Sec. III.A (with the truncation reading of peps.compress) applies with bonds D^2:
#   * down[r] (rows r..nrow-1, every site summed) does not depend on the sample: built once;
#   * row by row, up[r] holds the sampled rows above (site tensors T^S (x) T^S);
#   * in row r the sites left of c are sampled, site c takes each candidate state, the sites
#     right of c are summed: the candidate's weight is the one-row strip
#     (up[r], row r, down[r+1]), evaluated as left partial x site x right partial;
#   * after the row is drawn it is absorbed into up[r+1] and truncated to chi.
# At chi >= the largest exact bond this equals the exact form above.

def _rows(lat, E):
    return [[E[lat.site(r, c)] for c in range(lat.ncol)] for r in range(lat.nrow)]


def summed_down_envs(lat, theta, chi):
    """down[r] of the double layer with every site summed, r = 1..nrow (down[nrow] trivial)."""
    rows = _rows(lat, double_layer(lat, theta, -np.ones(lat.N, dtype=np.int64)))
    envs = [None] * (lat.nrow + 1)
    envs[lat.nrow] = trivial_env(lat.ncol)
    for r in range(lat.nrow - 1, 0, -1):
        t, ls = envs[r + 1]
        envs[r] = normalize(compress(absorb_down(t, rows[r]), chi), ls)
    return envs


def draw_bmps(lat, theta, u, chi, b_d=1.0, exponent=0.5, down=None):
    """draw() with the marginals from boundary-MPS environments at bond chi.  Returns
    (S, log q(S)); q is the probability of the draw under these (truncated) marginals."""
    if down is None:
        down = summed_down_envs(lat, theta, chi)
    T = lat.tensors(theta)
    summed = double_layer(lat, theta, -np.ones(lat.N, dtype=np.int64))
    S = np.zeros(lat.N, dtype=np.int64)
    logq = 0.0
    up, ls_up = trivial_env(lat.ncol)
    for r in range(lat.nrow):
        Dt = down[r + 1][0]
        row_sum = [summed[lat.site(r, c)] for c in range(lat.ncol)]
        _, R = strip1_partials(up, row_sum, Dt)
        L = np.ones((1, 1, 1))
        fixed_row = []
        for c in range(lat.ncol):
            i = lat.site(r, c)
            m = np.empty(4)
            cand = []
            for s in range(4):
                A = T[i][s]
                dl, dr, du, dd = lat.dims[i]
                E = np.einsum('lrud,LRUD->lLrRuUdD', A, A).reshape(dl * dl, dr * dr, du * du, dd * dd)
                Ls = strip1_step(L, up[c], E, Dt[c])
                m[s] = float(np.tensordot(Ls, R[c + 1], axes=([0, 1, 2], [0, 1, 2])))
                cand.append((E, Ls))
            m = np.maximum(m, 0.0)          # truncation can leave tiny negative sums
            p2c = m / m.sum() if m.sum() > 0 else np.zeros(4)
            w = site_weights(p2c, b_d, exponent)
            w = w / w.sum()
            cdf = np.cumsum(w)
            s = min(int(np.searchsorted(cdf, u[i] * cdf[-1], side='right')), 3)
            while w[s] == 0.0:
                s -= 1
            S[i] = s
            logq += np.log(w[s])
            fixed_row.append(cand[s][0])
            L = cand[s][1]
        if r < lat.nrow - 1:
            up, ls_up = normalize(compress(absorb_up(up, fixed_row), chi), ls_up)
    return S, logq
