"""Metropolis sampling and stochastic reconfiguration of the fermionic thermal state: the
Monte Carlo loop of Sec. II (MCMC, Eqs. 5-10) on the fermionic PEPS of Fig. 1b for the
Hubbard model of Sec. III.B (Eq. 14).

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.  Amplitudes, local energies and
log-derivatives come from oracle/fermion.py; the SR algebra from oracle/sr.py.

Readings (the paper states neither the moves nor the observables' estimators for fermions):
  * Moves.  A configuration holds sixteen-valued local indices S_i (bits: c_up, c_dn, d_up,
    d_dn).  Two kinds of proposal:
      (i)  pair: at site i and spin s (up, then down), where c_s and d_s are equally
           occupied, toggling both (a system-ancilla pair created or removed:
           S_i ^= 0b101 << s);
      (ii) hop: across a nearest-neighbour bond (i, j) and for mode k = 0..3 (c_up, c_dn,
           d_up, d_dn), exchanging the occupations of mode k at the two sites (one electron
           hops).
    One sweep visits the rows top to bottom: in row r, for every column c the pairs of site
    (r, c) and then the hops of its horizontal bond to (r, c+1); then, for every column, the
    hops of the vertical bond from (r, c) to (r+1, c) (the order of a sweep over row strips).
    A proposal whose condition fails (c_s != d_s in (i), equal occupations in (ii)) is
    skipped, its uniform unused.  Every move keeps the total parity even (a PEPS of even
    tensors vanishes elsewhere) and is its own inverse where it applies, so proposals are
    symmetric.  Both keep N_s(c) - N_s(d); from any configuration with N_s(c) = N_s(d) for
    both spins, hops align the ancilla electrons with the system ones and (i) removes the
    pairs, so the moves connect exactly the configurations with N_s(c) = N_s(d): the support
    of e^(-t calH)|I> (tests pin this).
  * Acceptance: target |psi|^p; accept iff log u < p (log|psi(S')| - log|psi(S)|), in float64;
    psi(S') = 0 is rejected.
  * Uniforms: the move m of sweep k of chain c draws u = Philox4x32-10(seed; counter = (c, k,
    m, TAG_FMC)).
  * Estimators (Eq. 11 with the weights of oracle/sr.py): E/N = sum_i w_i (E_sys,i +
    E_anc,i)/2 / N with its delta-method error; the double occupancy and the density per site
    are the weighted means of sum_j n_up n_dn and sum_j (n_up + n_dn), averaged over the two
    layers (for |rho|^2 weights both layers carry the same distribution).
  * Parameters: theta is the concatenation over sites (row-major) of T_i[16][dl][dr][du][dd].
"""
import numpy as np

from . import fermion as fm
from . import observables as obs_mod
from . import philox
from . import sr as sr_mod

TAG_FMC = 0x464D4331   # fermionic Metropolis acceptance uniforms


# ---------------------------------------------------------------- moves and the sweep

def moves(nrow, ncol):
    """The proposals of one sweep in order: per row, ('pair', i, s) and the horizontal
    ('hop', i, i + 1, k) column by column, then the vertical ('hop', i, i + ncol, k)."""
    out = []
    for r in range(nrow):
        for c in range(ncol):
            i = r * ncol + c
            out.extend(("pair", i, s) for s in (0, 1))
            if c + 1 < ncol:
                out.extend(("hop", i, i + 1, k) for k in range(4))
        if r + 1 < nrow:
            for c in range(ncol):
                i = r * ncol + c
                out.extend(("hop", i, i + ncol, k) for k in range(4))
    return out


def propose(S, move):
    """The configuration a move proposes, or None where it changes nothing."""
    S2 = [int(x) for x in S]
    if move[0] == "pair":
        _, i, s = move
        if ((S2[i] >> s) & 1) != ((S2[i] >> (2 + s)) & 1):
            return None
        S2[i] ^= (1 << s) | (1 << (2 + s))
        return S2
    _, i, j, k = move
    if ((S2[i] >> k) & 1) == ((S2[j] >> k) & 1):
        return None
    S2[i] ^= 1 << k
    S2[j] ^= 1 << k
    return S2


def uniforms(seed, chain, sweep_index, n_moves):
    """u of every move of one sweep of one chain."""
    m = np.arange(n_moves, dtype=np.uint64)
    return philox.uniform(seed, np.full(n_moves, chain, dtype=np.uint64),
                          np.full(n_moves, sweep_index, dtype=np.uint64), m, TAG_FMC)


def _log_abs(a):
    return np.log(abs(a)) if a != 0.0 else -np.inf


def sweep(nrow, ncol, T, S, p, u, amplitude=None):
    """One sweep of one chain with the uniforms u (one per move).  Returns (S, accepted,
    margin): margin is the smallest |log u - p (log|psi'| - log|psi|)| over the decisions
    taken (how close a decision came to its threshold)."""
    amp = amplitude or fm.fpeps_amplitude_function(nrow, ncol, T)
    S = [int(x) for x in S]
    la = _log_abs(amp(S))
    acc = 0
    margin = np.inf
    for m, mv in enumerate(moves(nrow, ncol)):
        S2 = propose(S, mv)
        if S2 is None:
            continue
        a2 = amp(S2)
        if a2 == 0.0:
            continue
        la2 = np.log(abs(a2))
        d = np.log(u[m]) - p * (la2 - la)
        if np.isfinite(d):
            margin = min(margin, abs(d))
        if d < 0:
            S, la = S2, la2
            acc += 1
    return np.array(S, dtype=np.uint8), acc, margin


def transition_matrix(nrow, ncol, psi_of, states, p):
    """The exact transition matrix of one sweep over `states` (a list of configurations
    closed under the moves): the product over moves, in sweep order, of the single-move
    Metropolis matrices (accept with probability min(1, |psi'/psi|^p))."""
    index = {tuple(s): n for n, s in enumerate(states)}
    n = len(states)
    P = np.eye(n)
    for mv in moves(nrow, ncol):
        Pm = np.zeros((n, n))
        for a, s in enumerate(states):
            s2 = propose(s, mv)
            pa = abs(psi_of(s))
            if s2 is None or pa == 0.0:
                Pm[a, a] = 1.0
                continue
            b = index[tuple(s2)]
            q = min(1.0, (abs(psi_of(s2)) / pa) ** p)
            Pm[a, b] = q
            Pm[a, a] += 1.0 - q
        P = P @ Pm
    return P


# ---------------------------------------------------------------- SR on sampled configurations

def theta_offsets(T):
    """Offset of every site's block in theta and the size of one of its sixteen slices."""
    off = [0]
    sz = []
    for A in T:
        sz.append(int(np.prod(A.shape[1:])))
        off.append(off[-1] + A.size)
    return off, sz


def flatten(T):
    return np.concatenate([A.ravel() for A in T])


def unflatten(theta, like):
    out = []
    off = 0
    for A in like:
        out.append(np.asarray(theta[off:off + A.size], dtype=np.float64).reshape(A.shape))
        off += A.size
    return out


def sample_quantities(nrow, ncol, T, S_batch, t_hop, U, mu):
    """log|psi|, sign, E_sys, E_anc and the compressed O row (sites' derivatives at S_i
    concatenated) of every configuration."""
    la, sg, es, ea, rows = [], [], [], [], []
    for S in S_batch:
        grads, psi = fm.fpeps_log_derivative(nrow, ncol, T, S)
        e_s, e_a = fm.fpeps_local_energy(nrow, ncol, T, S, t_hop, U, mu)
        la.append(np.log(abs(psi)))
        sg.append(np.sign(psi))
        es.append(e_s)
        ea.append(e_a)
        rows.append(np.concatenate([g.ravel() for g in grads]))
    return np.array(la), np.array(sg), np.array(es), np.array(ea), np.array(rows)


def expand_O(T, S_batch, rows):
    """Dense O (N_s x N_p): the site-j part of row n at theta_off_j + S_nj sz_j."""
    off, sz = theta_offsets(T)
    Of = np.zeros((len(S_batch), off[-1]))
    for n, S in enumerate(S_batch):
        o = 0
        for j in range(len(T)):
            t0 = off[j] + int(S[j]) * sz[j]
            Of[n, t0:t0 + sz[j]] = rows[n, o:o + sz[j]]
            o += sz[j]
    return Of


def observables(N, S_batch, w, es, ea):
    """E/N, its standard error, the double occupancy and the density per site."""
    h = 0.5 * (np.asarray(es) + np.asarray(ea))
    H1 = float(w @ h)
    err = obs_mod.standard_error(w, h)
    docc = np.zeros(len(S_batch))
    dens = np.zeros(len(S_batch))
    for n, S in enumerate(S_batch):
        for x in S:
            x = int(x)
            for layer in (0, 1):
                nu, nd = (x >> (2 * layer)) & 1, (x >> (2 * layer + 1)) & 1
                docc[n] += 0.5 * nu * nd
                dens[n] += 0.5 * (nu + nd)
    return {"E_site": H1 / N, "E_err": err / N, "docc": float(w @ docc) / N,
            "density": float(w @ dens) / N}


def sr_step(nrow, ncol, T, S_batch, t_hop, U, mu, p, tau, eps, tol, maxit, log_q=None):
    """One SR update of the fermionic PEPS from the configurations S_batch (Eqs. 5-10):
    weights of oracle/sr.py, E = E_sys + E_anc, the mean, gradient and CG solve in the full
    parameter space, theta' = theta - tau x.  Returns (T', x, g, iterations, residual,
    observables before the update)."""
    la, sg, es, ea, rows = sample_quantities(nrow, ncol, T, S_batch, t_hop, U, mu)
    w = sr_mod.weights(la, p, log_q)
    Of = expand_O(T, S_batch, rows)
    obar, _, g = sr_mod.sr_quantities(Of, w, es + ea)
    x, it, res = sr_mod.cg(lambda v: sr_mod.apply_G(Of, w, obar, v, eps), g, tol, maxit)
    obs = observables(nrow * ncol, S_batch, w, es, ea)
    return unflatten(flatten(T) - tau * x, T), x, g, it, res, obs
