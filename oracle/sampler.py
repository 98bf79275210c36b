"""Metropolis sampling of the vectorised density matrix.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

Sec. II samples configurations S with weight |rho(S)|^2 by MCMC; App. A (Eq. A1) samples
|rho(S)| instead at high temperature and reweights by r_1 = |rho|.  Both are the
acceptance test u < |rho(S')/rho(S)|^p with p = 2 or p = 1.

The paper does not state the proposal moves.  One sweep here visits the rows top to
bottom; in row r:
  phase H (one-row strip up[r], row r, down[r+1]), for c = 0..ncol-1:
      move 0  both-flip of site (r,c): (s, s') -> (1-s, 1-s'), i.e. S -> 3 - S;
      move 1  exchange of the system spins of (r,c) and (r,c+1) if they differ;
      move 2  exchange of the ancilla spins of (r,c) and (r,c+1) if they differ;
  phase V (two-row strip up[r], rows r and r+1, down[r+2]; r < nrow-1), for each c:
      move 3  exchange of the system spins of (r,c) and (r+1,c) if they differ;
      move 4  exchange of the ancilla spins of (r,c) and (r+1,c) if they differ;
  then row r (final) is absorbed into the up environment.
down[] is built once at the start of the sweep (rows below the one being updated are
still unchanged when they are used).  Move m at site (r,c) has id (r*ncol + c)*8 + m and
draws u = Philox(seed; counter = (chain, sweep, id, TAG_MC)).  The ratio is the strip
value at S' over the strip value at the current S, both with the same environments.
"""
import numpy as np

from . import philox
from .peps import (absorb_up, compress, down_envs, normalize, row_tensors, strip1_value,
                   strip2_value, swap_anc, swap_sys, trivial_env)


def accept(u, ratio, p):
    """Metropolis test for target |rho|^p: accept iff u < |ratio|^p."""
    q = ratio * ratio if p == 2 else abs(ratio)
    return u < q


def mc_sweep(lat, theta, S, chi, p, seed, chain, sweep):
    """One sweep of one chain.  Returns (new S, accepted, proposed)."""
    T = lat.tensors(theta)
    S = np.array(S, dtype=np.int64)
    down = down_envs(lat, T, S, chi)
    up_t, up_ls = trivial_env(lat.ncol)
    n_acc = n_prop = 0

    def try_move(Sp, mid, value):
        nonlocal S, n_acc, n_prop
        ratio = value(Sp) / value(S)
        u = float(philox.uniform(seed, chain, sweep, mid, philox.TAG_MC))
        n_prop += 1
        if accept(u, ratio, p):
            S = Sp
            n_acc += 1

    for r in range(lat.nrow):
        Dt = down[r + 1][0]
        v1 = lambda X: strip1_value(up_t, row_tensors(lat, T, X, r), Dt)
        for c in range(lat.ncol):
            i = lat.site(r, c)
            base = i * 8
            Sp = S.copy()
            Sp[i] = 3 - Sp[i]
            try_move(Sp, base + 0, v1)
            if c < lat.ncol - 1:
                j = lat.site(r, c + 1)
                if S[i] // 2 != S[j] // 2:
                    try_move(swap_sys(S, i, j), base + 1, v1)
                if S[i] % 2 != S[j] % 2:
                    try_move(swap_anc(S, i, j), base + 2, v1)
        if r < lat.nrow - 1:
            D2 = down[r + 2][0]
            v2 = lambda X: strip2_value(up_t, row_tensors(lat, T, X, r),
                                        row_tensors(lat, T, X, r + 1), D2)
            for c in range(lat.ncol):
                i, j = lat.site(r, c), lat.site(r + 1, c)
                base = i * 8
                if S[i] // 2 != S[j] // 2:
                    try_move(swap_sys(S, i, j), base + 3, v2)
                if S[i] % 2 != S[j] % 2:
                    try_move(swap_anc(S, i, j), base + 4, v2)
            C = compress(absorb_up(up_t, row_tensors(lat, T, S, r)), chi)
            up_t, up_ls = normalize(C, up_ls)
    return S.astype(np.uint8), n_acc, n_prop


def run_chains(lat, theta, S_batch, chi, p, seed, sweep0, n_sweeps):
    """n_sweeps sweeps of every chain; sweep numbers sweep0 .. sweep0 + n_sweeps - 1."""
    S_batch = np.array(S_batch, dtype=np.uint8)
    acc = prop = 0
    for ch in range(S_batch.shape[0]):
        for k in range(n_sweeps):
            S_batch[ch], a, b = mc_sweep(lat, theta, S_batch[ch], chi, p, seed, ch, sweep0 + k)
            acc += a
            prop += b
    return S_batch, acc, prop
