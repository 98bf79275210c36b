"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel
random numbers: as easy as 1, 2, 3"), written from its published definition.

TEST INFRASTRUCTURE (oracle): see oracle/__init__.py.

The method draws random numbers in two places: the perturbation of the zero entries of
the beta=0 PEPS (App. A) and the Metropolis acceptance tests (Sec. II, MCMC).  Both the
oracle and the CUDA path draw them from this generator, each side with its own code.

Round function (one of ten): with multipliers M0, M1 and key words (k0, k1)
    (hi0, lo0) = M0 * c0,   (hi1, lo1) = M1 * c2            (64-bit products)
    c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
and the key is bumped by the Weyl constants (W0, W1) between rounds.

Uniform double from one output block: u = ((x0 << 21) | (x1 >> 11)) * 2^-53 in [0, 1).
"""
import numpy as np

MASK32 = 0xFFFFFFFF
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

# Tags in the fourth counter word separate the independent random streams.
TAG_INIT = 0x494E4954   # initial-state perturbation
TAG_CFG = 0x43464731    # initial chain configurations
TAG_MC = 0x4D435357     # Metropolis acceptance uniforms


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block.  ctr: 4 uint32 (ints or equal-shape uint64 arrays);
    key: 2 uint32.  Returns the 4 output words in the same form."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) for x in ctr)
    k0, k1 = (np.uint64(int(k) & MASK32) for k in key)
    m32 = np.uint64(MASK32)
    sh = np.uint64(32)
    for rnd in range(10):
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> sh, p0 & m32
        hi1, lo1 = p1 >> sh, p1 & m32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m32, lo1, (hi0 ^ c3 ^ k1) & m32, lo0
        if rnd < 9:
            k0 = (k0 + np.uint64(PHILOX_W0)) & m32
            k1 = (k1 + np.uint64(PHILOX_W1)) & m32
    return c0, c1, c2, c3


def seed_key(seed):
    """Key words from a 64-bit seed: (low 32 bits, high 32 bits)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & MASK32, seed >> 32)


def uniform(seed, c0, c1, c2, tag):
    """Uniform double(s) in [0, 1) from counter (c0, c1, c2, tag) under key(seed)."""
    x0, x1, _, _ = philox4x32_10((c0, c1, c2, np.full(np.shape(c0), tag, dtype=np.uint64)),
                                 seed_key(seed))
    u53 = (x0 << np.uint64(21)) | (x1 >> np.uint64(11))
    return u53.astype(np.float64) * 2.0 ** -53


def bits(seed, c0, c1, c2, tag):
    """First output word(s) of the block (c0, c1, c2, tag), as uint64."""
    x0, _, _, _ = philox4x32_10((c0, c1, c2, np.full(np.shape(c0), tag, dtype=np.uint64)),
                                seed_key(seed))
    return x0
