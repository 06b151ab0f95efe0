"""Oracle: counter-based Philox4x32-10 and the Gaussian test matrix it defines.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper draws one random projection matrix P (N x l) per decomposition and
performs a single run ("Randomized matrix decompositions" paragraph, Fig. 1
step 1).  To compare a GPU run with this oracle on the *same* draw, the matrix
is fixed by a counter-based generator: entry (i, j) depends only on
(seed, i, j, tag), never on how the work is split.

Philox4x32-10 follows the round function of Salmon et al., SC'11, Sec. 3
("Philox"): each of 10 rounds takes the 128-bit counter as four 32-bit words
(c0, c1, c2, c3), forms the two 64-bit products M0*c0 and M1*c2, and emits
(hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1, lo(M0*c0)); the 64-bit
key (k0, k1) is bumped by the Weyl constants between rounds.

Gaussian entries:
  * FP64 form (the all-FP64 path): the four output words w0..w3 give two
    53-bit uniforms u1 = ((w0 >> 5) * 2^26 + (w1 >> 6) + 1/2) * 2^-53 and
    u2 likewise from (w2, w3); the entry is sqrt(-2 ln u1) cos(2 pi u2)
    (Box & Muller, Ann. Math. Stat. 29, 1958).
  * FP32 form (the mixed-precision path): 24-bit uniforms from the top bits of
    w0 and w2, u = ((w >> 8) + 1/2) * 2^-24, same Box-Muller formula.  Its
    values agree with the FP64 form to about 1e-6 relative; the mixed path
    rounds them to BF16 anyway.

Counter layout: (c0, c1, c2, c3) = (row i, column j, tag, 0); key = (seed low
32 bits, seed high 32 bits).  Tags separate independent streams:
TAG_OMEGA (sketch columns), TAG_PROBE (16-column probe sketch and residual
probes), TAG_NOISE (tile-rule noise, see ``tilerule``).

Parity: pinned by the published known-answer vectors of Philox4x32-10 and by
the first four moments of the Gaussian output (tests/test_oracle_philox.py).
"""

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

TAG_OMEGA = 0
TAG_PROBE = 1
TAG_NOISE = 2
TAG_RESID = 3


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counter words.

    All arguments are broadcastable integer arrays (values < 2^32).  Returns a
    tuple of four uint64 arrays holding the 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = np.uint64(k0 & MASK32)
    k1 = np.uint64(k1 & MASK32)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    for r in range(10):
        if r > 0:
            k0 = np.uint64((int(k0) + W0) & MASK32)
            k1 = np.uint64((int(k1) + W1) & MASK32)
        p0 = m0 * c0  # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK32)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK32)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & MASK32, seed >> 32


def words(rows, cols, seed, tag):
    """Philox words for the counters (rows[i], cols[j], tag, 0), shape (len(rows), len(cols))."""
    k0, k1 = _key(seed)
    r = np.asarray(rows, dtype=np.uint64)[:, None]
    c = np.asarray(cols, dtype=np.uint64)[None, :]
    return philox4x32_10(r, c, np.uint64(tag), np.uint64(0), k0, k1)


def gaussian_f64(rows, cols, seed, tag=TAG_OMEGA):
    """FP64 Box-Muller Gaussian entries from 53-bit uniforms (see module doc)."""
    w0, w1, w2, w3 = words(rows, cols, seed, tag)
    two26 = np.float64(2.0 ** 26)
    two_m53 = np.float64(2.0 ** -53)
    u1 = ((w0 >> np.uint64(5)).astype(np.float64) * two26
          + (w1 >> np.uint64(6)).astype(np.float64) + 0.5) * two_m53
    u2 = ((w2 >> np.uint64(5)).astype(np.float64) * two26
          + (w3 >> np.uint64(6)).astype(np.float64) + 0.5) * two_m53
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def gaussian_f32_spec(rows, cols, seed, tag=TAG_OMEGA):
    """The FP32-form entries, evaluated here in FP64 from the same 24-bit uniforms.

    The GPU evaluates this formula in FP32; the values differ from these by a
    few FP32 ulps, below the BF16 rounding the mixed path applies afterwards.
    """
    w0, _w1, w2, _w3 = words(rows, cols, seed, tag)
    two_m24 = np.float64(2.0 ** -24)
    u1 = ((w0 >> np.uint64(8)).astype(np.float64) + 0.5) * two_m24
    u2 = ((w2 >> np.uint64(8)).astype(np.float64) + 0.5) * two_m24
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def omega(n, l, seed, col0=0, tag=TAG_OMEGA):
    """The random projection matrix P (n x l) of Fig. 1 step 1, FP64 form.

    Columns are indexed globally from ``col0`` so that a block of columns drawn
    by the adaptive loop equals the same columns of a fixed-rank draw.
    """
    return gaussian_f64(np.arange(n), np.arange(col0, col0 + l), seed, tag)
