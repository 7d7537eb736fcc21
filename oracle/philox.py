"""Philox4x32-10 and Box-Muller normals (oracle side).

The randomised rank-revealing factorization draws an n-by-n matrix of i.i.d.
N(0,1) entries (Sec. 2, Algorithm 1, first step).  Both the oracle and the
GPU path generate it from the same published counter-based generator so the
draws agree without passing matrices around:

  Philox4x32-10, J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11.  Round function:
  (c0,c1,c2,c3) -> (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2), hi(M0*c0) ^ c3 ^ k1,
  lo(M0*c0)), key bumped by the Weyl constants (W0, W1) between rounds.

Counter layout used by this project (the GPU side implements the same one):
  c0 = pair index low 32 bits,
  c1 = (pair index bits 32..39) | (attempt & 0xFF) << 8 | purpose << 16,
  c2 = stream low 32 bits,     c3 = stream high 32 bits,
  key = (seed low 32, seed high 32).
The stream is a 64-bit node id of the recursion tree: the root is 1 and a
child's id is splitmix64(2 * parent + side + 1) (the splitmix64 finaliser of
Steele, Lea and Flood, OOPSLA 2014), so ids do not depend on the order in
which nodes are processed.
One call yields four 32-bit words -> two 52-bit uniforms
  u1 = (m1 + 1/2) 2^-52 in (0,1),   u2 = m2 2^-52 in [0,1),
  m1 = x0 << 20 | x1 >> 12,         m2 = x2 << 20 | x3 >> 12,
and Box-Muller gives z0 = r cos(2 pi u2), z1 = r sin(2 pi u2), r = sqrt(-2 ln u1).
Element e of a column-major matrix takes component e % 2 of pair e // 2.

Pinned by the published known-answer vectors (tests/golden/philox4x32_10_kat.txt)
and by moment tests of the normals.
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF

# purposes of the draws inside the method (counter word c1 bits 16..31)
PURPOSE_HAAR = 4
PURPOSE_SHIFT = 5
PURPOSE_HAAR_LEFT = 6
PURPOSE_POWER = 9        # start vector of the symmetric root's power iteration


def attempt_code(attempt, draw):
    """8-bit attempt word: shift attempt (6 bits) and Haar redraw index (2 bits)."""
    return ((attempt & 0x3F) << 2) | (draw & 0x3)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on arrays of 32-bit counters; returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.uint64(k0 & _MASK)
    k1 = np.uint64(k1 & _MASK)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    s32 = np.uint64(32)
    mask = np.uint64(_MASK)
    for _ in range(10):
        p0 = m0 * c0          # 32x32 -> 64-bit product, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(W0)) & mask
        k1 = (k1 + np.uint64(W1)) & mask
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def splitmix64(x):
    """splitmix64 finaliser (Steele, Lea, Flood 2014) on a Python int."""
    m = (1 << 64) - 1
    z = (x + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


ROOT_NODE = 1


def child_node(parent, side):
    """Node id of child `side` (0: eigenvalues outside / right, 1: inside / left)."""
    return splitmix64(((2 * parent) + side + 1) & ((1 << 64) - 1))


def _counters(npairs, purpose, stream, attempt=0):
    i = np.arange(npairs, dtype=np.uint64)
    c0 = i & np.uint64(_MASK)
    c1 = (((i >> np.uint64(32)) & np.uint64(0xFF))
          | np.uint64((attempt & 0xFF) << 8) | np.uint64((purpose & 0xFFFF) << 16))
    c2 = np.full(npairs, stream & _MASK, dtype=np.uint64)
    c3 = np.full(npairs, (stream >> 32) & _MASK, dtype=np.uint64)
    return c0, c1, c2, c3


def uniform_pairs(npairs, seed, purpose, stream, attempt=0):
    """(u1, u2) arrays: u1 in (0,1), u2 in [0,1), both exact multiples of 2^-53."""
    c0, c1, c2, c3 = _counters(npairs, purpose, stream, attempt)
    x0, x1, x2, x3 = philox4x32_10(c0, c1, c2, c3, seed & _MASK, (seed >> 32) & _MASK)
    x0 = x0.astype(np.uint64); x1 = x1.astype(np.uint64)
    x2 = x2.astype(np.uint64); x3 = x3.astype(np.uint64)
    m1 = (x0 << np.uint64(20)) | (x1 >> np.uint64(12))
    m2 = (x2 << np.uint64(20)) | (x3 >> np.uint64(12))
    u1 = (m1.astype(np.float64) + 0.5) * 2.0 ** -52
    u2 = m2.astype(np.float64) * 2.0 ** -52
    return u1, u2


def gaussian_matrix(rows, cols, seed, purpose, stream, attempt=0):
    """rows x cols matrix of N(0,1) draws, element order column-major."""
    count = rows * cols
    npairs = (count + 1) // 2
    u1, u2 = uniform_pairs(npairs, seed, purpose, stream, attempt)
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count].reshape(cols, rows).T.copy()


def uniform_scalar(seed, purpose, stream, attempt=0):
    """One uniform in [0,1) (the u2 word of pair 0) for shift jitter."""
    _, u2 = uniform_pairs(1, seed, purpose, stream, attempt)
    return float(u2[0])
