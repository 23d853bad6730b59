"""Philox4x32-10 and the sampler's random-draw contract (oracle side).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and
Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11): ten rounds of
two 32x32->64-bit multiplications on a 4-word counter with a 2-word key
bumped by the Weyl constants after every round.  Implemented here from that
published definition in numpy uint32/uint64 arithmetic.

Parity: pinned by the GPU test that compares this function with the
independent device implementation shipped in CUDA's curand header
(`curand_Philox4x32_10(counter, key)`), and by chi-square uniformity and
bijectivity checks on the CPU.

Draw contract (shared by definition with the CUDA path, implemented
independently on each side).  key = (seed mod 2^32, seed div 2^32);
counter = (index, sweep, chain, phase << 24 | sub).

* dual bit of edge slot e, table entry k, chain c, sweep t: entries come in
  groups g = k div 32 with position b = k mod 32.  The 8-bit prefix of the
  uniform is spread over eight "planes": bit (7 - p) of the prefix (p = 0 is
  the most significant) is bit b of word (p mod 4) of
        Philox(e, t, c, DUAL << 24 | 2g + p div 4),
  and the low 16 bits are half (k mod 8) of Philox(e, t, c, DUAL_LO << 24 | k div 8)
  (halves little-endian within the words, words in order 0..3).
    U24 = prefix << 16 | low16,  u = (U24 + 1/2) / 2^24,  theta = [u < p]
  The plane layout lets the device compare 32 entries at once bit-serially;
  the low bits only matter when the prefix equals the threshold's prefix.
* label draw of site v, chain c, sweep t (plain sweep):
    U = word 0 of Philox(v, t, c, PRIMAL << 24),  u = ((U >> 9) + 1/2) / 2^23
  (23 bits, so that u is exactly representable in single precision).
* label draw inside a tree block (blocked sweep): phase FFBS, same layout.
* initial label of site v, chain c:  a = ((U >> 8) * L) >> 24 with U = word 0 of
  Philox(v, 0, c, INIT << 24).
* block offset of the blocked sweep t: o_d = word d of Philox(0, t, 0, SPLASH << 24) >> 30.
* learned proposal (block b, chain c, sweep t): proposal bytes/words from
  phase PROPOSAL, accept uniform from phase ACCEPT (word 0, 24-bit form).
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)

PH_DUAL = 1
PH_DUAL_LO = 2
PH_PRIMAL = 3
PH_INIT = 4
PH_FFBS = 5
PH_SPLASH = 6
PH_PROPOSAL = 7
PH_ACCEPT = 8
PH_BOND = 9       # Swendsen-Wang bond of (edge, chain) (word 0, 23-bit uniform)
PH_CLUSTER = 10   # Swendsen-Wang cluster label, index = the cluster's smallest site (word 0)

_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on broadcastable uint32 arrays.  Returns four uint32 arrays."""
    c0 = np.asarray(c0, np.uint32); c1 = np.asarray(c1, np.uint32)
    c2 = np.asarray(c2, np.uint32); c3 = np.asarray(c3, np.uint32)
    k0 = np.asarray(k0, np.uint64) & _MASK32; k1 = np.asarray(k1, np.uint64) & _MASK32
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0 = c0.copy(); c1 = c1.copy(); c2 = c2.copy(); c3 = c3.copy()
    for r in range(10):
        p0 = PHILOX_M0 * c0.astype(np.uint64)
        p1 = PHILOX_M1 * c2.astype(np.uint64)
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32); lo0 = (p0 & _MASK32).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32); lo1 = (p1 & _MASK32).astype(np.uint32)
        n0 = hi1 ^ c1 ^ k0.astype(np.uint32)
        n2 = hi0 ^ c3 ^ k1.astype(np.uint32)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
        if r < 9:                                   # Weyl key schedule, mod 2^32
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK32
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK32
    return c0, c1, c2, c3


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.uint32(seed & 0xFFFFFFFF), np.uint32(seed >> 32)


def _words(index, sweep, chain, c3, seed):
    k0, k1 = seed_key(seed)
    return np.stack(philox4x32_10(index, sweep, chain, c3, k0, k1), axis=-1)   # [..., 4]


def dual_prefix(edge, k, chain, sweep, seed, m=None):
    """8-bit prefixes of dual uniforms from the bit planes; arguments broadcast.

    Plane p (bit 7 - p of the prefix).  Edges with m > 16 entries (or m not
    given): entry 32 g + b at bit b of word p mod 4 of Philox(e, t, c, DUAL,
    2 g + p div 4).  Edges with m <= 16 entries: all planes in one call, two
    per word: entry k at bit 16 (p div 4) + k of word p mod 4 of
    Philox(e, t, c, DUAL, 0)."""
    edge = np.asarray(edge, np.int64); k = np.asarray(k, np.int64); chain = np.asarray(chain, np.int64)
    prefix = 0
    if m is not None and m <= 16:
        w = _words(edge, sweep, chain, (PH_DUAL << 24) | 0, seed)                 # [..., 4]
        for p in range(8):
            bit = (w[..., p % 4] >> (16 * (p // 4) + k).astype(np.uint32)) & np.uint32(1)
            prefix = prefix | (bit.astype(np.int64) << (7 - p))
        return prefix
    g, b = k >> 5, (k & 31).astype(np.uint32)
    for half in range(2):
        w = _words(edge, sweep, chain, (PH_DUAL << 24) | (2 * g + half), seed)      # [..., 4]
        for q in range(4):
            p = 4 * half + q                                                       # plane index
            bit = (w[..., q] >> b) & np.uint32(1)
            prefix = prefix | (bit.astype(np.int64) << (7 - p))
    return prefix


def dual_u24(edge, k, chain, sweep, seed, m=None):
    """24-bit integer uniforms U24 of dual draws (m: entries per edge); all arguments broadcast."""
    edge = np.asarray(edge, np.int64); k = np.asarray(k, np.int64); chain = np.asarray(chain, np.int64)
    prefix = dual_prefix(edge, k, chain, sweep, seed, m)
    lo = _words(edge, sweep, chain, (PH_DUAL_LO << 24) | (k >> 3), seed)
    kk = np.broadcast_to(k, lo.shape[:-1])
    wsel = np.take_along_axis(lo, ((kk & 7) >> 1)[..., None], axis=-1)[..., 0]
    low = (wsel >> (16 * (kk & 1)).astype(np.uint32)) & np.uint32(0xFFFF)
    return (prefix.astype(np.int64) << 16) | low.astype(np.int64)


def u24_to_unit(u24):
    """u = (U24 + 1/2) / 2^24 (exact in float64)."""
    return (np.asarray(u24, np.float64) + 0.5) / 16777216.0


def u23_to_unit(u23):
    """u = (U23 + 1/2) / 2^23 (exact in float32 and float64)."""
    return (np.asarray(u23, np.float64) + 0.5) / 8388608.0


def dual_uniform(edge, k, chain, sweep, seed, m=None):
    return u24_to_unit(dual_u24(edge, k, chain, sweep, seed, m))


def site_uniform(site, chain, sweep, seed, phase=PH_PRIMAL):
    """Uniform of a label draw (plain sweep: phase PRIMAL; tree blocks: FFBS)."""
    w = _words(np.asarray(site, np.int64), sweep, np.asarray(chain, np.int64), phase << 24, seed)[..., 0]
    return u23_to_unit(w >> np.uint32(9))


def init_labels(n_vars: int, n_labels: int, n_chains: int, seed: int):
    """Initial labels [C][N]: a = ((U >> 8) * L) >> 24 with U from phase INIT."""
    v = np.arange(n_vars, dtype=np.int64)[None, :]
    c = np.arange(n_chains, dtype=np.int64)[:, None]
    w = _words(v, 0, c, PH_INIT << 24, seed)[..., 0]
    return (((w >> np.uint32(8)).astype(np.int64) * n_labels) >> 24).astype(np.int64)


def splash_offset(sweep: int, seed: int):
    """Block-grid offset (ox, oy, oz) in [0,4)^3 for blocked sweep `sweep`."""
    w = _words(0, sweep, 0, PH_SPLASH << 24, seed)
    return tuple(int(x) >> 30 for x in w[:3])
