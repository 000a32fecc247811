"""Counter-based random numbers for the oracle (test infrastructure only).

Philox4x32-10 follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): 10 rounds of the
S-box-free round function with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl
key increments 0x9E3779B9 / 0xBB67AE85.  Pinned by the published known-answer
vectors in tests/golden/philox4x32_10_kat.txt.

Draw allocation (the same scheme is implemented independently in the CUDA
library, from this description):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (c0 = item index, c1 = step n, c2 = purpose << 16 | sub, c3 = block)

Normal variates: Box-Muller on a pair of uniforms.  Gamma variates:
Marsaglia & Tsang (2000), "A simple method for generating gamma variables",
one Philox block per attempt, at most MAX_GAMMA_ATTEMPTS attempts.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

# purposes (c2 >> 16)
MT_PREDICT = 1
ETA_PREDICT = 2
PF_GAUSS = 3
PF_GAMMA = 4
BIRTH = 5
RESAMPLE = 6
JITTER_MT = 7
JITTER_PF = 8
JITTER_ETA = 9
INIT_MT = 10
INIT_ETA = 11
SYNTH_NOISE = 12
BIRTH_CAND = 13      # candidate SFV positions of the birth proposal (item = candidate index, sub = partition)
BIRTH_PROP = 14      # normals of particles drawn from the birth proposal (sub = PF slot)
LEARNED_PROP = 15    # normals of the learned MT proposal (item = particle)
LP_DATA = 16         # draws of the proposal network's training samples

MAX_GAMMA_ATTEMPTS = 16


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of counters (broadcast); returns 4 uint32 arrays."""
    c0, c1, c2, c3 = [np.asarray(v, dtype=np.uint64) & MASK for v in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
        k0 = (k0 + W0) & MASK
        k1 = (k1 + W1) & MASK
    return [v.astype(np.uint32) for v in (c0, c1, c2, c3)]


def draw(seed: int, c0, n: int, purpose: int, sub: int, block):
    """Four uint32 per counter (c0 may be an array)."""
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    c2 = ((purpose & 0xFFFF) << 16) | (sub & 0xFFFF)
    return philox4x32_10(c0, n, c2, block, k0, k1)


def u24(x):
    """Uniform in (0,1) from the top 24 bits: ((x >> 8) + 1/2) * 2^-24 (exact in FP64)."""
    return ((np.asarray(x, np.uint32) >> np.uint32(8)).astype(np.float64) + 0.5) * (2.0 ** -24)


def u32d(x):
    """Uniform in (0,1) from all 32 bits: (x + 1/2) * 2^-32 (exact in FP64)."""
    return (np.asarray(x, np.uint32).astype(np.float64) + 0.5) * (2.0 ** -32)


def box_muller(ua, ub):
    """Box-Muller pair (r cos 2 pi ub, r sin 2 pi ub), r = sqrt(-2 ln ua)."""
    r = np.sqrt(-2.0 * np.log(ua))
    t = 2.0 * np.pi * ub
    return r * np.cos(t), r * np.sin(t)


def normals4(seed, c0, n, purpose, sub, block):
    """Four standard normals per counter from 24-bit uniforms (pairs (0,1), (2,3))."""
    x = draw(seed, c0, n, purpose, sub, block)
    a0, a1 = box_muller(u24(x[0]), u24(x[1]))
    b0, b1 = box_muller(u24(x[2]), u24(x[3]))
    return [a0, a1, b0, b1]


def normals(seed, c0, n, purpose, sub, count):
    """`count` normals per counter, drawn from blocks 0, 1, ... in order."""
    out = []
    block = 0
    while len(out) < count:
        out.extend(normals4(seed, c0, n, purpose, sub, block))
        block += 1
    return out[:count]


def uniforms24(seed, c0, n, purpose, sub, count):
    out = []
    block = 0
    while len(out) < count:
        x = draw(seed, c0, n, purpose, sub, block)
        out.extend([u24(v) for v in x])
        block += 1
    return out[:count]


def gamma(seed, c0, n, purpose, sub, shape: float, scale):
    """Gamma(shape, scale) by Marsaglia-Tsang; one Philox block per attempt.

    Attempt a uses block a: x0, x1 -> normal g by Box-Muller (cos branch, FP64
    uniforms), x2 -> acceptance uniform.  Accept when v = (1 + c g)^3 > 0 and
    log u < g^2/2 + d - d v + d log v; the value is d v scale.  If all
    MAX_GAMMA_ATTEMPTS attempts reject, the mean shape*scale is returned."""
    if shape < 1.0:
        raise ValueError("shape must be >= 1")
    c0 = np.asarray(c0)
    scale = np.broadcast_to(np.asarray(scale, np.float64), c0.shape).astype(np.float64)
    d = shape - 1.0 / 3.0
    c = 1.0 / np.sqrt(9.0 * d)
    out = shape * scale
    done = np.zeros(c0.shape, bool)
    for a in range(MAX_GAMMA_ATTEMPTS):
        x = draw(seed, c0, n, purpose, sub, a)
        g = np.sqrt(-2.0 * np.log(u32d(x[0]))) * np.cos(2.0 * np.pi * u32d(x[1]))
        v = (1.0 + c * g) ** 3
        u = u32d(x[2])
        with np.errstate(invalid="ignore", divide="ignore"):
            ok = (v > 0) & (np.log(u) < 0.5 * g * g + d - d * v + d * np.log(np.where(v > 0, v, 1.0)))
        take = ok & ~done
        out = np.where(take, d * v * scale, out)
        done |= ok
        if done.all():
            break
    return out
