"""Counter-based random numbers for the oracle (test infrastructure).

Philox4x64-10 as published by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64->128 bit
multiplies on a four-word counter, with a two-word key bumped by Weyl
constants between rounds.  The paper leaves the generator open (any valid
sampler of Ex. 1 / Ex. 2 will do); this mapping fixes it so that the CUDA path
and the oracle draw identical inputs:

  key     = (seed, 0)
  counter = (c0 = call index inside a stream, c1 = sample index i,
             c2 = level l, c3 = stream id)
  stream 0      : interface uniforms; interface t uses word t%4 of call t//4
  stream 1      : layer normals Z_t of Ex. 1; normal t is entry t%4 of call t//4
  stream 2 + f  : complex normals xi_q of circulant-embedding field pair f,
                  q = q2*M + q1; xi_q is pair q%2 of call q//2

A 64-bit word w becomes the uniform u = ((w >> 12) + 1/2) * 2^-52, which is
exact in FP64 and lies strictly inside (0, 1).  Uniforms (u_a, u_b) become a
normal pair by Box-Muller:
  re = sqrt(-2 ln u_a) cos(2 pi u_b),  im = sqrt(-2 ln u_a) sin(2 pi u_b).
Call c gives words (w0, w1, w2, w3); its normals are, in order,
  BM(u0, u1).re, BM(u0, u1).im, BM(u2, u3).re, BM(u2, u3).im.
"""
import numpy as np

# Published Philox4x64 multipliers and Weyl key increments (Salmon et al. 2011).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
PHILOX_ROUNDS = 10

STREAM_INTERFACE = 0
STREAM_LAYER_Z = 1
STREAM_FIELD0 = 2

_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """128-bit product of uint64 arrays a*b split into (hi, lo) words."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    p0 = a_lo * b_lo
    p1 = a_lo * b_hi
    p2 = a_hi * b_lo
    p3 = a_hi * b_hi
    mid = (p0 >> _S32) + (p1 & _LO32) + (p2 & _LO32)
    hi = p3 + (p1 >> _S32) + (p2 >> _S32) + (mid >> _S32)
    lo = a * b  # wraps modulo 2^64
    return hi, lo


def philox4x64(c0, c1, c2, c3, k0, k1):
    """Philox4x64-10 bijection of counter (c0..c3) under key (k0, k1).

    Arguments broadcast; returns four uint64 arrays (w0, w1, w2, w3)."""
    c = [np.asarray(x, dtype=np.uint64) for x in np.broadcast_arrays(
        np.asarray(c0, dtype=np.uint64), np.asarray(c1, dtype=np.uint64),
        np.asarray(c2, dtype=np.uint64), np.asarray(c3, dtype=np.uint64))]
    k0 = np.uint64(k0)
    k1 = np.uint64(k1)
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    with np.errstate(over="ignore"):
        for rnd in range(PHILOX_ROUNDS):
            if rnd > 0:  # key schedule: bump between rounds
                k0 = np.uint64((int(k0) + PHILOX_W0) & 0xFFFFFFFFFFFFFFFF)
                k1 = np.uint64((int(k1) + PHILOX_W1) & 0xFFFFFFFFFFFFFFFF)
            hi0, lo0 = _mulhilo(m0, c[0])
            hi1, lo1 = _mulhilo(m1, c[2])
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c[0], c[1], c[2], c[3]


def stream_words(seed, level, sample, stream, calls):
    """Words of calls ``calls`` (array of c0) for one (sample, level, stream).

    Returns a uint64 array of shape (len(calls), 4)."""
    calls = np.asarray(calls, dtype=np.uint64)
    w = philox4x64(calls, np.uint64(sample), np.uint64(level), np.uint64(stream),
                   np.uint64(seed), np.uint64(0))
    return np.stack(w, axis=-1)


def uniform(words):
    """u = ((w >> 12) + 1/2) * 2^-52 in (0, 1), exact in FP64."""
    k = (np.asarray(words, dtype=np.uint64) >> np.uint64(12)).astype(np.float64)
    return (k + 0.5) * 2.0 ** -52


def box_muller(ua, ub):
    """Normal pair (re, im) from two uniforms in (0, 1)."""
    rad = np.sqrt(-2.0 * np.log(ua))
    ang = 2.0 * np.pi * ub
    return rad * np.cos(ang), rad * np.sin(ang)


def call_normals(words):
    """Four normals of each call (rows of ``words``), in the documented order."""
    u = uniform(words)
    re0, im0 = box_muller(u[..., 0], u[..., 1])
    re1, im1 = box_muller(u[..., 2], u[..., 3])
    return np.stack([re0, im0, re1, im1], axis=-1)


def interface_uniforms(seed, level, sample, n):
    """First n uniforms of stream 0 (one per interface draw)."""
    calls = np.arange((n + 3) // 4)
    return uniform(stream_words(seed, level, sample, STREAM_INTERFACE, calls)).reshape(-1)[:n]


def layer_normals(seed, level, sample, n):
    """First n standard normals of stream 1 (Ex. 1 layer variables Z_t)."""
    calls = np.arange((n + 3) // 4)
    return call_normals(stream_words(seed, level, sample, STREAM_LAYER_Z, calls)).reshape(-1)[:n]


def field_normals(seed, level, sample, pair, M, dim=2):
    """Complex normals of field pair ``pair``: xi[q2, q1] (M x M), or with
    dim = 3 xi[q3, q2, q1] (M x M x M); the flat index q = q1 + M q2 (+ M^2 q3)
    is the complex index of the Philox stream."""
    nq = M ** dim
    calls = np.arange(nq // 2)
    z = call_normals(stream_words(seed, level, sample, STREAM_FIELD0 + pair, calls)).reshape(-1)
    xi = z[0::2] + 1j * z[1::2]  # entry 2q is Re xi_q, entry 2q+1 is Im xi_q
    return xi.reshape((M,) * dim)
