"""Counter-based noise for conditional simulation -- oracle (test infrastructure).

Philox4x64-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter and a 2-word key,
ten rounds of two 64x64->128-bit multiplies with a Weyl-sequence key bump.

Uniforms and normals (the definition shared with the CUDA library, which has
its own independent implementation):

* each 64-bit word w gives two 32-bit halves, h = w >> 32 and l = w mod 2^32,
  and u(x) = (x + 1/2) * 2^-32 is a uniform in (0, 1) from a half;
* Box-Muller on one word: r = sqrt(-2 ln u(h)); (xi, eta) =
  (r cos 2 pi u(l), r sin 2 pi u(l)).

Counter layout (key = (seed, 0)); one generator call serves four
consecutive indices, index j taking word j mod 4:

* stream 1, the circulant-embedding noise of realisation pair p at torus
  index k (column-major, k = kx * Qy + ky): counter (k >> 2, p, 1, 0), word
  k mod 4, giving (xi_k, eta_k).
* stream 2, the site noise of realisation t at site i: counter
  (i >> 2, t, 2, 0), word i mod 4, giving (xi'_i, eps_i).
"""
import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

STREAM_CE = 1
STREAM_OBS = 2


def _mulhilo(a, b):
    """(high, low) 64-bit halves of the 128-bit product a * b, elementwise."""
    a0, a1 = a & _LO32, a >> _S32
    b0, b1 = b & _LO32, b >> _S32
    p00 = a0 * b0
    p01 = a0 * b1
    p10 = a1 * b0
    p11 = a1 * b1
    mid = (p00 >> _S32) + (p01 & _LO32) + (p10 & _LO32)
    hi = p11 + (p01 >> _S32) + (p10 >> _S32) + (mid >> _S32)
    return hi, a * b


def philox4x64(c0, c1, c2, c3, k0, k1, rounds=10):
    """Philox4x64-`rounds` of the counter (c0..c3) under key (k0, k1), elementwise."""
    with np.errstate(over="ignore"):
        c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) for x in (c0, c1, c2, c3))
        c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
        k0 = np.uint64(k0)
        k1 = np.uint64(k1)
        for _ in range(rounds):
            hi0, lo0 = _mulhilo(M0, c0)
            hi1, lo1 = _mulhilo(M1, c2)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = k0 + W0
            k1 = k1 + W1
    return c0, c1, c2, c3


def uniform(x):
    """u(x) = (x + 1/2) 2^-32 in (0, 1) for a 32-bit half x, exact in FP64."""
    return (np.asarray(x, np.uint64).astype(np.float64) + 0.5) * 2.0 ** -32


def box_muller(w):
    """Two independent N(0, 1) from the two halves of a 64-bit word."""
    w = np.asarray(w, np.uint64)
    r = np.sqrt(-2.0 * np.log(uniform(w >> _S32)))
    t = 2.0 * np.pi * uniform(w & _LO32)
    return r * np.cos(t), r * np.sin(t)


def normal_pairs(index, sub, stream, seed):
    """The normal pair assigned to element `index` of realisation `sub` in `stream`."""
    index = np.asarray(index, dtype=np.uint64)
    w = philox4x64(index >> np.uint64(2), np.uint64(sub), np.uint64(stream), 0,
                   np.uint64(seed), 0)
    j = (index & np.uint64(3)).astype(np.int64)
    return box_muller(np.choose(j, w))
