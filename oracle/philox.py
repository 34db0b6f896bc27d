"""Counter-based noise for conditional simulation -- oracle (test infrastructure).

Philox4x64-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4-word counter and a 2-word key,
ten rounds of two 64x64->128-bit multiplies with a Weyl-sequence key bump.

Uniforms and normals (the definition shared with the CUDA library, which has
its own independent implementation):

* u(w) = ((w >> 11) + 1/2) * 2^-53, a uniform in (0, 1) from a 64-bit word.
* Box-Muller: r = sqrt(-2 ln u1); (xi, eta) = (r cos 2 pi u2, r sin 2 pi u2).

Counter layout (key = (seed, 0)):

* stream 1, the circulant-embedding noise of realisation pair p at torus
  index k (column-major, k = kx * Qy + ky): counter (k >> 1, p, 1, 0); the
  words (w0, w1) serve even k, (w2, w3) odd k, giving (xi_k, eta_k).
* stream 2, the site noise of realisation t at site i: counter
  (i >> 1, t, 2, 0), words (w0, w1) for even i, (w2, w3) for odd i, giving
  (xi'_i, eps_i).
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


def uniform(w):
    """u(w) = ((w >> 11) + 1/2) 2^-53 in (0, 1), exact in FP64."""
    return ((np.asarray(w, np.uint64) >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def box_muller(w1, w2):
    """Two independent N(0, 1) from two 64-bit words."""
    r = np.sqrt(-2.0 * np.log(uniform(w1)))
    t = 2.0 * np.pi * uniform(w2)
    return r * np.cos(t), r * np.sin(t)


def normal_pairs(index, sub, stream, seed):
    """The normal pair assigned to element `index` of realisation `sub` in `stream`."""
    index = np.asarray(index, dtype=np.uint64)
    w = philox4x64(index >> np.uint64(1), np.uint64(sub), np.uint64(stream), 0,
                   np.uint64(seed), 0)
    odd = (index & np.uint64(1)).astype(bool)
    wa = np.where(odd, w[2], w[0])
    wb = np.where(odd, w[3], w[1])
    return box_muller(wa, wb)
