"""Philox4x32-10 counter-based generator (Salmon et al., SC 2011) and Box-Muller normals.

One Philox call maps a 128-bit counter and a 64-bit key to 128 random bits.  Ten rounds; each
round multiplies counter words 0 and 2 by the published multipliers, mixes the high halves with
words 1 and 3 and the key, and the key is advanced by the published Weyl increments between
rounds.  Implemented with numpy uint64 arithmetic on whole index arrays.
"""
import ctypes
import os

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Return the four 32-bit output words (uint32 arrays) for counters (c0..c3) and key (k0, k1).

    Counter words may be arrays (broadcast together); the key words are scalars.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


_LIB = None


def _compiled():
    """The compiled word generator of philox.c (built by lqcd_inputs/build.py), or None."""
    global _LIB
    if _LIB is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libphilox.so")
        _LIB = False
        if os.path.exists(path):
            lib = ctypes.CDLL(path)
            lib.philox_words.restype = None
            lib.philox_words.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_uint32, ctypes.c_uint64,
                                         ctypes.c_void_p]
            lib.gaussian_pairs.restype = None
            lib.gaussian_pairs.argtypes = lib.philox_words.argtypes
            lib.su3_links.restype = None
            lib.su3_links.argtypes = [ctypes.c_void_p, ctypes.c_long, ctypes.c_uint32, ctypes.c_uint64,
                                      ctypes.c_double, ctypes.c_void_p]
            _LIB = lib
    return _LIB or None


def philox_words(seed, purpose, index):
    """The four Philox words (uint32 arrays) of counter (index lo, index hi, purpose, 0) and key
    (seed lo, seed hi): the compiled generator when built, else the numpy rounds above."""
    index = np.asarray(index, dtype=np.uint64)
    lib = _compiled()
    if lib is None or index.size < 4096:
        seed = int(seed)
        return philox4x32_10(index & _MASK, index >> np.uint64(32), np.uint64(purpose), 0,
                             seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    flat = np.ascontiguousarray(index.ravel())
    out = np.empty((flat.size, 4), dtype=np.uint32)
    lib.philox_words(flat.ctypes.data, flat.size, int(purpose) & 0xFFFFFFFF, int(seed) & 0xFFFFFFFFFFFFFFFF,
                     out.ctypes.data)
    return tuple(out[:, w].reshape(index.shape) for w in range(4))


def uniforms(seed, purpose, index):
    """Two uniforms in (0, 1) with 53-bit resolution per index: shape index.shape + (2,).

    Counter = (index low word, index high word, purpose, 0); key = (seed low, seed high).
    """
    w = [x.astype(np.float64) for x in philox_words(seed, purpose, index)]
    # 27 high bits of one word and 26 of the next make a 53-bit integer; +0.5 keeps it off 0 and 1.
    u1 = (np.floor(w[0] / 32.0) * 67108864.0 + np.floor(w[1] / 64.0) + 0.5) / 9007199254740992.0
    u2 = (np.floor(w[2] / 32.0) * 67108864.0 + np.floor(w[3] / 64.0) + 0.5) / 9007199254740992.0
    return np.stack([u1, u2], axis=-1)


def gaussians(seed, purpose, index):
    """Two independent N(0,1) numbers per index (Box-Muller): shape index.shape + (2,).
    Large index arrays use the compiled generator (same recipe; libm's log / cos / sin, so the
    numbers can differ from numpy's in the last bit)."""
    index = np.asarray(index, dtype=np.uint64)
    lib = _compiled()
    if lib is not None and index.size >= 4096:
        flat = np.ascontiguousarray(index.ravel())
        out = np.empty((flat.size, 2), dtype=np.float64)
        lib.gaussian_pairs(flat.ctypes.data, flat.size, int(purpose) & 0xFFFFFFFF,
                           int(seed) & 0xFFFFFFFFFFFFFFFF, out.ctypes.data)
        return out.reshape(index.shape + (2,))
    u = uniforms(seed, purpose, index)
    r = np.sqrt(-2.0 * np.log(u[..., 0]))
    th = 2.0 * np.pi * u[..., 1]
    return np.stack([r * np.cos(th), r * np.sin(th)], axis=-1)
