"""Counter-based random numbers the method draws on the GPU -- test oracle.

The sketch matrix Phi of Sec. 2.3 (Gaussian JL, entries N(0, 1/s)) and the
CountSketch hash h(t) and signs s_t are random draws.  The library makes
them on the device from a 64-bit seed; this module makes the same draws on
the host from the published definitions, so that tests compare the two
streams and the oracle can sketch with the very matrix the GPU used without
taking it from the GPU.

* ``philox4x32_10`` -- the Philox4x32 counter-based generator with 10
  rounds (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
  as 1, 2, 3", SC'11): a 128-bit counter (four 32-bit words) and a 64-bit
  key (two words); each round multiplies words 0 and 2 by the constants
  0xD2511F53 and 0xCD9E8D57 (64-bit products split into high and low
  halves) and mixes the halves with words 1 and 3 and the key; the key is
  bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 between rounds.
* ``gaussian_sketch_t`` -- Phi^T (s x T): entry (j, t) comes from the Philox
  block with key (seed mod 2^32, seed div 2^32) and counter (t div 4, j, 0, 0).
  Its four words give u_a = ((w_a >> 8) + 1) 2^-24 in (0, 1] (a = 0, 2) and
  v_b = (w_b >> 8) 2^-24 in [0, 1) (b = 1, 3), both exact in FP32; the
  Box--Muller transform (Box and Muller, 1958) r = sqrt(-2 ln u),
  (r cos 2 pi v, r sin 2 pi v) turns (u_0, v_1) and (u_2, v_3) into four
  standard normals, taken by t mod 4 = 0, 1, 2, 3 in that order; the entry
  is that normal divided by sqrt(s).  Computed here in FP64 (the angle
  reduced exactly to a quarter turn first, so cos and sin keep their
  relative accuracy next to their zeros).
* ``round_bf16`` -- rounding to the nearest BF16 value (8 significant bits),
  ties to even, straight from FP64; ``gaussian_sketch_bf16`` is the sketch
  stored that way (the library's stored Phi).
* ``countsketch_draw`` -- h(t) and s_t from the block with the same key and
  counter (t, 0, 1, 0): h(t) = floor(w_0 s / 2^32) (multiply-shift, bias
  below s / 2^32 per bucket) and s_t = 1 - 2 (w_1 mod 2).
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, key):
    """Philox4x32-10 on arrays of counters (broadcast); returns four uint32 arrays."""
    c = [np.asarray(x, dtype=np.uint64) & _MASK for x in (c0, c1, c2, c3)]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c[0]
        p1 = _M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return [x.astype(np.uint32) for x in c]


def seed_key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def _sincospi(x):
    """(sin pi x, cos pi x) for x in [0, 2) given exactly: x = k/2 + r with
    |r| <= 1/4 (exact), then the quarter-turn identities."""
    k = np.rint(2.0 * x)
    r = x - 0.5 * k
    sr, cr = np.sin(np.pi * r), np.cos(np.pi * r)
    q = k.astype(np.int64) % 4
    sn = np.select([q == 0, q == 1, q == 2, q == 3], [sr, cr, -sr, -cr])
    cs = np.select([q == 0, q == 1, q == 2, q == 3], [cr, -sr, -cr, sr])
    return sn, cs


def round_bf16(x):
    """Nearest BF16 value (8 significant bits, ties to even), as FP64."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                    # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(m * 256.0), e - 8)


def gaussian_sketch_t(seed: int, s: int, T: int, rows=None) -> np.ndarray:
    """Phi^T (s x T, FP64): rows j of ``rows`` (default all), N(0, 1/s) entries."""
    rows = np.arange(s) if rows is None else np.asarray(rows)
    key = seed_key(seed)
    q = np.arange((T + 3) // 4, dtype=np.uint64)
    out = np.empty((rows.size, T), dtype=np.float64)
    two24 = 2.0 ** -24
    for i, j in enumerate(rows):
        w = philox4x32_10(q, np.uint64(j), 0, 0, key)
        u0 = ((w[0] >> 8).astype(np.float64) + 1.0) * two24
        v1 = (w[1] >> 8).astype(np.float64) * two24
        u2 = ((w[2] >> 8).astype(np.float64) + 1.0) * two24
        v3 = (w[3] >> 8).astype(np.float64) * two24
        r0, r2 = np.sqrt(-2.0 * np.log(u0)), np.sqrt(-2.0 * np.log(u2))
        s1, c1 = _sincospi(2.0 * v1)
        s3, c3 = _sincospi(2.0 * v3)
        z = np.stack([r0 * c1, r0 * s1, r2 * c3, r2 * s3], axis=1).reshape(-1)
        out[i] = z[:T] / np.sqrt(s)
    return out


def gaussian_sketch_bf16(seed: int, s: int, T: int, rows=None) -> np.ndarray:
    """The sketch as stored: each entry of ``gaussian_sketch_t`` rounded to BF16."""
    return round_bf16(gaussian_sketch_t(seed, s, T, rows))


def countsketch_draw(seed: int, T: int, s: int):
    """(h int64 [T] in [0, s), sign int8 [T] in {-1, +1})."""
    key = seed_key(seed)
    t = np.arange(T, dtype=np.uint64)
    w = philox4x32_10(t, 0, 1, 0, key)
    h = ((w[0].astype(np.uint64) * np.uint64(s)) >> np.uint64(32)).astype(np.int64)
    sign = (1 - 2 * (w[1] & np.uint32(1)).astype(np.int64)).astype(np.int8)
    return h, sign
