"""Entropy coding of the residual codes, plain Python (test infrastructure).

Only the test suite and ``bench.py``'s CPU baseline may import this module; it
shares no code with the CUDA library.

The paper stores the quantised residual after a lossless coding stage (MGARD's
Huffman and Zstd, Sec. III Stage 4 and the ADIOS buffer of Stage 5); it does
not fix a format.  Reading: one Golomb-Rice code per histogram (the residual
codes of a good decoder are close to a two-sided geometric law, for which Rice
codes are near-optimal), with

* symbols: the zero-level code -> 0, a level q -> zigzag(q) + 1
  (zigzag(q) = 2q for q >= 0, -2q - 1 for q < 0), the escape code -> 65535;
* per histogram the parameter k in 0..15 that gives the fewest bits (ties to
  the smaller k);
* per symbol s: u = s >> k; if u < 24: u one-bits, a zero-bit, then the k low
  bits of s (least significant first); else 24 one-bits and the 16 bits of s
  (least significant first);
* bit i of a histogram's stream is bit (i mod 32) of 32-bit word i // 32; the
  unused high bits of the last word are zero.

Pins (tests/test_oracle_rice.py): hand-encoded streams, decode(encode(c)) = c,
stream lengths equal to the sum of the per-symbol lengths, and on geometric
sources the chosen k and the mean length equal to the closed form of Rice
codes (u = s >> k is geometric with parameter theta^(2^k)).
"""
from __future__ import annotations

import numpy as np

ESCAPE = -32768
ZERO_CODE = -32767
CAP = 24
K_MAX = 15


def symbol(code: int) -> int:
    if code == ZERO_CODE:
        return 0
    if code == ESCAPE:
        return 65535
    return (2 * code if code >= 0 else -2 * code - 1) + 1


def code_of(s: int) -> int:
    if s == 0:
        return ZERO_CODE
    if s == 65535:
        return ESCAPE
    z = s - 1
    return z // 2 if z % 2 == 0 else -(z + 1) // 2


def symbol_bits(s: int, k: int) -> int:
    u = s >> k
    return u + 1 + k if u < CAP else CAP + 16


def best_k(symbols) -> int:
    best, arg = None, 0
    for k in range(K_MAX + 1):
        t = sum(symbol_bits(s, k) for s in symbols)
        if best is None or t < best:
            best, arg = t, k
    return arg


def encode_one(codes):
    """(k, nbits, words uint32) for one histogram's codes."""
    syms = [symbol(int(c)) for c in codes]
    k = best_k(syms)
    bits = []
    for s in syms:
        u = s >> k
        if u < CAP:
            bits += [1] * u + [0]
            bits += [(s >> i) & 1 for i in range(k)]
        else:
            bits += [1] * CAP
            bits += [(s >> i) & 1 for i in range(16)]
    nbits = len(bits)
    words = np.zeros((nbits + 31) // 32, dtype=np.uint32)
    for i, b in enumerate(bits):
        if b:
            words[i // 32] |= np.uint32(1 << (i % 32))
    return k, nbits, words


def decode_one(k: int, words, P: int):
    """P codes from one histogram's stream."""
    def bit(i):
        return (int(words[i // 32]) >> (i % 32)) & 1
    pos, out = 0, []
    for _ in range(P):
        u = 0
        while u < CAP and bit(pos):
            u += 1
            pos += 1
        if u < CAP:
            pos += 1  # the terminating zero
            low = sum(bit(pos + i) << i for i in range(k))
            pos += k
            s = (u << k) | low
        else:
            s = sum(bit(pos + i) << i for i in range(16))
            pos += 16
        out.append(code_of(s))
    return np.array(out, dtype=np.int16)


def encode(codes: np.ndarray):
    """Batch [n][P]: (k [n] uint8, nbits [n] uint32, offsets [n+1] int64 in
    words, words uint32 = the streams back to back)."""
    n = codes.shape[0]
    ks = np.zeros(n, dtype=np.uint8)
    nb = np.zeros(n, dtype=np.uint32)
    parts = []
    for b in range(n):
        k, nbits, w = encode_one(codes[b])
        ks[b], nb[b] = k, nbits
        parts.append(w)
    off = np.zeros(n + 1, dtype=np.int64)
    off[1:] = np.cumsum([len(w) for w in parts])
    words = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint32)
    return ks, nb, off, words


def decode(ks, off, words, P: int) -> np.ndarray:
    n = len(ks)
    out = np.zeros((n, P), dtype=np.int16)
    for b in range(n):
        out[b] = decode_one(int(ks[b]), words[off[b]:off[b + 1]], P)
    return out
