"""Pins of the residual-code entropy coder oracle (Golomb-Rice, one parameter
per histogram) against hand-encoded streams, round trips and the coding
bound of Rice codes on geometric sources."""
import numpy as np
import pytest

from oracle import rice

ZERO, ESC = rice.ZERO_CODE, rice.ESCAPE


def test_hand_encoded_stream():
    # codes 0, -1, 1, zero level, escape -> symbols 1, 2, 3, 0, 65535.
    # k = 0: 2 + 3 + 4 + 1 + 40 = 50 bits; k = 1: 2 + 3 + 3 + 2 + 40 = 50 (tie,
    # smaller k wins); k = 2: 52.  Stream (bit 0 first):
    #   1 0 | 1 1 0 | 1 1 1 0 | 0 | 24 ones | 16 ones
    # word 0 has bits 0, 2, 3, 5, 6, 7 and 10..31 set; word 1 bits 0..17.
    k, nbits, words = rice.encode_one(np.array([0, -1, 1, ZERO, ESC], dtype=np.int16))
    assert (k, nbits) == (0, 50)
    w0 = 1 + 4 + 8 + 32 + 64 + 128 + (2 ** 32 - 2 ** 10)
    assert words.tolist() == [w0, 2 ** 18 - 1]


def test_hand_encoded_with_k():
    # all codes 5 -> symbol 11 = 0b1011; k = 2: u = 2 -> "1 1 0" + low bits
    # 1, 1 (least significant first) = 5 bits; k = 3 also gives 5 (tie: k = 2)
    k, nbits, words = rice.encode_one(np.array([5, 5], dtype=np.int16))
    assert k == 2 and nbits == 10
    one = 0b11011  # bits 1, 1, 0, 1, 1
    assert words.tolist() == [one | (one << 5)]


@pytest.mark.parametrize("scale", [0.3, 3.0, 300.0, 20000.0])
def test_round_trip(scale):
    rng = np.random.default_rng(int(scale * 10))
    q = np.clip(np.rint(rng.laplace(0, scale, size=(6, 150))), -32766, 32766).astype(np.int16)
    q[0, :10] = ZERO
    q[1, 5] = ESC
    q[2, :] = ZERO
    q[3, 7] = 32766
    q[3, 8] = -32766
    ks, nb, off, words = rice.encode(q)
    np.testing.assert_array_equal(rice.decode(ks, off, words, q.shape[1]), q)
    for b in range(q.shape[0]):
        syms = [rice.symbol(int(c)) for c in q[b]]
        assert nb[b] == sum(rice.symbol_bits(s, int(ks[b])) for s in syms)
        assert off[b + 1] - off[b] == (int(nb[b]) + 31) // 32


def test_symbol_map_is_a_bijection_on_codes():
    codes = list(range(-32766, 32767)) + [ZERO, ESC]
    syms = [rice.symbol(c) for c in codes]
    assert len(set(syms)) == len(codes)
    assert all(rice.code_of(s) == c for s, c in zip(syms, codes))
    assert rice.symbol(0) == 1 and rice.symbol(-1) == 2 and rice.symbol(1) == 3


@pytest.mark.parametrize("theta", [0.5, 0.84, 0.97])
def test_rice_length_matches_geometric_closed_form(theta):
    # symbols ~ Geometric(1 - theta) on {0, 1, ...}: u = s >> k is geometric
    # with parameter theta^(2^k), so the expected length is
    # E(k) = theta^m / (1 - theta^m) + 1 + k with m = 2^k (no cap reached)
    rng = np.random.default_rng(7)
    s = rng.geometric(1 - theta, size=40000) - 1
    expect = [theta ** (2 ** k) / (1 - theta ** (2 ** k)) + 1 + k for k in range(16)]
    k = rice.best_k(s.tolist())
    assert k == int(np.argmin(expect))
    lens = np.array([rice.symbol_bits(int(v), k) for v in s], dtype=np.float64)
    se = lens.std() / np.sqrt(len(lens))
    assert abs(lens.mean() - expect[k]) <= 4 * se
