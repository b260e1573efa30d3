"""Pins of the Rabin fingerprint window (the LBFS-style variant window hash).

Every check here is a fact of polynomial arithmetic over GF(2) that the
fingerprint must satisfy, not a second copy of its long division.
"""
import numpy as np
import pytest

import oracle
from gen import inputs as G
from tests.pins import brute_window_cuts_with

P = oracle.RABIN_POLY


# ---- GF(2)[x] helpers for the facts below (polynomials as Python ints) -----
def _mod(a, p):
    dp = p.bit_length() - 1
    while a and a.bit_length() - 1 >= dp:
        a ^= p << (a.bit_length() - 1 - dp)
    return a


def _mulmod(a, b, p):
    r = 0
    while b:
        if b & 1:
            r ^= a
        b >>= 1
        a <<= 1
    return _mod(r, p)


def _gcd(a, b):
    while b:
        a, b = b, _mod(a, b)
    return a


def test_polynomial_is_irreducible_of_degree_31():
    # Ben-Or: P of degree n is irreducible iff gcd(x^(2^i) - x, P) = 1 for i <= n/2
    assert P.bit_length() - 1 == 31
    xp = 2
    for _ in range(1, 16):
        xp = _mulmod(xp, xp, P)
        assert _gcd(xp ^ 2, P) == 1


def test_polynomial_is_primitive():
    # 2^31 - 1 is prime, so x has order 2^31 - 1 modulo an irreducible P of degree 31
    r, e, b = 1, (1 << 31) - 1, 2
    while e:
        if e & 1:
            r = _mulmod(r, b, P)
        b = _mulmod(b, b, P)
        e >>= 1
    assert r == 1


def test_low_degree_strings_are_their_own_remainder():
    g = np.random.default_rng(1)
    for n in range(0, 4):
        for _ in range(50):
            s = bytes(g.integers(0, 256, n, dtype=np.uint8))
            assert oracle.rabin_fingerprint(s) == int.from_bytes(s, "big")
    for _ in range(50):
        s = bytes(g.integers(0, 256, 4, dtype=np.uint8))
        s = bytes([s[0] & 0x7F]) + s[1:]
        assert oracle.rabin_fingerprint(s) == int.from_bytes(s, "big")
    # leading zero bytes do not change the polynomial
    assert oracle.rabin_fingerprint(b"\0\0\0" + b"\x12\x34") == 0x1234


def test_hand_reduced_powers_of_x():
    assert oracle.rabin_fingerprint(b"\x80\0\0\0") == P ^ (1 << 31)          # x^31 = P - x^31
    assert oracle.rabin_fingerprint(b"\x01\0\0\0\0") == (P ^ (1 << 31)) << 1  # x^32, no carry out
    assert oracle.rabin_fingerprint(b"\x80\0\0\0\0") == _mulmod(1 << 39, 1, P)


def test_linear_over_gf2():
    g = np.random.default_rng(2)
    for n in (5, 20, 48, 100, 1000):
        a = g.integers(0, 256, n, dtype=np.uint8)
        b = g.integers(0, 256, n, dtype=np.uint8)
        fa, fb = oracle.rabin_fingerprint(a), oracle.rabin_fingerprint(b)
        assert oracle.rabin_fingerprint(a ^ b) == fa ^ fb


def test_remainder_and_shift_identities():
    g = np.random.default_rng(3)
    for n in (4, 7, 48, 333):
        s = bytes(g.integers(0, 256, n, dtype=np.uint8))
        t = bytes(g.integers(0, 256, 9, dtype=np.uint8))
        f = oracle.rabin_fingerprint(s)
        assert f < (1 << 31)
        # s = q P + f, so s x^(8k) + t and f x^(8k) + t leave the same remainder
        assert oracle.rabin_fingerprint(s + t) == oracle.rabin_fingerprint(f.to_bytes(4, "big") + t)
        # the remainder equals the product rule of GF(2)[x]/P
        assert oracle.rabin_fingerprint(s + t) == \
            _mod(_mulmod(f, 1 << 72, P) ^ int.from_bytes(t, "big"), P)


@pytest.mark.parametrize("window,mask_bits,magic", [(48, 4, 5), (16, 3, 0), (1, 2, 1), (31, 5, 0x1F)])
def test_candidates_match_per_window_fingerprints(window, mask_bits, magic):
    data = G.uniform_bytes(3000, seed=window).tobytes()
    got = oracle.window_candidates(data, window, mask_bits, magic, kind=oracle.WIN_RABIN)
    want = brute_window_cuts_with(data, window, mask_bits, magic, oracle.rabin_fingerprint)
    assert got.tolist() == want
    got8 = oracle.window_candidates(data, window, mask_bits, magic, nthreads=8, kind=oracle.WIN_RABIN)
    assert got8.tolist() == want


def test_candidate_density_on_uniform_and_text():
    for data in (G.uniform_bytes(1 << 20, 1), G.text_like_bytes(1 << 20, 5)):
        c = oracle.window_candidates(data, 48, 13, 0x0F0F, nthreads=8, kind=oracle.WIN_RABIN)
        assert 60 < len(c) < 260       # about 128 expected at 2^-13 per window


def test_unknown_kind_rejected():
    L = oracle.lib()
    a = np.zeros(100, np.uint8)
    assert L.hgo_window_candidates_kind(a.ctypes.data, 100, 7, 20, 4, 1, None, 0, 1) == 2 ** 64 - 1
