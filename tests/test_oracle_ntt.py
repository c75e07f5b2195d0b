"""Pins the oracle's negacyclic NTT (section 2.2).

The transform is pinned by (i) the O(n^2) definition equalling the radix-2
butterfly form, (ii) NTT and INTT being mutual inverses, and (iii) products
through the NTT equalling the schoolbook negacyclic convolution in Z_q[X]/(X^256+1)
(exhaustive on monomials, random otherwise).  The output *order* (bit-reversed,
zeta = 1753) is the round-3 specification's reading and is not pinned by any
printed value.
"""
import numpy as np
import pytest

Q = 8380417


def schoolbook(a, b):
    a = [int(x) for x in a]
    b = [int(x) for x in b]
    c = [0] * 256
    for i in range(256):
        if a[i] == 0:
            continue
        for j in range(256):
            if i + j < 256:
                c[i + j] += a[i] * b[j]
            else:
                c[i + j - 256] -= a[i] * b[j]
    return np.array([x % Q for x in c], dtype=np.int64)


def test_root_of_unity():
    assert pow(1753, 256, Q) == Q - 1     # order exactly 512
    assert pow(1753, 512, Q) == 1


def test_definition_equals_butterflies(orc):
    rng = np.random.default_rng(11)
    for _ in range(6):
        a = rng.integers(0, Q, 256).astype(np.int32)
        assert np.array_equal(orc.ntt_def(a), orc.ntt(a))
        assert np.array_equal(orc.intt_def(a), orc.intt(a))


def test_inverse_pairs(orc):
    rng = np.random.default_rng(12)
    for _ in range(50):
        a = rng.integers(0, Q, 256).astype(np.int32)
        assert np.array_equal(orc.intt(orc.ntt(a)), a)
        assert np.array_equal(orc.ntt(orc.intt(a)), a)
    a = rng.integers(0, Q, 256).astype(np.int32)
    assert np.array_equal(orc.intt_def(orc.ntt_def(a)), a)


def test_linearity_and_constant(orc):
    one = np.zeros(256, dtype=np.int32)
    one[0] = 1
    assert np.all(orc.ntt(one) == 1)            # the constant 1 evaluates to 1 everywhere
    rng = np.random.default_rng(13)
    a = rng.integers(0, Q, 256)
    b = rng.integers(0, Q, 256)
    lhs = orc.ntt(((a + b) % Q).astype(np.int32)).astype(np.int64)
    rhs = (orc.ntt(a.astype(np.int32)).astype(np.int64) + orc.ntt(b.astype(np.int32))) % Q
    assert np.array_equal(lhs, rhs)


def test_monomial_products_exhaustive(orc):
    # X^a * X^b = X^(a+b) if a+b < 256 else -X^(a+b-256)
    for a in range(256):
        fa = np.zeros(256, dtype=np.int32)
        fa[a] = 1
        for b in range(0, 256, 1 if a % 16 == 0 else 17):
            fb = np.zeros(256, dtype=np.int32)
            fb[b] = 1
            want = np.zeros(256, dtype=np.int64)
            if a + b < 256:
                want[a + b] = 1
            else:
                want[a + b - 256] = Q - 1
            assert np.array_equal(orc.poly_mul(fa, fb), want), (a, b)


@pytest.mark.parametrize("seed", range(6))
def test_random_products_match_schoolbook(orc, seed):
    rng = np.random.default_rng(100 + seed)
    if seed % 2:
        a = rng.integers(0, Q, 256)
        b = rng.integers(0, Q, 256)
    else:  # the shapes the scheme multiplies: sparse +-1 times a full polynomial
        a = np.zeros(256, dtype=np.int64)
        a[rng.choice(256, 39, replace=False)] = rng.choice([1, Q - 1], 39)
        b = rng.integers(0, Q, 256)
    assert np.array_equal(orc.poly_mul(a.astype(np.int32), b.astype(np.int32)), schoolbook(a, b))


def test_definition_form_products(orc):
    rng = np.random.default_rng(14)
    a = rng.integers(0, Q, 256)
    b = rng.integers(-4, 5, 256) % Q
    orc.use_def_ntt(True)
    try:
        got = orc.poly_mul(a.astype(np.int32), b.astype(np.int32))
    finally:
        orc.use_def_ntt(False)
    assert np.array_equal(got, schoolbook(a, b))
