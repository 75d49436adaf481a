"""Second, independent formulation of the xorshift update as a linear map.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Listing S5 updates the 64-bit state with three xorshifts: left by 21, right
by 35, left by 4 (Marsaglia's xorshift generator, which the paper cites).
Each xorshift ``s ^= s << k`` is the linear map ``I + L^k`` over GF(2)^64,
where ``L`` moves bit j to bit j+1 and ``R`` moves bit j to bit j-1.  The
update is therefore the matrix

    M = (I + L^4) (I + R^35) (I + L^21)

and ``k`` updates are ``M^k``.  Here a matrix is a tuple of 64 column words:
column ``j`` is the image of the unit vector ``e_j``, so ``M v`` is the XOR
of the columns selected by the set bits of ``v``.  Nothing in this module
calls the oracle's C code; it is built from shift matrices alone.
"""
from __future__ import annotations

from typing import Sequence, Tuple

W = 64
MASK = (1 << W) - 1
Matrix = Tuple[int, ...]


def identity() -> Matrix:
    return tuple(1 << j for j in range(W))


def shift_left(k: int) -> Matrix:
    """L^k: bit j goes to bit j+k (dropped past bit 63)."""
    return tuple(((1 << (j + k)) & MASK) if j + k < W else 0 for j in range(W))


def shift_right(k: int) -> Matrix:
    """R^k: bit j goes to bit j-k (dropped below bit 0)."""
    return tuple((1 << (j - k)) if j - k >= 0 else 0 for j in range(W))


def add(a: Matrix, b: Matrix) -> Matrix:
    """Sum over GF(2): column-wise XOR."""
    return tuple(x ^ y for x, y in zip(a, b))


def apply(m: Matrix, v: int) -> int:
    """Matrix-vector product over GF(2)."""
    acc = 0
    j = 0
    while v:
        if v & 1:
            acc ^= m[j]
        v >>= 1
        j += 1
    return acc


def mul(a: Matrix, b: Matrix) -> Matrix:
    """Product ``a b`` (apply ``b`` first): column j of ab is a (b e_j)."""
    return tuple(apply(a, col) for col in b)


def power(m: Matrix, e: int) -> Matrix:
    """``m^e`` by repeated squaring (e >= 0)."""
    result = identity()
    base = m
    while e:
        if e & 1:
            result = mul(base, result)
        base = mul(base, base)
        e >>= 1
    return result


def xorshift_matrix(a: int = 21, b: int = 35, c: int = 4) -> Matrix:
    """The update of Listing S5 as ``(I + L^c)(I + R^b)(I + L^a)``."""
    i = identity()
    first = add(i, shift_left(a))
    second = add(i, shift_right(b))
    third = add(i, shift_left(c))
    return mul(third, mul(second, first))


def rank(m: Sequence[int]) -> int:
    """Rank over GF(2) of the columns of ``m`` (Gaussian elimination)."""
    basis: list[int] = []
    for col in m:
        v = col
        for bvec in basis:
            v = min(v, v ^ bvec)
        if v:
            basis.append(v)
            basis.sort(reverse=True)
    return len(basis)


# Prime factors of 2^64 - 1 = 3 * 5 * 17 * 257 * 641 * 65537 * 6700417.
PERIOD_PRIMES = (3, 5, 17, 257, 641, 65537, 6700417)
