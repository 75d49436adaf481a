"""Jump-ahead (rng_skip) against the oracle: small skips against stepping
one iteration at a time, huge skips against the independent GF(2) matrix
formulation (matrix powers), and the full period 2^64 - 1."""
import numpy as np
import pytest

import oracle
import paper_1609_01257_gb300 as rng
from oracle import gf2

pytestmark = pytest.mark.gpu

M = gf2.xorshift_matrix()


@pytest.mark.parametrize("k", [0, 1, 2, 7, 64, 1000, 4097])
@pytest.mark.parametrize("fuse", [True, False])
def test_small_skip_equals_stepping(k, fuse):
    n = 3001
    g = rng.Generator(n, 5, fuse_init=fuse)
    g.skip(k)
    assert g.position == k
    got = g.generate(3).cpu().numpy()
    g.close()
    assert np.array_equal(got, oracle.generate(n, 5, 3, p0=k))


def test_skip_between_generates():
    n = 1000
    g = rng.Generator(n, 9)
    a = g.generate(3).cpu().numpy()
    g.skip(5)
    b = g.generate(2).cpu().numpy()
    g.close()
    want = oracle.generate(n, 9, 10)
    assert np.array_equal(a, want[:3]) and np.array_equal(b, want[8:10])


@pytest.mark.parametrize("k", [1 << 40, (1 << 63) + 5, (1 << 64) - 2])
def test_huge_skip_matches_matrix_power(k):
    n = 64
    g = rng.Generator(n, 77)
    g.skip(k)
    got = g.generate(2).cpu().numpy()
    g.close()
    for i in range(2):
        mk = gf2.power(M, (k + i) % ((1 << 64) - 1))
        for s in range(0, n, 7):
            assert int(got[i, s]) == gf2.apply(mk, oracle.initial_state(s, 77)), (i, s)


def test_full_period_returns_to_start():
    n = 4096
    g = rng.Generator(n, 3)
    first = g.generate(1).cpu().numpy()
    g.init()
    g.skip((1 << 64) - 1)
    again = g.generate(1).cpu().numpy()
    g.close()
    assert np.array_equal(first, again)


def test_checkpoint_and_resume():
    # Save (states, position) mid-run, restore into a new generator, continue.
    n = 5000
    a = rng.Generator(n, 44)
    a.generate(7)
    states, pos = a.state(), a.position
    rest_a = a.generate(5).cpu().numpy()
    a.close()
    b = rng.Generator(n, 44, init=False)
    b.set_state(states, pos)
    rest_b = b.generate(5).cpu().numpy()
    assert b.position == 12
    b.close()
    assert np.array_equal(rest_a, rest_b)
    assert np.array_equal(rest_b, oracle.generate(n, 44, 5, p0=7))
