"""The oracle against what the paper and the mathematics fix (CPU only)."""
import pytest

import oracle
from tests import pins


@pytest.mark.parametrize("check", pins.ALL_CHECKS, ids=lambda f: f.__name__)
def test_pin(check):
    check(oracle.lib())


def test_full_period_of_update_matrix():
    pins.check_full_period()


def test_seed_zero_is_the_papers_generator():
    # Reading R1: with seed 0 the hash input is the 32-bit id alone.
    for g in [0, 1, 2, 1000, 2**32 - 1]:
        x = oracle.hash_low(g)
        assert oracle.initial_state(g, 0) == (oracle.hash_high(x) << 32) | x


def test_first_values_nonzero_over_many_ids():
    o = oracle.lib()
    out = o.generate(1 << 14, 0, 3)
    assert (out != 0).all()
    assert len(set(out[0].tolist())) == out.shape[1]  # hash of distinct ids: a permutation


def test_empty_sizes():
    o = oracle.lib()
    assert o.generate(0, 1, 5).shape == (5, 0)
    assert o.generate(4, 1, 0).shape == (0, 4)
    rx, rs, _ = o.row_checksums(0, 1, 3)
    assert (rx == 0).all() and (rs == 0).all()
