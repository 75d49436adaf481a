"""Pins of the CPU oracle to facts other than itself.

Each ``check_*`` function takes an oracle handle (``oracle.OracleLib``) and
raises ``AssertionError`` on a mismatch.  ``test_oracle_pins`` runs them on
the real oracle; ``test_oracle_mutants`` runs them on copies of the oracle
with planted mistakes and requires that every mistake is caught.

What pins what:
* the two 32-bit hashes of Listing S4 and the splitmix64 finaliser used for
  the seed (reading R1) are pinned by round trips through inverses derived
  here by algebra from each printed round (modular inverses of the
  multipliers, inversion of xorshifts), not by re-evaluating the rounds;
* the xorshift update of Listing S5 is pinned by the independent GF(2)
  matrix formulation in ``oracle.gf2`` and by the maximal period 2^64 - 1
  that the shift triple (21, 35, 4) must give;
* the iteration-major layout and readings R2/R3 are pinned by brute force
  against matrix powers on tiny inputs;
* the XOR row checksum by its closed form (linearity), the wrapping sum by
  Python integers;
* the alternative output mode (reading R11, xorshift64*: state times an odd
  published constant) by undoing the multiplication with the constant's
  modular inverse, which must give back the paper's pinned state sequence,
  and its checksums by Python integers over the emitted values.
"""
from __future__ import annotations

import random

from oracle import gf2

M32 = (1 << 32) - 1
M64 = (1 << 64) - 1

EDGE32 = [0, 1, 2, 3, 61, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, M32, 0x12345678, 0xDEADBEEF]
EDGE64 = [0, 1, 2, M64, 1 << 63, (1 << 63) - 1, 0x0123456789ABCDEF, 0xFEDCBA9876543210]


def _unxorshift_right(y: int, k: int, mask: int, bits: int) -> int:
    """Solve ``y = a ^ (a >> k)`` for ``a`` (each pass fixes k more top bits)."""
    a = y
    for _ in range(bits // k + 1):
        a = (y ^ (a >> k)) & mask
    return a


def inverse_hash_low(y: int) -> int:
    """Inverse of the six-round low-word hash of Listing S4, round by round.

    Rounds of the form ``(a + c) + (a << k)`` are the affine maps
    ``a * (1 + 2^k) + c`` mod 2^32 and are undone with the modular inverse of
    the odd factor.  The fourth round, printed as ``(a + c) ^ (a << 9)``, is
    solved from the low bits up: if ``a`` is right in its low m bits then
    ``(y ^ (a << 9)) - c`` is right in its low m+9 bits.
    """
    a = _unxorshift_right(y ^ 0xB55A4F09, 16, M32, 32)               # round 6
    a = ((a - 0xFD7046C5) * pow(9, -1, 1 << 32)) & M32               # round 5
    y4 = a
    a = 0
    for _ in range(5):                                               # round 4
        a = ((y4 ^ ((a << 9) & M32)) - 0xD3A2646C) & M32
    a = ((a - 0x165667B1) * pow(33, -1, 1 << 32)) & M32              # round 3
    a = _unxorshift_right(a ^ 0xC761C23C, 19, M32, 32)               # round 2
    a = ((a - 0x7ED55D16) * pow(4097, -1, 1 << 32)) & M32            # round 1
    return a


def inverse_hash_high(y: int) -> int:
    """Inverse of the five-round high-word hash of Listing S4."""
    a = _unxorshift_right(y, 15, M32, 32)                            # round 5
    a = (a * pow(0x27D4EB2D, -1, 1 << 32)) & M32                     # round 4
    a = _unxorshift_right(a, 4, M32, 32)                             # round 3
    a = (a * pow(9, -1, 1 << 32)) & M32                              # round 2: a + (a << 3)
    a = _unxorshift_right(a ^ 61, 16, M32, 32)                       # round 1
    return a


def inverse_mix64(y: int) -> int:
    """Inverse of the splitmix64 output finaliser (reading R1)."""
    a = _unxorshift_right(y, 31, M64, 64)
    a = (a * pow(0x94D049BB133111EB, -1, 1 << 64)) & M64
    a = _unxorshift_right(a, 27, M64, 64)
    a = (a * pow(0xBF58476D1CE4E5B9, -1, 1 << 64)) & M64
    a = _unxorshift_right(a, 30, M64, 64)
    return a


def _rand32(rng, n):
    return EDGE32 + [rng.getrandbits(32) for _ in range(n)]


def _rand64(rng, n):
    return EDGE64 + [rng.getrandbits(64) for _ in range(n)]


def check_hash_low(o, n=2000):
    rng = random.Random(1)
    for a in _rand32(rng, n):
        y = o.hash_low(a)
        assert inverse_hash_low(y) == a, f"hash_low round trip fails at {a:#x}"


def check_hash_high(o, n=2000):
    rng = random.Random(2)
    for a in _rand32(rng, n):
        y = o.hash_high(a)
        assert inverse_hash_high(y) == a, f"hash_high round trip fails at {a:#x}"
    # Nonzero invariant: the high hash of 0 is nonzero, so no initial state is 0.
    assert o.hash_high(0) != 0


def check_mix64(o, n=2000):
    assert o.mix64(0) == 0, "mix64(0) must be 0 so that seed 0 is the paper's generator"
    rng = random.Random(3)
    for z in _rand64(rng, n):
        assert inverse_mix64(o.mix64(z)) == z, f"mix64 round trip fails at {z:#x}"


def check_seed_key(o, n=500):
    assert o.seed_key(0) == 0
    rng = random.Random(4)
    for s in _rand64(rng, n):
        m = o.mix64(s)
        assert o.seed_key(s) == ((m & M32) ^ (m >> 32))


def check_initial_state(o, n=2000):
    """R1/R3/R4: low word = hash_low(g32 ^ key), high word = hash_high(low)."""
    rng = random.Random(5)
    seeds = [0, 1, 12345, 99, 7, M64, rng.getrandbits(64)]
    for seed in seeds:
        key = o.seed_key(seed)
        gs = [0, 1, 2, 1023, 65535, M32, (1 << 32), (1 << 32) + 5, rng.getrandbits(40)]
        gs += [rng.getrandbits(32) for _ in range(n // len(seeds))]
        for g in gs:
            s0 = o.initial_state(g, seed)
            lo, hi = s0 & M32, s0 >> 32
            assert inverse_hash_low(lo) == (g & M32) ^ key, (g, seed)
            assert inverse_hash_high(hi) == lo, (g, seed)
            assert s0 != 0


def check_seed_alias_property(o):
    """Documented consequence of R1: (seed, g) and (seed', g') start the same
    stream exactly when g32 ^ key(seed) == g'32 ^ key(seed')."""
    for seed, seed2 in [(0, 1), (12345, 99), (7, 1 << 40)]:
        k1, k2 = o.seed_key(seed), o.seed_key(seed2)
        for g in (0, 5, 1000, M32):
            g2 = (g & M32) ^ k1 ^ k2
            assert o.initial_state(g, seed) == o.initial_state(g2, seed2)
            assert o.initial_state(g, seed) != o.initial_state(g2 ^ 1, seed2)


_M = gf2.xorshift_matrix(21, 35, 4)


def check_step_gf2(o, n=2000):
    rng = random.Random(6)
    for j in range(64):
        assert o.step(1 << j) == _M[j], f"column {j} of the update differs from the GF(2) matrix"
    for s in _rand64(rng, n):
        assert o.step(s) == gf2.apply(_M, s)
    for _ in range(200):
        a, b = rng.getrandbits(64), rng.getrandbits(64)
        assert o.step(a ^ b) == o.step(a) ^ o.step(b)
    assert o.step(0) == 0


def check_full_period():
    """The GF(2) matrix itself: order exactly 2^64 - 1 (maximal period)."""
    assert gf2.rank(_M) == 64
    assert gf2.power(_M, M64) == gf2.identity()
    for p in gf2.PERIOD_PRIMES:
        assert gf2.power(_M, M64 // p) != gf2.identity(), p


def check_step_k(o):
    rng = random.Random(7)
    for k in list(range(0, 70)) + [100, 1000, 4097]:
        mk = gf2.power(_M, k)
        s = rng.getrandbits(64) | 1
        assert o.step_k(s, k) == gf2.apply(mk, s), k


def check_generate_layout(o):
    """R2 + iteration-major layout: out[i, g] = M^i s0(g), brute force."""
    for n_streams, seed, t in [(1, 0, 1), (5, 0, 7), (3, 12345, 9), (8, 99, 4)]:
        out = o.generate(n_streams, seed, t)
        assert out.shape == (t, n_streams)
        for i in range(t):
            mi = gf2.power(_M, i)
            for g in range(n_streams):
                assert int(out[i, g]) == gf2.apply(mi, o.initial_state(g, seed)), (i, g)


def check_generate_offsets(o):
    """Position p0 and stream offset g0 select a window of a larger run."""
    full = o.generate(12, 3, 10)
    assert (o.generate(5, 3, 6, p0=4, g0=7) == full[4:10, 7:12]).all()
    assert (o.generate(12, 3, 3, p0=2) == full[2:5]).all()
    for i, g in [(0, 0), (9, 11), (4, 5)]:
        assert o.value(g, 3, i) == int(full[i, g])


def check_row_checksums(o):
    n_streams, seed, t = 37, 12345, 11
    out = o.generate(n_streams, seed, t)
    rx, rs, samples = o.row_checksums(n_streams, seed, t, sample_every=4)
    x0 = 0
    for g in range(n_streams):
        x0 ^= o.initial_state(g, seed)
    for i in range(t):
        # XOR over streams commutes with the linear update: closed form.
        assert int(rx[i]) == gf2.apply(gf2.power(_M, i), x0), i
        assert int(rs[i]) == sum(int(v) for v in out[i]) % (1 << 64), i
    assert (samples == out[::4]).all()
    rx2, rs2, _ = o.row_checksums(n_streams, seed, 5, p0=6)
    assert (rx2 == rx[6:]).all() and (rs2 == rs[6:]).all()


# xorshift64* multiplier (Vigna, "An experimental exploration of Marsaglia's
# xorshift generators, scrambled", ACM TOMS 42(4), 2016).
STAR_MULTIPLIER = 2685821657736338717
STAR_INVERSE = pow(STAR_MULTIPLIER, -1, 1 << 64)


def check_star_output(o):
    """R11: every value of output mode 1, multiplied by the inverse of the
    xorshift64* constant modulo 2^64, is the mode-0 value (the state), at the
    same (iteration, stream); windows and single values agree with it."""
    assert STAR_MULTIPLIER % 2 == 1 and (STAR_MULTIPLIER * STAR_INVERSE) % (1 << 64) == 1
    for n_streams, seed, t, p0, g0 in [(1, 0, 3, 0, 0), (9, 12345, 6, 0, 0), (7, 99, 5, 4, 11)]:
        plain = o.generate(n_streams, seed, t, p0=p0, g0=g0)
        star = o.generate(n_streams, seed, t, p0=p0, g0=g0, output_mode=1)
        for i in range(t):
            for g in range(n_streams):
                assert (int(star[i, g]) * STAR_INVERSE) % (1 << 64) == int(plain[i, g]), (seed, i, g)
        c = 2 % n_streams
        assert o.value(g0 + c, seed, p0 + t - 1, 1) == int(star[t - 1, c])
    for s in EDGE64:
        assert (o.output(s, 1) * STAR_INVERSE) % (1 << 64) == s and o.output(s, 0) == s


def check_star_row_checksums(o):
    n_streams, seed, t = 29, 7, 9
    star = o.generate(n_streams, seed, t, output_mode=1)
    rx, rs, samples = o.row_checksums(n_streams, seed, t, sample_every=3, output_mode=1)
    for i in range(t):
        x = 0
        for v in star[i]:
            x ^= int(v)
        assert int(rx[i]) == x, i
        assert int(rs[i]) == sum(int(v) for v in star[i]) % (1 << 64), i
    assert (samples == star[::3]).all()


ALL_CHECKS = [
    check_hash_low, check_hash_high, check_mix64, check_seed_key, check_initial_state,
    check_seed_alias_property, check_step_gf2, check_step_k, check_generate_layout,
    check_generate_offsets, check_row_checksums, check_star_output, check_star_row_checksums,
]
