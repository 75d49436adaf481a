// Generator arithmetic of the cf4ocl PRNG example (Section 5), written for
// the GPU library.  Host and device share these inline functions so the
// host can derive launch constants (the seed key) exactly as kernels would.
//
//  * init hash (Listing S4): a six-round 32-bit hash of the stream id gives
//    the low word x; a five-round multiply/shift hash of x gives the high
//    word y; the state is (y << 32) | x -- the {x, y} pair of 32-bit words
//    stored by the init kernel and read back as one little-endian 64-bit
//    word by the rng kernel.
//  * update (Listing S5): 64-bit xorshift with the triple (21, 35, 4).
//  * seed: the paper hashes the id alone; a run seed is folded in by XORing
//    the 32-bit id with key(seed) = lo32(m) ^ hi32(m), m = splitmix64
//    finaliser of the seed.  key(0) = 0 reproduces the paper's generator.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define PRNG_HD __host__ __device__ __forceinline__
#else
#define PRNG_HD inline
#endif

namespace prng {

// Rounds of the form (v + c) + (v << k) are written as v * (2^k + 1) + c,
// which is the same value modulo 2^32 and maps to one integer multiply-add.
PRNG_HD uint32_t id_hash_low(uint32_t v) {
  v = v * 4097u + 0x7ed55d16u;            // (v + c) + (v << 12)
  v = v ^ 0xc761c23cu ^ (v >> 19);
  v = v * 33u + 0x165667b1u;              // (v + c) + (v << 5)
  v = (v + 0xd3a2646cu) ^ (v << 9);       // mixed add/xor round, as printed
  v = v * 9u + 0xfd7046c5u;               // (v + c) + (v << 3)
  v = v ^ 0xb55a4f09u ^ (v >> 16);
  return v;
}

PRNG_HD uint32_t id_hash_high(uint32_t v) {
  v = v ^ 61u ^ (v >> 16);
  v = v * 9u;                             // v + (v << 3)
  v = v ^ (v >> 4);
  v = v * 0x27d4eb2du;
  v = v ^ (v >> 15);
  return v;
}

PRNG_HD uint64_t splitmix_finalise(uint64_t z) {
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

PRNG_HD uint32_t seed_key(uint64_t seed) {
  const uint64_t m = splitmix_finalise(seed);
  return static_cast<uint32_t>(m) ^ static_cast<uint32_t>(m >> 32);
}

// Initial state (= iteration-0 output) of the stream with global id `id`.
PRNG_HD uint64_t initial_state(uint64_t id, uint32_t key) {
  const uint32_t lo = id_hash_low(static_cast<uint32_t>(id) ^ key);
  const uint32_t hi = id_hash_high(lo);
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

PRNG_HD uint64_t xorshift_update(uint64_t s) {
  s ^= s << 21;
  s ^= s >> 35;
  s ^= s << 4;
  return s;
}

// Alternative output mode: the xorshift64* scrambler (Vigna, "An experimental
// exploration of Marsaglia's xorshift generators, scrambled", ACM TOMS 42(4),
// 2016) -- the value emitted for a state is the state times this odd
// constant modulo 2^64; the state sequence itself is unchanged.
constexpr uint64_t kStarMultiplier = 0x2545F4914F6CDD1Dull;

// Value emitted for state s in output mode OUT (0: the state, as in the
// paper; 1: xorshift64*).
template <int OUT>
PRNG_HD uint64_t emitted(uint64_t s) {
  return OUT ? s * kStarMultiplier : s;
}

}  // namespace prng
