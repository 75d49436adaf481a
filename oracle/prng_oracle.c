/*
 * CPU oracle for the massive pseudo-random number generator of the cf4ocl
 * paper (Fachada et al., "cf4ocl: a C framework for OpenCL", Section 5,
 * "Example: massive pseudo-random number generator", with its init and rng
 * kernels in Listings S4 and S5).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the GPU library is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may build, load or
 * call it; the product path never does.  It shares no code, header or
 * constant table with the CUDA library.
 *
 * Everything is unsigned integer arithmetic: 32-bit words for the hash
 * (wrapping modulo 2^32) and 64-bit words for the generator state (wrapping
 * modulo 2^64).  Shifts are logical.
 *
 * Readings of points the paper leaves open (each one is listed with its
 * reason in the design notes):
 *   R1  seed: the paper hashes the work-item id alone.  A run seed enters as
 *       key(seed) = lo32(mix64(seed)) XOR hi32(mix64(seed)), XORed into the
 *       32-bit id before the hash.  mix64 is the splitmix64 output finaliser
 *       (Steele, Lea and Flood, OOPSLA 2014).  mix64(0) = 0, so seed 0 is the
 *       paper's generator exactly.
 *   R2  iteration 0 is the init value itself; iteration i > 0 is the state
 *       after i xorshift steps (Section 5: the init values are the first
 *       batch and also seed the next one).
 *   R3  the init kernel stores a pair of 32-bit words {x, y} which the rng
 *       kernel reads back as one 64-bit word; on a little-endian device the
 *       state is (y << 32) | x.
 *   R4  the id is reduced to 32 bits before hashing (Listing S4 casts it).
 *   R8  row checksums are the XOR and the wrapping sum of one iteration's
 *       values over all streams.
 *   R11 alternative output (the stronger generator the paper suggests
 *       could replace plain xorshift): the xorshift64* scrambler of Vigna
 *       ("An experimental exploration of Marsaglia's xorshift generators,
 *       scrambled", ACM TOMS 42(4), 2016), i.e. the emitted value is the
 *       state times the odd constant 2685821657736338717 modulo 2^64.  The
 *       state sequence is the paper's, unchanged.  Output mode 0 is the
 *       paper's (the state itself), mode 1 the scrambled value.
 *
 * Build: gcc -O2 -shared -fPIC prng_oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Listing S4, low word: six add/xor/shift rounds on a 32-bit word.    */
/* ------------------------------------------------------------------ */
uint32_t oracle_hash_low(uint32_t a)
{
    uint32_t r = a;
    r = (r + 0x7ed55d16u) + (r << 12);
    r = (r ^ 0xc761c23cu) ^ (r >> 19);
    r = (r + 0x165667b1u) + (r << 5);
    r = (r + 0xd3a2646cu) ^ (r << 9);   /* printed with a mixed + and ^ */
    r = (r + 0xfd7046c5u) + (r << 3);
    r = (r ^ 0xb55a4f09u) ^ (r >> 16);
    return r;
}

/* ------------------------------------------------------------------ */
/* Listing S4, high word: five rounds applied to the low word (the     */
/* multiply-shift integer hash the paper cites to Wang).               */
/* ------------------------------------------------------------------ */
uint32_t oracle_hash_high(uint32_t a)
{
    uint32_t r = a;
    r = (r ^ 61u) ^ (r >> 16);
    r = r + (r << 3);
    r = r ^ (r >> 4);
    r = r * 0x27d4eb2du;
    r = r ^ (r >> 15);
    return r;
}

/* ------------------------------------------------------------------ */
/* Reading R1: splitmix64 output finaliser, and the 32-bit seed key.   */
/* ------------------------------------------------------------------ */
uint64_t oracle_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    z = z ^ (z >> 31);
    return z;
}

uint32_t oracle_seed_key(uint64_t seed)
{
    uint64_t m = oracle_mix64(seed);
    return (uint32_t)(m & 0xffffffffu) ^ (uint32_t)(m >> 32);
}

/* ------------------------------------------------------------------ */
/* Section 5 / Listing S4: the initial state of stream g (readings R1, */
/* R3, R4).  This value is also the stream's output for iteration 0.   */
/* ------------------------------------------------------------------ */
uint64_t oracle_initial_state(uint64_t g, uint64_t seed)
{
    uint32_t id32 = (uint32_t)(g & 0xffffffffu);
    uint32_t x = oracle_hash_low(id32 ^ oracle_seed_key(seed));
    uint32_t y = oracle_hash_high(x);
    return ((uint64_t)y << 32) | (uint64_t)x;
}

/* ------------------------------------------------------------------ */
/* Listing S5: one xorshift update, shift triple (21, 35, 4), applied  */
/* as left 21, right 35, left 4 (Marsaglia's xorshift, cited in S5).   */
/* ------------------------------------------------------------------ */
uint64_t oracle_step(uint64_t s)
{
    s = s ^ (s << 21);
    s = s ^ (s >> 35);
    s = s ^ (s << 4);
    return s;
}

/* k applications of the update, one at a time. */
uint64_t oracle_step_k(uint64_t s, uint64_t k)
{
    for (uint64_t j = 0; j < k; ++j)
        s = oracle_step(s);
    return s;
}

/* Output value of stream g at iteration i (reading R2), computed alone. */
uint64_t oracle_value(uint64_t g, uint64_t seed, uint64_t i)
{
    return oracle_step_k(oracle_initial_state(g, seed), i);
}

/* Reading R11: the value emitted for state s in output mode `mode`. */
uint64_t oracle_output(uint64_t s, int mode)
{
    return mode ? s * 2685821657736338717ull : s;
}

/* Output value of stream g at iteration i in output mode `mode`. */
uint64_t oracle_value_mode(uint64_t g, uint64_t seed, uint64_t i, int mode)
{
    return oracle_output(oracle_value(g, seed, i), mode);
}

/* ------------------------------------------------------------------ */
/* Iterations p0 .. p0+T-1 of N streams, in the iteration-major layout */
/* of Section 5 (one batch of N values per iteration, Eq. 1 gives the  */
/* total 8*N*T bytes): out[(i - p0) * N + g].                           */
/* Streams are numbered from g0 (a shard of a larger generator).       */
/* Returns 0, or -1 if the state array cannot be allocated.            */
/* ------------------------------------------------------------------ */
int oracle_generate_mode(uint64_t n_streams, uint64_t g0, uint64_t seed,
                         uint64_t p0, uint64_t iterations, int mode,
                         uint64_t *out);

int oracle_generate(uint64_t n_streams, uint64_t g0, uint64_t seed,
                    uint64_t p0, uint64_t iterations, uint64_t *out)
{
    return oracle_generate_mode(n_streams, g0, seed, p0, iterations, 0, out);
}

/* The same in output mode `mode` (reading R11). */
int oracle_generate_mode(uint64_t n_streams, uint64_t g0, uint64_t seed,
                         uint64_t p0, uint64_t iterations, int mode,
                         uint64_t *out)
{
    if (n_streams == 0 || iterations == 0)
        return 0;
    uint64_t *state = (uint64_t *)malloc(n_streams * sizeof(uint64_t));
    if (!state)
        return -1;
    for (uint64_t g = 0; g < n_streams; ++g)
        state[g] = oracle_step_k(oracle_initial_state(g0 + g, seed), p0);
    for (uint64_t i = 0; i < iterations; ++i) {
        uint64_t *row = out + i * n_streams;
        for (uint64_t g = 0; g < n_streams; ++g) {
            row[g] = oracle_output(state[g], mode);
            state[g] = oracle_step(state[g]);
        }
    }
    free(state);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Reading R8: per-iteration XOR and wrapping sum over all N streams,  */
/* for iterations p0 .. p0+T-1, without storing the output.  Rows      */
/* whose index (i - p0) is a multiple of sample_every are also copied  */
/* out, one after another, into sample_rows (if it is not NULL).       */
/* ------------------------------------------------------------------ */
int oracle_row_checksums_mode(uint64_t n_streams, uint64_t g0, uint64_t seed,
                              uint64_t p0, uint64_t iterations, int mode,
                              uint64_t *row_xor, uint64_t *row_sum,
                              uint64_t sample_every, uint64_t *sample_rows);

int oracle_row_checksums(uint64_t n_streams, uint64_t g0, uint64_t seed,
                         uint64_t p0, uint64_t iterations,
                         uint64_t *row_xor, uint64_t *row_sum,
                         uint64_t sample_every, uint64_t *sample_rows)
{
    return oracle_row_checksums_mode(n_streams, g0, seed, p0, iterations, 0,
                                     row_xor, row_sum, sample_every, sample_rows);
}

/* The same over the values of output mode `mode` (reading R11). */
int oracle_row_checksums_mode(uint64_t n_streams, uint64_t g0, uint64_t seed,
                              uint64_t p0, uint64_t iterations, int mode,
                              uint64_t *row_xor, uint64_t *row_sum,
                              uint64_t sample_every, uint64_t *sample_rows)
{
    if (iterations == 0)
        return 0;
    uint64_t *state = NULL;
    if (n_streams > 0) {
        state = (uint64_t *)malloc(n_streams * sizeof(uint64_t));
        if (!state)
            return -1;
    }
    for (uint64_t g = 0; g < n_streams; ++g)
        state[g] = oracle_step_k(oracle_initial_state(g0 + g, seed), p0);
    uint64_t n_samples = 0;
    for (uint64_t i = 0; i < iterations; ++i) {
        uint64_t x = 0, s = 0;
        int keep = sample_rows && sample_every && (i % sample_every == 0);
        uint64_t *dst = keep ? sample_rows + n_samples * n_streams : NULL;
        for (uint64_t g = 0; g < n_streams; ++g) {
            uint64_t v = oracle_output(state[g], mode);
            x ^= v;
            s += v;
            if (dst)
                dst[g] = v;
            state[g] = oracle_step(state[g]);
        }
        row_xor[i] = x;
        row_sum[i] = s;
        if (keep)
            ++n_samples;
    }
    free(state);
    return 0;
}
