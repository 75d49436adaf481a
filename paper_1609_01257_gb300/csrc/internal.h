// Library-internal declarations shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/rng.h"

namespace rngi {

// Sets *err (when err != NULL and *err == NULL) and returns `code`.
int fail(rng_err **err, int code, const char *fmt, ...) __attribute__((format(printf, 3, 4)));
// Wraps a CUDA status: RNG_OK, or RNG_ECUDA / RNG_ENOMEM with the call named.
int cuda_fail(rng_err **err, cudaError_t st, const char *what);

void live_inc();
void live_dec();
void count_launch(uint64_t n = 1);

// Kernel launch descriptors -------------------------------------------------

// One launch of the row kernel: streams [s_begin, s_end) of a generator,
// `rows` consecutive iterations, value (r, s) stored at out[r * pitch + (s - s_begin)].
struct RowsLaunch {
  uint64_t *state;      // state array of the whole generator (index s)
  uint64_t *out;        // nullptr: do not store (state advance only)
  uint64_t pitch;
  uint64_t s_begin, s_end;
  uint64_t id_base;     // global id of stream 0
  uint64_t rows;
  uint32_t key;
  int from_hash;        // initial state from the hash instead of `state`
  int write_state;      // store the advanced states back
};

struct LaunchShape {
  uint32_t vpt;
  uint32_t block;
  uint32_t grid;
};

// Picks values-per-thread (if vpt == 0), block size and a persistent grid.
LaunchShape rows_shape(uint64_t streams, uint32_t vpt, uint32_t block, int device);
cudaError_t launch_rows(const RowsLaunch &a, const LaunchShape &sh, int store_policy,
                        cudaStream_t st);
cudaError_t launch_init(uint64_t *state, uint64_t n, uint64_t id_base, uint32_t key,
                        cudaStream_t st);
cudaError_t launch_checksum(const RowsLaunch &a, const LaunchShape &sh, uint64_t *row_xor,
                            uint64_t *row_sum, cudaStream_t st);
int device_sm_count(int device);

// Batched kernel tables.
struct BatchInstance {
  uint64_t *out;
  uint64_t streams;
  uint64_t rows;
  uint32_t key;
  uint32_t vec;     // 1: rows are 16-byte aligned (vector stores allowed)
};
struct BatchUnit {
  uint32_t inst;
  uint32_t count;   // streams in this unit (<= tile)
  uint64_t s_begin;
};
cudaError_t launch_batch(const BatchInstance *inst, const BatchUnit *units, uint32_t n_units,
                         uint32_t *counter, uint32_t vpt, uint32_t block, uint32_t grid,
                         cudaStream_t st);
int batch_blocks_per_sm(uint32_t vpt, uint32_t block);

}  // namespace rngi
