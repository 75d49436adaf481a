// Library-internal declarations shared by the translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/rng.h"

namespace rngi {

constexpr uint32_t kGenBlock = 256;  // threads per block of the generation kernels
constexpr int kStoreDefault = 0;     // st.global
constexpr int kStoreStreaming = 1;   // st.global.cs (evict-first)
constexpr int kStoreBulk = 2;        // rows staged in shared memory, written by TMA bulk copies

// Kernel entry points (kernels.cu); nullptr for shapes that are not compiled.
// banded: the variant that splits rows into bands (few values per thread
// only; store policy is always streaming there).
// out: output mode (0: the state, 1: xorshift64*; mode 1 is compiled for
// 256-thread blocks, streaming stores and 1, 2, 4, 8, 16, 24 or 32 values per
// thread only).
const void *rows_kernel_fn(uint32_t vpt, int width, int policy, uint32_t block, bool banded = false,
                           uint32_t out = 0);
// Row kernel that stages each row in shared memory and stores it in
// line-aligned pieces (for rows that do not start on 128-byte lines); 1, 2,
// 4, 6 or 8 values per thread, 256-thread blocks.
const void *rows_staged_kernel_fn(uint32_t vpt, bool banded, uint32_t out);
// Row kernel whose rows are written by TMA bulk copies from `nb` shared
// buffers (2 or 4 values per thread with 8 buffers, 8 with 4 or 8, 16 with
// 4; 256-thread blocks), and its dynamic shared memory in bytes.
const void *rows_bulk_kernel_fn(uint32_t vpt, uint32_t nb, bool banded, uint32_t out);
size_t rows_bulk_smem_bytes(uint32_t vpt, uint32_t nb);
const void *checksum_kernel_fn(uint32_t vpt, bool banded = false, uint32_t out = 0);
const void *worklist_kernel_fn(uint32_t vpt);
const void *batch_work_kernel_fn(uint32_t vpt);
// Batched form with bulk copies for units of at least 16 rows: (4, 8),
// (8, 6) or (8, 12) values per thread and row buffers; dynamic shared memory
// rows_bulk_smem_bytes(vpt, nb).
const void *batch_work_bulk_kernel_fn(uint32_t vpt, uint32_t nb);
const void *init_kernel_fn();
const void *jump_kernel_fn();
const void *copy_kernel_fn();

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
  uint64_t ring_rows;   // 0, or rows wrap around a ring of this many rows
  uint64_t band_rows;   // 0, or rows are split into bands of this many rows
  const uint64_t *jump; // bands: matrices M^(band * band_rows) for band = 0, 1, ..., 64 columns each
  uint64_t *state_out;  // where final states go (== state unless banded)
  uint32_t out_mode;    // value emitted per state: 0 the state, 1 xorshift64* (selects the kernel)
};

// Values per thread and row buffers of the bulk-copy row kernel (nb == 0:
// not used).
struct BulkChoice {
  uint32_t vpt = 0;
  uint32_t nb = 0;
};

struct LaunchShape {
  uint32_t vpt;
  uint32_t block;
  uint32_t grid;
  uint32_t width;         // widest store in values (1, 2, 4) the shape may use
  bool staged = false;    // rows off the 128-byte lines: the staged row kernel
  bool bulk_auto = false;  // resolve_shape may pick the bulk-copy kernel for each launch
  BulkChoice bulk_forced;  // store_policy 2: this bulk-copy shape for every device row
  uint32_t sms = 0;        // SMs of the device the shape is for
  uint32_t bulk_nb = 0;    // set by resolve_shape: this launch runs the bulk kernel (vpt values per thread)
};

// What one row-kernel launch ran (rng_launch_info without struct_size).
struct LaunchInfo {
  uint32_t kernel = 0;
  uint32_t vpt = 0, block = 0, grid = 0, row_buffers = 0;
  uint64_t band_rows = 0;
};

// Values-per-thread counts the row kernel is compiled for (256-thread
// blocks), and the (values-per-thread, block) pairs of the other block sizes.
bool rows_vpt_supported(uint32_t vpt);
bool rows_shape_supported(uint32_t vpt, uint32_t block);
// Picks values-per-thread (if vpt == 0), block size, store width (if width ==
// 0) and the grid: one block per tile, or max_grid blocks if set (blocks then
// stride over tiles).  `policy` names the variant that will run.
LaunchShape rows_shape(uint64_t streams, uint32_t vpt, uint32_t block, int device, uint32_t max_grid = 0,
                       uint32_t width = 0, int policy = 1);
// The shape one launch with output a.out runs: the bulk-copy kernel when
// the shape names one for the alignment of a.out's rows (device outputs
// only: the caller passes no host destination here), else `sh` as chosen.
LaunchShape resolve_shape(const LaunchShape &sh, const RowsLaunch &a);
// store_policy: 0 default, 1 streaming (.cs), 2 bulk copies.  Register
// stores are the widest of sh.width and what the output's alignment allows.
// `sh` must come from resolve_shape.  info (optional) receives what ran.
cudaError_t launch_rows(const RowsLaunch &a, const LaunchShape &sh, int store_policy, cudaStream_t st,
                        LaunchInfo *info = nullptr);
cudaError_t launch_init(uint64_t *state, uint64_t n, uint64_t id_base, uint32_t key,
                        cudaStream_t st);
// n words from device memory `src` to page-locked host memory `dst` (a
// device-side address) by SMs, on stream st.
cudaError_t launch_copy(uint64_t *dst, const uint64_t *src, uint64_t n, cudaStream_t st);
// Columns of M^k, where M is the update's matrix over GF(2) (host side).
void jump_matrix(uint64_t k, uint64_t *cols);
// state[s] := the matrix with columns `cols` (64 words) applied to the state
// of stream s (from the hash when from_hash).
cudaError_t launch_jump(uint64_t *state, uint64_t n, uint64_t id_base, uint32_t key, int from_hash,
                        const uint64_t *cols, cudaStream_t st);
// Values per thread of a generate-and-checksum launch over `span` streams
// (vpt = 0: choose; else a power of two up to 64).
uint32_t checksum_vpt(uint64_t span, uint32_t vpt, int device, uint32_t out_mode);
// Generate-and-checksum launch with `vpt` values per thread; a.band_rows != 0
// selects the banded variant (a.jump, a.state_out as for the row kernel).
cudaError_t launch_checksum(const RowsLaunch &a, uint32_t vpt, uint64_t *row_xor, uint64_t *row_sum,
                            cudaStream_t st);
int device_sm_count(int device);

// Work-list kernel tables (batched and served forms).  One entry is a chunk
// of consecutive iterations of one generator instance: rows `rows` of its
// output starting at `out` (row pitch = streams).  Its streams start from the
// id hash (from_hash) or from `state`, and end states are stored back to
// `state` when write_state is set.
struct BatchInstance {
  uint64_t *out;
  uint64_t *state;
  uint64_t streams;
  uint64_t rows;
  uint32_t key;
  uint32_t vec;         // 1: rows are 16-byte aligned (vector stores allowed)
  uint32_t from_hash;
  uint32_t write_state;
};
struct BatchUnit {
  uint32_t inst;
  uint32_t count;   // streams in this unit (<= tile)
  uint64_t s_begin;
};
// Self-contained work unit of the batched form: the instance's fields travel
// with the unit, so a block needs one 64-byte load (no dependent second load)
// before it can start.
struct BatchWork {
  uint64_t *out;      // instance output (row pitch = streams)
  uint64_t streams;
  uint64_t rows;
  uint64_t s_begin;   // first stream of the unit
  uint32_t count;     // streams in the unit (<= one tile)
  uint32_t key;
  uint32_t vec;       // rows 16-byte aligned
  uint32_t pad[5];
};
static_assert(sizeof(BatchWork) == 64, "BatchWork is one 64-byte record");
// Batched-form launch over `n` self-contained units (from the hash; no state):
// one unit per block when counter == nullptr, else persistent blocks taking
// units from the counter.
// bulk_nb > 0: the bulk-copy variant with that many row buffers.
cudaError_t launch_batch_work(const BatchWork *work, uint32_t n, uint32_t *counter, uint32_t vpt, uint32_t grid,
                              cudaStream_t st, uint32_t bulk_nb = 0);
int batch_work_blocks_per_sm(uint32_t vpt, uint32_t bulk_nb = 0);
cudaError_t launch_batch(const BatchInstance *inst, const BatchUnit *units, uint32_t n_units,
                         uint32_t *counter, uint32_t vpt, uint32_t block, uint32_t grid,
                         cudaStream_t st);
int batch_blocks_per_sm(uint32_t vpt, uint32_t block);
// Rows per band when a launch should split its rows across blocks (few
// streams, many rows: too few tiles to fill the GPU); 0 for no split.
// `checksum`: for the generate-and-checksum kernel instead of the row kernel.
uint64_t choose_band_rows(uint64_t streams, uint64_t rows, const LaunchShape &sh, int device,
                          bool checksum = false, uint32_t out = 0);
// Most bands one banded launch is split into (one jump matrix each).
constexpr uint32_t kMaxBands = 1024;
// Host-side GF(2) tables for banded launches: writes `count` matrices
// M^(band * band_rows), band = 0 .. count-1, as 64 column words each.
void jump_table(uint64_t band_rows, uint32_t count, uint64_t *cols);
// Values per thread the work-list kernel is compiled for.
bool batch_vpt_supported(uint32_t vpt);

}  // namespace rngi
