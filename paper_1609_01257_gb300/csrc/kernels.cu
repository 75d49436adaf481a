// GPU kernels of the massive PRNG (Section 5 of the cf4ocl paper) for sm_103a.
//
// The paper's rng kernel reads a state, applies one xorshift update and
// writes one value per work-item per launch, with the host swapping two
// buffers between launches.  Here one launch covers many iterations: each
// thread keeps its streams' states in registers for the whole launch and
// writes one row (iteration) after another in the iteration-major layout,
// each warp store covering a contiguous run (one 8-byte streaming store per
// value from six streams per thread up, 16- or 32-byte vector stores below).
// Nothing is read per value; the state array is touched once at the start
// and once at the end.
//
// Also here: the generate-and-checksum kernel, the work-list kernels of the
// batched, served and allocation-free forms, the init and jump-ahead kernels,
// and the copy kernel of the double buffer's copy-kernel reads.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "internal.h"
#include "prng_math.cuh"

namespace rngi {
namespace {

constexpr int kPolicyDefault = kStoreDefault;
constexpr int kPolicyStreaming = kStoreStreaming;

template <int POLICY>
__device__ __forceinline__ void store_pair(uint64_t *p, uint64_t a, uint64_t b) {
  if (POLICY == kPolicyStreaming)
    asm volatile("st.global.cs.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
  else
    asm volatile("st.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

template <int POLICY>
__device__ __forceinline__ void store_one(uint64_t *p, uint64_t a) {
  if (POLICY == kPolicyStreaming)
    asm volatile("st.global.cs.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
  else
    asm volatile("st.global.u64 [%0], %1;" ::"l"(p), "l"(a) : "memory");
}

// 32-byte store (256-bit vector stores exist for global memory on sm_100+).
template <int POLICY>
__device__ __forceinline__ void store_quad(uint64_t *p, uint64_t a, uint64_t b, uint64_t c, uint64_t d) {
  if (POLICY == kPolicyStreaming)
    asm volatile("st.global.cs.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
                 : "memory");
  else
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d)
                 : "memory");
}

// W consecutive values with one store (W = 1, 2 or 4; p aligned to 8*W bytes).
template <int W, int POLICY>
__device__ __forceinline__ void store_vec(uint64_t *p, const uint64_t *v) {
  if (W == 4)
    store_quad<POLICY>(p, v[0], v[1], v[2], v[3]);
  else if (W == 2)
    store_pair<POLICY>(p, v[0], v[1]);
  else
    store_one<POLICY>(p, v[0]);
}

// Stream offset (within a tile) of value q of store slot j for thread t:
// slot j of all threads of the block forms one contiguous run of
// blockDim * P values, so every warp-wide store is 32 * 8 * P contiguous bytes.
constexpr int kBlock = static_cast<int>(kGenBlock);

template <int P, int BLOCK>
__device__ __forceinline__ uint64_t slot_offset(int j, int q) {
  return static_cast<uint64_t>(P) * (threadIdx.x + static_cast<uint64_t>(BLOCK) * j) + q;
}

// Emits `rows` rows of one tile, W values per store.  CHECK: some values of
// the tile lie past the end of the stream range and must not be stored.
// ring != 0: rows wrap around a ring of `ring` rows starting at `row`.
// OUT: output mode (the value emitted for each state, prng::emitted).
template <int VPT, int W, int POLICY, bool CHECK, int BLOCK = kBlock, int OUT = 0>
__device__ __forceinline__ void emit_rows(uint64_t (&st)[VPT], uint64_t *row, uint64_t pitch,
                                          uint64_t rows, uint64_t rel0, uint64_t span,
                                          uint64_t ring = 0) {
  constexpr int J = VPT / W;
  uint64_t *const first = row;
  uint64_t in_ring = 0;
  for (uint64_t r = 0; r < rows; ++r) {
#pragma unroll
    for (int j = 0; j < J; ++j) {
      const uint64_t rel = rel0 + slot_offset<W, BLOCK>(j, 0);
      uint64_t v[W];
#pragma unroll
      for (int q = 0; q < W; ++q) v[q] = prng::emitted<OUT>(st[W * j + q]);
      if (!CHECK || rel + W <= span) {
        store_vec<W, POLICY>(row + rel, v);
      } else {
#pragma unroll
        for (int q = 0; q < W; ++q)
          if (rel + q < span) store_one<POLICY>(row + rel + q, v[q]);
      }
    }
#pragma unroll
    for (int v = 0; v < VPT; ++v) st[v] = prng::xorshift_update(st[v]);
    row += pitch;
    if (ring && ++in_ring == ring) {
      row = first;
      in_ring = 0;
    }
  }
}

template <int VPT, int P, int BLOCK = kBlock>
__device__ __forceinline__ void load_tile(uint64_t (&st)[VPT], const RowsLaunch &a, uint64_t rel0,
                                          uint64_t span) {
#pragma unroll
  for (int j = 0; j < VPT / P; ++j)
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const uint64_t rel = rel0 + slot_offset<P, BLOCK>(j, q);
      const uint64_t s = a.s_begin + rel;
      uint64_t v = 0;
      if (rel < span) v = a.from_hash ? prng::initial_state(a.id_base + s, a.key) : a.state[s];
      st[j * P + q] = v;
    }
}

template <int VPT, int P, int BLOCK = kBlock>
__device__ __forceinline__ void store_tile_state(const uint64_t (&st)[VPT], uint64_t *dst, const RowsLaunch &a,
                                                 uint64_t rel0, uint64_t span) {
#pragma unroll
  for (int j = 0; j < VPT / P; ++j)
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const uint64_t rel = rel0 + slot_offset<P, BLOCK>(j, q);
      if (rel < span) dst[a.s_begin + rel] = st[j * P + q];
    }
}

// Rows of one tile whose segments do not start on 128-byte lines (the row
// pitch is not a multiple of 16 values, or the output is not line aligned).
// A warp-wide run of 8-byte stores that starts off a line touches nine
// 32-byte sectors instead of eight, which costs about an eighth of the write
// rate over whole rows.  So each row is staged in shared memory (the
// thread's values at their places in the tile, two buffers used in turn, one
// barrier per row) and stored as 16-byte pieces aligned to the lines, with
// 8-byte stores for the ragged head and tail of the segment.  Values past
// `span` are staged but not stored.  Every thread of the block must call it.
template <int VPT>
__host__ __device__ constexpr int staged_words() {
  return VPT <= 8 ? 2 * kBlock * VPT : 2;  // 2 x tile (up to 32 KiB); larger tiles store directly
}

template <int VPT, int OUT = 0>
__device__ __forceinline__ void emit_rows_staged(uint64_t (&st)[VPT], uint64_t *row, uint64_t pitch,
                                                 uint64_t rows, uint64_t span, uint64_t *buf) {
  constexpr int kTile = kBlock * VPT;
  const int n = span < static_cast<uint64_t>(kTile) ? static_cast<int>(span) : kTile;
  for (uint64_t r = 0; r < rows; ++r) {
    uint64_t *b = buf + (r & 1) * kTile;
#pragma unroll
    for (int j = 0; j < VPT; ++j) b[threadIdx.x + kBlock * j] = prng::emitted<OUT>(st[j]);
#pragma unroll
    for (int v = 0; v < VPT; ++v) st[v] = prng::xorshift_update(st[v]);
    __syncthreads();
    // Values before the segment's first line boundary, then line-aligned pairs.
    const int mis = static_cast<int>((reinterpret_cast<uintptr_t>(row) >> 3) & 15);
    const int h = min(n, (16 - mis) & 15);
    if (static_cast<int>(threadIdx.x) < h) store_one<kPolicyStreaming>(row + threadIdx.x, b[threadIdx.x]);
    const int pairs = (n - h) >> 1;
    for (int c = threadIdx.x; c < pairs; c += kBlock) {
      const int k = h + 2 * c;
      store_pair<kPolicyStreaming>(row + k, b[k], b[k + 1]);
    }
    if (((n - h) & 1) && threadIdx.x == 0) store_one<kPolicyStreaming>(row + n - 1, b[n - 1]);
    row += pitch;
  }
  __syncthreads();  // the buffers are free for the next tile or unit
}

// TMA bulk copies (cp.async.bulk, shared::cta -> global) ---------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Orders this thread's earlier shared-memory writes before later copies of
// the async proxy (the bulk copies read shared memory through it).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// `bytes` (a multiple of 16) from shared `src` to global `dst`, both 16-byte
// aligned, as part of the issuing thread's current bulk group.
__device__ __forceinline__ void bulk_store(uint64_t *dst, const uint64_t *src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Waits until at most N of this thread's committed groups still read shared memory.
template <int N>
__device__ __forceinline__ void bulk_wait_read() {
  asm volatile("cp.async.bulk.wait_group.read %0;" ::"n"(N) : "memory");
}
// Waits until all of this thread's groups are complete (their writes done).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Shared words of the bulk row kernel: NB row buffers of one tile plus two
// words (a row whose segment starts on an odd word is staged one word
// further on, so that its 16-byte-aligned body is 16-byte aligned in shared
// memory too).
template <int VPT, int NB>
__host__ __device__ constexpr int bulk_words() {
  return NB * (kBlock * VPT + 2);
}

// Rows of one tile written by the TMA unit: each row's values go to one of
// NB shared buffers (used in turn: `kb` is the next buffer and `warm` the
// rows this block has staged, up to NB; both continue across the block's
// tiles), one barrier per row, then one thread
// issues a bulk copy of the row segment's 16-byte-aligned body and plain
// 8-byte stores of an odd head or tail.  The SMs' store path then carries
// only shared-memory writes.  A buffer is refilled only after the copy that
// read it NB rows earlier has finished reading.  Values past `span` are
// staged but not copied.  ring != 0: rows wrap around a ring of `ring` rows.
// Every thread of the block must call it; the issuing thread must wait for
// its groups (bulk_wait_all) before the block exits.
template <int VPT, int NB, int OUT = 0>
__device__ __forceinline__ void emit_rows_bulk(uint64_t (&st)[VPT], uint64_t *row, uint64_t pitch, uint64_t rows,
                                               uint64_t span, uint64_t ring, uint64_t *buf, uint32_t &kb,
                                               uint32_t &warm) {
  static_assert(NB >= 2, "NB: at least 2");
  constexpr int kTile = kBlock * VPT;
  constexpr int kBuf = kTile + 2;
  const int n = span < static_cast<uint64_t>(kTile) ? static_cast<int>(span) : kTile;
  uint64_t *const first = row;
  uint64_t in_ring = 0;
  for (uint64_t r = 0; r < rows; ++r) {
    const int p = static_cast<int>((reinterpret_cast<uintptr_t>(row) >> 3) & 1);  // segment starts on an odd word
    uint64_t *b = buf + kb * kBuf;
#pragma unroll
    for (int j = 0; j < VPT; ++j) b[p + threadIdx.x + kBlock * j] = prng::emitted<OUT>(st[j]);
#pragma unroll
    for (int v = 0; v < VPT; ++v) st[v] = prng::xorshift_update(st[v]);
    fence_proxy_async_smem();
    // After this barrier the block fills the next buffer, last read by the
    // copy issued NB - 1 rows before this one: at most NB - 2 later copies
    // may still be reading.
    if (threadIdx.x == 0 && warm + 1 >= NB) bulk_wait_read<NB - 2>();
    __syncthreads();
    if (threadIdx.x == 0) {
      const int body = (n - p) & ~1;
      if (p) store_one<kPolicyStreaming>(row, b[1]);
      if ((n - p) & 1) store_one<kPolicyStreaming>(row + n - 1, b[p + n - 1]);
      if (body > 0) bulk_store(row + p, b + 2 * p, 8u * static_cast<uint32_t>(body));
      bulk_commit();
    }
    kb = kb + 1 == NB ? 0 : kb + 1;
    if (warm < NB) ++warm;
    row += pitch;
    if (ring && ++in_ring == ring) {
      row = first;
      in_ring = 0;
    }
  }
}

// Whether every row of a segment starting at `row0` with pitch `pitch` starts
// on a 128-byte line.
__device__ __forceinline__ bool rows_line_aligned(const uint64_t *row0, uint64_t pitch) {
  return (reinterpret_cast<uintptr_t>(row0) & 127) == 0 && (pitch & 15) == 0;
}

// Nibble tables of a 64x64 matrix over GF(2) given by its columns (col[j] =
// image of bit j): tab[q][e] = XOR of columns 4q+i over the bits i set in the
// 4-bit value e.  The product with a vector is then 16 table reads and XORs
// instead of 64 masked XORs, and each table is 16 words (128 bytes), so a
// warp's reads of one table never conflict on the shared-memory banks.
// Filled by the whole block.
__device__ __forceinline__ void fill_jump_tables(uint64_t (*tab)[16], const uint64_t *__restrict__ cols) {
  for (int idx = threadIdx.x; idx < 16 * 16; idx += blockDim.x) {
    const int q = idx >> 4, e = idx & 15;
    uint64_t acc = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) acc ^= cols[4 * q + i] & (0ull - static_cast<uint64_t>((e >> i) & 1));
    tab[q][e] = acc;
  }
}

__device__ __forceinline__ uint64_t apply_jump_tables(const uint64_t (*tab)[16], uint64_t x) {
  uint64_t acc = 0;
#pragma unroll
  for (int q = 0; q < 16; ++q) acc ^= tab[q][(x >> (4 * q)) & 15];
  return acc;
}

// Advances the states by band * band_rows iterations: one multiplication over
// GF(2) by M^(band * band_rows), whose 64 columns are jump[64 band ..
// 64 band + 63].  Called by every thread of the block (it synchronises the
// block around refilling the shared tables).
template <int VPT>
__device__ __forceinline__ void jump_states(uint64_t (&st)[VPT], const uint64_t *__restrict__ jump,
                                            uint64_t band, uint64_t (*tab)[16]) {
  __syncthreads();  // the previous unit's reads of the tables are done
  fill_jump_tables(tab, jump + 64 * band);
  __syncthreads();
#pragma unroll
  for (int v = 0; v < VPT; ++v) st[v] = apply_jump_tables(tab, st[v]);
}

// Row kernel.  Unbanded (BANDED = false): a work unit is a tile of BLOCK *
// VPT streams with all rows; each thread holds VPT states in registers
// across all rows.  Banded: a unit is (tile, band of band_rows rows); the
// unit jumps its states ahead to the band's first row, and the final states
// (from the last band) go to state_out, which must not alias `state` (other
// bands still read the starting states).  Blocks stride over units when the
// grid is smaller than the unit count.
template <int VPT, int W, int POLICY, int BLOCK, bool BANDED, int OUT = 0>
__global__ void __launch_bounds__(BLOCK) rows_kernel(const RowsLaunch a) {
  const uint64_t span = a.s_end - a.s_begin;
  const uint64_t tile_vals = static_cast<uint64_t>(BLOCK) * VPT;
  const uint64_t n_tiles = (span + tile_vals - 1) / tile_vals;
  if constexpr (!BANDED) {
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const uint64_t rel0 = tile * tile_vals;
      uint64_t st[VPT];
      load_tile<VPT, W, BLOCK>(st, a, rel0, span);
      if (a.out) {
        if (rel0 + tile_vals <= span)
          emit_rows<VPT, W, POLICY, false, BLOCK, OUT>(st, a.out, a.pitch, a.rows, rel0, span, a.ring_rows);
        else
          emit_rows<VPT, W, POLICY, true, BLOCK, OUT>(st, a.out, a.pitch, a.rows, rel0, span, a.ring_rows);
      } else {
        for (uint64_t r = 0; r < a.rows; ++r)
#pragma unroll
          for (int v = 0; v < VPT; ++v) st[v] = prng::xorshift_update(st[v]);
      }
      if (a.write_state) store_tile_state<VPT, W, BLOCK>(st, a.state, a, rel0, span);
    }
  } else {
    __shared__ uint64_t jtab[16][16];
    const uint64_t band_rows = a.band_rows;
    const uint64_t n_bands = (a.rows + band_rows - 1) / band_rows;
    for (uint64_t w = blockIdx.x; w < n_tiles * n_bands; w += gridDim.x) {
      const uint64_t tile = w % n_tiles;
      const uint64_t band = w / n_tiles;
      const uint64_t rel0 = tile * tile_vals;
      uint64_t st[VPT];
      load_tile<VPT, W, BLOCK>(st, a, rel0, span);
      if (band) jump_states<VPT>(st, a.jump, band, jtab);  // band is the same for the whole block
      const uint64_t r0 = band * band_rows;
      const uint64_t rows = a.rows - r0 < band_rows ? a.rows - r0 : band_rows;
      uint64_t *out = a.out + r0 * a.pitch;
      if (rel0 + tile_vals <= span)
        emit_rows<VPT, W, POLICY, false, BLOCK, OUT>(st, out, a.pitch, rows, rel0, span);
      else
        emit_rows<VPT, W, POLICY, true, BLOCK, OUT>(st, out, a.pitch, rows, rel0, span);
      if (a.write_state && band == n_bands - 1) store_tile_state<VPT, W, BLOCK>(st, a.state_out, a, rel0, span);
    }
  }
}

// Row kernel for outputs whose rows do not start on 128-byte lines (a stream
// count that is not a multiple of 16, or an output that does not start on a
// line): the same work units (tiles, or (tile, band) units when banded), one
// thread per stream slot of the tile, each row staged in shared memory and
// stored in line-aligned pieces (emit_rows_staged).
template <int VPT, bool BANDED, int OUT = 0>
__global__ void __launch_bounds__(kBlock) rows_staged_kernel(const RowsLaunch a) {
  __shared__ uint64_t stage[staged_words<VPT>()];
  const uint64_t span = a.s_end - a.s_begin;
  constexpr uint64_t tile_vals = static_cast<uint64_t>(kBlock) * VPT;
  const uint64_t n_tiles = (span + tile_vals - 1) / tile_vals;
  const uint64_t band_rows = BANDED ? a.band_rows : a.rows;
  const uint64_t n_bands = BANDED ? (a.rows + band_rows - 1) / band_rows : 1;
  for (uint64_t w = blockIdx.x; w < n_tiles * n_bands; w += gridDim.x) {
    const uint64_t tile = w % n_tiles;
    const uint64_t band = BANDED ? w / n_tiles : 0;
    const uint64_t rel0 = tile * tile_vals;
    uint64_t st[VPT];
    load_tile<VPT, 1>(st, a, rel0, span);
    if constexpr (BANDED) {
      __shared__ uint64_t jtab[16][16];
      if (band) jump_states<VPT>(st, a.jump, band, jtab);  // band is the same for the whole block
    }
    const uint64_t r0 = band * band_rows;
    const uint64_t rows = BANDED ? (a.rows - r0 < band_rows ? a.rows - r0 : band_rows) : a.rows;
    emit_rows_staged<VPT, OUT>(st, a.out + r0 * a.pitch + rel0, a.pitch, rows, span - rel0, stage);
    if (a.write_state && band == n_bands - 1)
      store_tile_state<VPT, 1>(st, BANDED ? a.state_out : a.state, a, rel0, span);
  }
}

// Row kernel whose rows are written by TMA bulk copies from shared memory
// (emit_rows_bulk): the same work units as rows_staged_kernel, any row
// alignment, and rings when unbanded.  The dynamic shared memory holds the
// NB row buffers (bulk_words<VPT, NB>() words).
template <int VPT, int NB, bool BANDED, int OUT = 0>
__global__ void __launch_bounds__(kBlock) rows_bulk_kernel(const RowsLaunch a) {
  extern __shared__ __align__(128) uint64_t bulk_buf[];
  const uint64_t span = a.s_end - a.s_begin;
  constexpr uint64_t tile_vals = static_cast<uint64_t>(kBlock) * VPT;
  const uint64_t n_tiles = (span + tile_vals - 1) / tile_vals;
  const uint64_t band_rows = BANDED ? a.band_rows : a.rows;
  const uint64_t n_bands = BANDED ? (a.rows + band_rows - 1) / band_rows : 1;
  uint32_t kb = 0, warm = 0;
  for (uint64_t w = blockIdx.x; w < n_tiles * n_bands; w += gridDim.x) {
    const uint64_t tile = w % n_tiles;
    const uint64_t band = BANDED ? w / n_tiles : 0;
    const uint64_t rel0 = tile * tile_vals;
    uint64_t st[VPT];
    load_tile<VPT, 1>(st, a, rel0, span);
    if constexpr (BANDED) {
      __shared__ uint64_t jtab[16][16];
      if (band) jump_states<VPT>(st, a.jump, band, jtab);  // band is the same for the whole block
    }
    const uint64_t r0 = band * band_rows;
    const uint64_t rows = BANDED ? (a.rows - r0 < band_rows ? a.rows - r0 : band_rows) : a.rows;
    emit_rows_bulk<VPT, NB, OUT>(st, a.out + r0 * a.pitch + rel0, a.pitch, rows, span - rel0,
                                 BANDED ? 0 : a.ring_rows, bulk_buf, kb, warm);
    if (a.write_state && band == n_bands - 1)
      store_tile_state<VPT, 1>(st, BANDED ? a.state_out : a.state, a, rel0, span);
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// Separate init kernel (Listing S4): state[s] = initial state of id_base + s.
__global__ void init_kernel(uint64_t *__restrict__ state, uint64_t n, uint64_t id_base,
                            uint32_t key) {
  for (uint64_t s = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    state[s] = prng::initial_state(id_base + s, key);
}

// Jump-ahead: every state is multiplied by a 64x64 matrix over GF(2) given
// by its columns (col[j] = image of bit j), i.e. advanced by the number of
// iterations the matrix stands for.  The update is linear over GF(2), so k
// iterations are the k-th power of its matrix.
struct JumpMatrix {
  uint64_t col[64];
};

// The product goes through the nibble tables above, which each block fills
// from the matrix (a kernel parameter).
__global__ void jump_kernel(uint64_t *__restrict__ state, uint64_t n, uint64_t id_base, uint32_t key,
                            int from_hash, const __grid_constant__ JumpMatrix m) {
  __shared__ uint64_t tab[16][16];
  fill_jump_tables(tab, m.col);
  __syncthreads();
  for (uint64_t s = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x; s < n;
       s += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const uint64_t v = from_hash ? prng::initial_state(id_base + s, key) : state[s];
    state[s] = apply_jump_tables(tab, v);
  }
}

// Device-to-host read of one double-buffer chunk done by SMs instead of the
// copy engine: n words from a device buffer into page-locked host memory
// (addressed from the device), four independent loads in flight per thread,
// streaming stores.
__global__ void copy_kernel(uint64_t *__restrict__ dst, const uint64_t *__restrict__ src, uint64_t n) {
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  uint64_t i = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const uint64_t a = __ldcs(src + i), b = __ldcs(src + i + stride);
    const uint64_t c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
    store_one<kPolicyStreaming>(dst + i, a);
    store_one<kPolicyStreaming>(dst + i + stride, b);
    store_one<kPolicyStreaming>(dst + i + 2 * stride, c);
    store_one<kPolicyStreaming>(dst + i + 3 * stride, d);
  }
  for (; i < n; i += stride) store_one<kPolicyStreaming>(dst + i, __ldcs(src + i));
}

// 64-bit XOR and wrapping sum across a warp with 32-bit reductions: the sum
// is split into two 16-bit low parts (no carry can be lost over 32 lanes)
// and the high word, whose sum only matters modulo 2^32.
__device__ __forceinline__ void warp_xor_sum(uint64_t &x, uint64_t &s) {
  const unsigned full = 0xffffffffu;
  const uint32_t xl = __reduce_xor_sync(full, static_cast<uint32_t>(x));
  const uint32_t xh = __reduce_xor_sync(full, static_cast<uint32_t>(x >> 32));
  const uint32_t lo = static_cast<uint32_t>(s);
  const uint32_t a = __reduce_add_sync(full, lo & 0xffffu);
  const uint32_t b = __reduce_add_sync(full, lo >> 16);
  const uint32_t c = __reduce_add_sync(full, static_cast<uint32_t>(s >> 32));
  x = (static_cast<uint64_t>(xh) << 32) | xl;
  s = static_cast<uint64_t>(a) + (static_cast<uint64_t>(b) << 16) + (static_cast<uint64_t>(c) << 32);
}

// Generate-and-checksum: per row, XOR and sum of all values of the launch's
// stream range, reduced per warp, then per block (double-buffered shared
// slots, one barrier per row), then one atomic pair per block and row.
// Banded (BANDED = true): work units are (tile, band of band_rows rows), each
// unit jumping its states ahead to its band over GF(2) as in the row kernel;
// final states go to state_out (from the last band).
template <int VPT, bool BANDED, int OUT = 0>
__global__ void __launch_bounds__(kBlock) checksum_kernel(const RowsLaunch a,
                                                       unsigned long long *row_xor,
                                                       unsigned long long *row_sum) {
  __shared__ uint64_t sx[2][kBlock / 32], ss[2][kBlock / 32];
  const uint64_t span = a.s_end - a.s_begin;
  const uint64_t tile_vals = static_cast<uint64_t>(kBlock) * VPT;
  const uint64_t n_tiles = (span + tile_vals - 1) / tile_vals;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int n_warps = kBlock / 32;
  const uint64_t band_rows = BANDED ? a.band_rows : (a.rows ? a.rows : 1);
  const uint64_t n_bands = BANDED ? (a.rows + band_rows - 1) / band_rows : 1;
  for (uint64_t w = blockIdx.x; w < n_tiles * n_bands; w += gridDim.x) {
    const uint64_t tile = w % n_tiles;
    const uint64_t band = BANDED ? w / n_tiles : 0;
    const uint64_t rel0 = tile * tile_vals;
    uint64_t st[VPT];
    load_tile<VPT, 1>(st, a, rel0, span);
    if constexpr (BANDED) {
      __shared__ uint64_t jtab[16][16];
      if (band) jump_states<VPT>(st, a.jump, band, jtab);  // band is the same for the whole block
    }
    const uint64_t r0 = band * band_rows;
    const uint64_t rows = BANDED ? (a.rows - r0 < band_rows ? a.rows - r0 : band_rows) : a.rows;
    for (uint64_t r = 0; r < rows; ++r) {
      uint64_t x = 0, s = 0;
#pragma unroll
      for (int v = 0; v < VPT; ++v) {
        const uint64_t e = prng::emitted<OUT>(st[v]);
        x ^= e;
        s += e;
        st[v] = prng::xorshift_update(st[v]);
      }
      warp_xor_sum(x, s);
      const int buf = static_cast<int>(r & 1);
      if (lane == 0) {
        sx[buf][warp] = x;
        ss[buf][warp] = s;
      }
      __syncthreads();
      if (warp == 0) {
        uint64_t bx = lane < n_warps ? sx[buf][lane] : 0;
        uint64_t bs = lane < n_warps ? ss[buf][lane] : 0;
        warp_xor_sum(bx, bs);
        if (lane == 0) {
          atomicXor(row_xor + r0 + r, static_cast<unsigned long long>(bx));
          atomicAdd(row_sum + r0 + r, static_cast<unsigned long long>(bs));
        }
      }
    }
    // Values past the end of the range were loaded as 0 and advance to 0,
    // so they add nothing; the states of real streams are written back.
    if (a.write_state && band == n_bands - 1)
      store_tile_state<VPT, 1>(st, BANDED ? a.state_out : a.state, a, rel0, span);
    __syncthreads();
  }
}

// One work unit of the work-list kernel: `count` streams of one chunk from
// s_begin, all rows of the chunk, processed one tile (kBlock * VPT streams)
// at a time.  Units of instances with few rows span several tiles so that
// units carry similar numbers of bytes.
template <int VPT>
__device__ __forceinline__ void process_unit(const BatchInstance *__restrict__ inst,
                                             const BatchUnit *__restrict__ units, uint32_t u, uint64_t *stage) {
  const BatchUnit wu = units[u];
  const BatchInstance in = inst[wu.inst];
  const uint64_t tile_vals = static_cast<uint64_t>(kBlock) * VPT;
  for (uint64_t off = 0; off < wu.count; off += tile_vals) {
    RowsLaunch a;
    a.state = in.state;
    a.out = in.out;
    a.pitch = in.streams;
    a.s_begin = wu.s_begin + off;
    a.s_end = wu.s_begin + wu.count;
    a.id_base = 0;
    a.rows = in.rows;
    a.key = in.key;
    a.from_hash = in.from_hash;
    a.write_state = in.write_state;
    a.ring_rows = 0;
    const uint64_t span = wu.count - off;
    uint64_t *row = in.out + a.s_begin;
    // Rows off the 128-byte lines: staged through shared memory.  Otherwise
    // 16-byte stores for few values per thread on aligned rows, one
    // streaming 8-byte store per value from six values per thread up.
    if (staged_words<VPT>() > 2 && !rows_line_aligned(row, a.pitch)) {
      uint64_t st[VPT];
      load_tile<VPT, 1>(st, a, 0, span);
      emit_rows_staged<VPT>(st, row, a.pitch, a.rows, span, stage);
      if (a.write_state) store_tile_state<VPT, 1>(st, a.state, a, 0, span);
    } else if (VPT % 2 == 0 && VPT < 6 && in.vec) {
      constexpr int V2 = VPT >= 2 ? VPT : 2;
      uint64_t st[V2];
      load_tile<V2, 2>(st, a, 0, span);
      if (span >= tile_vals)
        emit_rows<V2, 2, kPolicyStreaming, false>(st, row, a.pitch, a.rows, 0, span);
      else
        emit_rows<V2, 2, kPolicyStreaming, true>(st, row, a.pitch, a.rows, 0, span);
      if (a.write_state) store_tile_state<V2, 2>(st, a.state, a, 0, span);
    } else {
      uint64_t st[VPT];
      load_tile<VPT, 1>(st, a, 0, span);
      if (span >= tile_vals)
        emit_rows<VPT, 1, kPolicyStreaming, false>(st, row, a.pitch, a.rows, 0, span);
      else
        emit_rows<VPT, 1, kPolicyStreaming, true>(st, row, a.pitch, a.rows, 0, span);
      if (a.write_state) store_tile_state<VPT, 1>(st, a.state, a, 0, span);
    }
  }
}

// Work-list kernel (batched, served and allocation-free forms).  With a
// counter, a persistent grid of blocks takes units from it; without one
// (counter == nullptr), block b runs unit b and the hardware hands units out
// in table order as blocks finish.  Either way the table lists the largest
// units first.
template <int VPT>
__global__ void __launch_bounds__(kBlock) worklist_kernel(const BatchInstance *__restrict__ inst,
                                                          const BatchUnit *__restrict__ units,
                                                          uint32_t n_units, uint32_t *counter) {
  __shared__ uint64_t stage[staged_words<VPT>()];
  if (counter == nullptr) {
    if (blockIdx.x < n_units) process_unit<VPT>(inst, units, blockIdx.x, stage);
    return;
  }
  __shared__ uint32_t s_unit;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t u = s_unit;
    __syncthreads();
    if (u >= n_units) return;
    process_unit<VPT>(inst, units, u, stage);
  }
}

// Batched form over self-contained units (see BatchWork): every unit starts
// from the id hash and writes all rows of one tile of one instance.
template <int VPT>
__device__ __forceinline__ void process_work(const BatchWork &w, uint64_t *stage) {
  RowsLaunch a;
  a.state = nullptr;
  a.out = w.out;
  a.pitch = w.streams;
  a.s_begin = w.s_begin;
  a.s_end = w.s_begin + w.count;
  a.id_base = 0;
  a.rows = w.rows;
  a.key = w.key;
  a.from_hash = 1;
  a.write_state = 0;
  a.ring_rows = 0;
  const uint64_t span = w.count;
  const uint64_t tile_vals = static_cast<uint64_t>(kBlock) * VPT;
  uint64_t *row = w.out + w.s_begin;
  if (staged_words<VPT>() > 2 && !rows_line_aligned(row, a.pitch)) {
    uint64_t st[VPT];
    load_tile<VPT, 1>(st, a, 0, span);
    emit_rows_staged<VPT>(st, row, a.pitch, a.rows, span, stage);
  } else if (VPT % 2 == 0 && VPT < 6 && w.vec) {
    constexpr int V2 = VPT >= 2 ? VPT : 2;
    uint64_t st[V2];
    load_tile<V2, 2>(st, a, 0, span);
    if (span >= tile_vals)
      emit_rows<V2, 2, kPolicyStreaming, false>(st, row, a.pitch, a.rows, 0, span);
    else
      emit_rows<V2, 2, kPolicyStreaming, true>(st, row, a.pitch, a.rows, 0, span);
  } else {
    uint64_t st[VPT];
    load_tile<VPT, 1>(st, a, 0, span);
    if (span >= tile_vals)
      emit_rows<VPT, 1, kPolicyStreaming, false>(st, row, a.pitch, a.rows, 0, span);
    else
      emit_rows<VPT, 1, kPolicyStreaming, true>(st, row, a.pitch, a.rows, 0, span);
  }
}

template <int VPT>
__global__ void __launch_bounds__(kBlock) batch_work_kernel(const BatchWork *__restrict__ work, uint32_t n,
                                                            uint32_t *counter) {
  __shared__ uint64_t stage[staged_words<VPT>()];
  if (counter == nullptr) {
    if (blockIdx.x < n) {
      const BatchWork w = work[blockIdx.x];
      process_work<VPT>(w, stage);
    }
    return;
  }
  __shared__ uint32_t s_unit;
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
    __syncthreads();
    const uint32_t u = s_unit;
    __syncthreads();
    if (u >= n) return;
    const BatchWork w = work[u];
    process_work<VPT>(w, stage);
  }
}

// Batched form with the bulk-copy row path: units of at least
// kBulkUnitRows rows stage each row in one of NB shared buffers and write it
// with a TMA bulk copy (emit_rows_bulk); shorter units take process_work's
// stores, with the same dynamic shared memory as their staging buffer once
// the earlier units' copies have finished reading it.  Every thread of the
// block calls it.
constexpr uint64_t kBulkUnitRows = 16;

template <int VPT, int NB>
__device__ __forceinline__ void process_work_bulk(const BatchWork &w, uint64_t *buf, uint32_t &kb, uint32_t &warm) {
  if (w.rows < kBulkUnitRows) {
    if (warm) {
      if (threadIdx.x == 0) bulk_wait_read<0>();
      __syncthreads();
      kb = 0;
      warm = 0;
    }
    process_work<VPT>(w, buf);
    return;
  }
  RowsLaunch a;
  a.state = nullptr;
  a.out = w.out;
  a.pitch = w.streams;
  a.s_begin = w.s_begin;
  a.s_end = w.s_begin + w.count;
  a.id_base = 0;
  a.rows = w.rows;
  a.key = w.key;
  a.from_hash = 1;
  a.write_state = 0;
  a.ring_rows = 0;
  uint64_t st[VPT];
  load_tile<VPT, 1>(st, a, 0, w.count);
  emit_rows_bulk<VPT, NB>(st, w.out + w.s_begin, w.streams, w.rows, w.count, 0, buf, kb, warm);
}

template <int VPT, int NB>
__global__ void __launch_bounds__(kBlock) batch_work_bulk_kernel(const BatchWork *__restrict__ work, uint32_t n,
                                                                 uint32_t *counter) {
  extern __shared__ __align__(128) uint64_t bulk_buf[];
  static_assert(bulk_words<VPT, NB>() >= staged_words<VPT>(), "short units stage in the bulk buffers");
  uint32_t kb = 0, warm = 0;
  if (counter == nullptr) {
    if (blockIdx.x < n) {
      const BatchWork w = work[blockIdx.x];
      process_work_bulk<VPT, NB>(w, bulk_buf, kb, warm);
    }
  } else {
    __shared__ uint32_t s_unit;
    for (;;) {
      if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1u);
      __syncthreads();
      const uint32_t u = s_unit;
      __syncthreads();
      if (u >= n) break;
      const BatchWork w = work[u];
      process_work_bulk<VPT, NB>(w, bulk_buf, kb, warm);
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

const void *select_batch_work(uint32_t vpt) {
  switch (vpt) {
    case 1: return reinterpret_cast<const void *>(&batch_work_kernel<1>);
    case 2: return reinterpret_cast<const void *>(&batch_work_kernel<2>);
    case 4: return reinterpret_cast<const void *>(&batch_work_kernel<4>);
    case 6: return reinterpret_cast<const void *>(&batch_work_kernel<6>);
    case 8: return reinterpret_cast<const void *>(&batch_work_kernel<8>);
    case 12: return reinterpret_cast<const void *>(&batch_work_kernel<12>);
    case 16: return reinterpret_cast<const void *>(&batch_work_kernel<16>);
    case 24: return reinterpret_cast<const void *>(&batch_work_kernel<24>);
    case 32: return reinterpret_cast<const void *>(&batch_work_kernel<32>);
    default: return nullptr;
  }
}

template <int VPT, int W>
const void *rows_fn_policy(int policy) {
  return policy == kPolicyStreaming
             ? reinterpret_cast<const void *>(&rows_kernel<VPT, W, kPolicyStreaming, kBlock, false>)
             : reinterpret_cast<const void *>(&rows_kernel<VPT, W, kPolicyDefault, kBlock, false>);
}

// Larger blocks (one store per value, streaming policy): wider contiguous
// runs per block and row with the same registers per thread.
template <int BLOCK>
const void *rows_fn_wide(uint32_t vpt) {
  switch (vpt) {
    case 2: return reinterpret_cast<const void *>(&rows_kernel<2, 1, kPolicyStreaming, BLOCK, false>);
    case 4: return reinterpret_cast<const void *>(&rows_kernel<4, 1, kPolicyStreaming, BLOCK, false>);
    case 6: return reinterpret_cast<const void *>(&rows_kernel<6, 1, kPolicyStreaming, BLOCK, false>);
    case 8: return reinterpret_cast<const void *>(&rows_kernel<8, 1, kPolicyStreaming, BLOCK, false>);
    case 12: return reinterpret_cast<const void *>(&rows_kernel<12, 1, kPolicyStreaming, BLOCK, false>);
    case 16: return reinterpret_cast<const void *>(&rows_kernel<16, 1, kPolicyStreaming, BLOCK, false>);
    case 24: return reinterpret_cast<const void *>(&rows_kernel<24, 1, kPolicyStreaming, BLOCK, false>);
    default: return nullptr;
  }
}

// Widest store width W <= width that divides VPT (W in {1, 2, 4}).
template <int VPT>
const void *rows_fn_dispatch(int width, int policy) {
  if constexpr (VPT % 4 == 0) {
    if (width >= 4) return rows_fn_policy<VPT, 4>(policy);
  }
  if constexpr (VPT % 2 == 0) {
    if (width >= 2) return rows_fn_policy<VPT, 2>(policy);
  }
  return rows_fn_policy<VPT, 1>(policy);
}

#define RNG_FOR_EACH_VPT(X) \
  X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(10) X(12) X(14) X(16) X(18) X(20) X(22) X(24) X(26) X(28) \
  X(32) X(36) X(40) X(48) X(64)

// Banded variants (few streams, many rows): 256-thread blocks, streaming
// stores, the widest store width for the values per thread.
const void *select_rows_banded(uint32_t vpt, int width) {
  switch (vpt) {
    case 1: return reinterpret_cast<const void *>(&rows_kernel<1, 1, kPolicyStreaming, kBlock, true>);
    case 2:
      return width >= 2 ? reinterpret_cast<const void *>(&rows_kernel<2, 2, kPolicyStreaming, kBlock, true>)
                        : reinterpret_cast<const void *>(&rows_kernel<2, 1, kPolicyStreaming, kBlock, true>);
    case 4:
      return width >= 4   ? reinterpret_cast<const void *>(&rows_kernel<4, 4, kPolicyStreaming, kBlock, true>)
             : width >= 2 ? reinterpret_cast<const void *>(&rows_kernel<4, 2, kPolicyStreaming, kBlock, true>)
                          : reinterpret_cast<const void *>(&rows_kernel<4, 1, kPolicyStreaming, kBlock, true>);
    case 8: return reinterpret_cast<const void *>(&rows_kernel<8, 1, kPolicyStreaming, kBlock, true>);
    case 16: return reinterpret_cast<const void *>(&rows_kernel<16, 1, kPolicyStreaming, kBlock, true>);
    default: return nullptr;
  }
}

// Output mode 1 (xorshift64*): 256-thread blocks and streaming stores only;
// 8-byte stores from six values per thread up, as in the default shapes.
template <int VPT, bool BANDED>
const void *rows_star_dispatch(int width) {
  if constexpr (VPT % 4 == 0 && VPT < 6) {
    if (width >= 4) return reinterpret_cast<const void *>(&rows_kernel<VPT, 4, kPolicyStreaming, kBlock, BANDED, 1>);
  }
  if constexpr (VPT % 2 == 0 && VPT < 6) {
    if (width >= 2) return reinterpret_cast<const void *>(&rows_kernel<VPT, 2, kPolicyStreaming, kBlock, BANDED, 1>);
  }
  return reinterpret_cast<const void *>(&rows_kernel<VPT, 1, kPolicyStreaming, kBlock, BANDED, 1>);
}

const void *select_rows_star(uint32_t vpt, int width, bool banded) {
  switch (vpt) {
    case 1: return banded ? rows_star_dispatch<1, true>(width) : rows_star_dispatch<1, false>(width);
    case 2: return banded ? rows_star_dispatch<2, true>(width) : rows_star_dispatch<2, false>(width);
    case 4: return banded ? rows_star_dispatch<4, true>(width) : rows_star_dispatch<4, false>(width);
    case 8: return banded ? rows_star_dispatch<8, true>(width) : rows_star_dispatch<8, false>(width);
    case 16: return banded ? rows_star_dispatch<16, true>(width) : rows_star_dispatch<16, false>(width);
    case 24: return banded ? nullptr : rows_star_dispatch<24, false>(width);
    case 32: return banded ? nullptr : rows_star_dispatch<32, false>(width);
    default: return nullptr;
  }
}

const void *select_rows(uint32_t vpt, int width, int policy, uint32_t block = kBlock) {
  if (block == 512) return rows_fn_wide<512>(vpt);
  if (block == 1024) return rows_fn_wide<1024>(vpt);
  if (block == 128) return rows_fn_wide<128>(vpt);
  if (block != kBlock) return nullptr;
  switch (vpt) {
#define RNG_CASE(V) \
  case V:           \
    return rows_fn_dispatch<V>(width, policy);
    RNG_FOR_EACH_VPT(RNG_CASE)
#undef RNG_CASE
    default:
      return nullptr;
  }
}

template <bool BANDED, int OUT>
const void *select_checksum_t(uint32_t vpt) {
  switch (vpt) {
    case 1: return reinterpret_cast<const void *>(&checksum_kernel<1, BANDED, OUT>);
    case 2: return reinterpret_cast<const void *>(&checksum_kernel<2, BANDED, OUT>);
    case 4: return reinterpret_cast<const void *>(&checksum_kernel<4, BANDED, OUT>);
    case 8: return reinterpret_cast<const void *>(&checksum_kernel<8, BANDED, OUT>);
    case 16: return reinterpret_cast<const void *>(&checksum_kernel<16, BANDED, OUT>);
    case 32: return reinterpret_cast<const void *>(&checksum_kernel<32, BANDED, OUT>);
    case 64: return reinterpret_cast<const void *>(&checksum_kernel<64, BANDED, OUT>);
    default: return nullptr;
  }
}

const void *select_checksum(uint32_t vpt, bool banded, uint32_t out) {
  if (out == 1) return banded ? select_checksum_t<true, 1>(vpt) : select_checksum_t<false, 1>(vpt);
  if (out != 0) return nullptr;
  return banded ? select_checksum_t<true, 0>(vpt) : select_checksum_t<false, 0>(vpt);
}

const void *select_batch(uint32_t vpt) {
  switch (vpt) {
    case 1: return reinterpret_cast<const void *>(&worklist_kernel<1>);
    case 2: return reinterpret_cast<const void *>(&worklist_kernel<2>);
    case 4: return reinterpret_cast<const void *>(&worklist_kernel<4>);
    case 6: return reinterpret_cast<const void *>(&worklist_kernel<6>);
    case 8: return reinterpret_cast<const void *>(&worklist_kernel<8>);
    case 12: return reinterpret_cast<const void *>(&worklist_kernel<12>);
    case 16: return reinterpret_cast<const void *>(&worklist_kernel<16>);
    case 24: return reinterpret_cast<const void *>(&worklist_kernel<24>);
    case 32: return reinterpret_cast<const void *>(&worklist_kernel<32>);
    default: return nullptr;
  }
}

}  // namespace

// Kernel entry points for the host-side launch code (launch.cpp); nullptr
// when a shape is not compiled.
template <bool BANDED, int OUT>
const void *select_rows_staged_t(uint32_t vpt) {
  switch (vpt) {
    case 1: return reinterpret_cast<const void *>(&rows_staged_kernel<1, BANDED, OUT>);
    case 2: return reinterpret_cast<const void *>(&rows_staged_kernel<2, BANDED, OUT>);
    case 4: return reinterpret_cast<const void *>(&rows_staged_kernel<4, BANDED, OUT>);
    case 6: return reinterpret_cast<const void *>(&rows_staged_kernel<6, BANDED, OUT>);
    case 8: return reinterpret_cast<const void *>(&rows_staged_kernel<8, BANDED, OUT>);
    default: return nullptr;
  }
}

template <bool BANDED, int OUT>
const void *select_rows_bulk_t(uint32_t vpt, uint32_t nb) {
  if (vpt == 4 && nb == 8) return reinterpret_cast<const void *>(&rows_bulk_kernel<4, 8, BANDED, OUT>);
  if (vpt == 8 && nb == 12) return reinterpret_cast<const void *>(&rows_bulk_kernel<8, 12, BANDED, OUT>);
  if (vpt == 16 && nb == 4) return reinterpret_cast<const void *>(&rows_bulk_kernel<16, 4, BANDED, OUT>);
  return nullptr;
}

const void *rows_bulk_kernel_fn(uint32_t vpt, uint32_t nb, bool banded, uint32_t out) {
  if (out == 1) return banded ? select_rows_bulk_t<true, 1>(vpt, nb) : select_rows_bulk_t<false, 1>(vpt, nb);
  if (out != 0) return nullptr;
  return banded ? select_rows_bulk_t<true, 0>(vpt, nb) : select_rows_bulk_t<false, 0>(vpt, nb);
}

size_t rows_bulk_smem_bytes(uint32_t vpt, uint32_t nb) {
  return size_t(nb) * (size_t(kBlock) * vpt + 2) * sizeof(uint64_t);
}

const void *rows_kernel_fn(uint32_t vpt, int width, int policy, uint32_t block, bool banded, uint32_t out) {
  if (out == 1) return block == kBlock ? select_rows_star(vpt, width, banded) : nullptr;
  if (out != 0) return nullptr;
  if (banded) return block == kBlock ? select_rows_banded(vpt, width) : nullptr;
  return select_rows(vpt, width, policy, block);
}
const void *rows_staged_kernel_fn(uint32_t vpt, bool banded, uint32_t out) {
  if (out == 1) return banded ? select_rows_staged_t<true, 1>(vpt) : select_rows_staged_t<false, 1>(vpt);
  if (out != 0) return nullptr;
  return banded ? select_rows_staged_t<true, 0>(vpt) : select_rows_staged_t<false, 0>(vpt);
}
const void *checksum_kernel_fn(uint32_t vpt, bool banded, uint32_t out) { return select_checksum(vpt, banded, out); }
const void *worklist_kernel_fn(uint32_t vpt) { return select_batch(vpt); }
const void *batch_work_kernel_fn(uint32_t vpt) { return select_batch_work(vpt); }
const void *batch_work_bulk_kernel_fn(uint32_t vpt, uint32_t nb) {
  if (vpt == 4 && nb == 8) return reinterpret_cast<const void *>(&batch_work_bulk_kernel<4, 8>);
  if (vpt == 8 && nb == 6) return reinterpret_cast<const void *>(&batch_work_bulk_kernel<8, 6>);
  if (vpt == 8 && nb == 12) return reinterpret_cast<const void *>(&batch_work_bulk_kernel<8, 12>);
  return nullptr;
}
const void *init_kernel_fn() { return reinterpret_cast<const void *>(&init_kernel); }
const void *jump_kernel_fn() { return reinterpret_cast<const void *>(&jump_kernel); }
const void *copy_kernel_fn() { return reinterpret_cast<const void *>(&copy_kernel); }

}  // namespace rngi
