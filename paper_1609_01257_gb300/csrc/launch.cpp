// Host-side launch code of the kernels: shape selection (values per thread,
// store width, grid, bands), the GF(2) jump matrices of rng_skip and of
// banded launches, and the launches themselves.  The kernels are in
// kernels.cu; this file holds no device code.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "prng_math.cuh"

namespace rngi {
namespace {

int occupancy(const void *fn, uint32_t block) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, static_cast<int>(block), 0) !=
          cudaSuccess ||
      n < 1)
    n = 1;
  return n;
}


}  // namespace

int device_sm_count(int device) {
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || sms < 1)
    sms = 1;
  return sms;
}

// Values per thread for 256-thread blocks, from sweeps of the row kernel on
// GB300 (152 SMs) writing 4-32 GiB per launch with one tile per block:
//  - 24 streams per thread (one 48 KiB run per block and row, one resident
//    block per SM) was fastest from 2^22 to 2^26 streams;
//  - from 2^20 up to that, one stream per thread (thousands of short tiles):
//    7.14-7.23 TB/s at 2^20 and 7.33-7.38 at 2^21 on every GPU tried, where
//    shapes of about 128 tiles (fewer blocks than SMs) ran at 7.4 TB/s on some
//    GPUs but 6.1 on others;
//  - below 2^20 about 128 tiles (one long-running block on most SMs) stayed
//    fastest on average: 8 per thread at 2^18 (6.3-7.6 TB/s against 6.5 for
//    one per thread), 2 at 2^16 (6.2-7.4 against 6.5).
uint32_t default_vpt(uint64_t streams, int sms) {
  const uint64_t M = uint64_t(1) << 20;
  if (streams >= 7 * M / 2) return 24;
  if (streams >= M) return 1;
  (void)sms;
  const uint64_t v = streams / (uint64_t(kGenBlock) * 128);
  for (uint32_t c : {32u, 16u, 8u, 4u, 2u})
    if (v >= c) return c;
  return 1;
}

// Values per thread of the staged row kernel for rows that do not start on
// 128-byte lines (a stream count that is not a multiple of 16), or 0 to keep
// the unstaged kernel.  Measured on GB300 (1024 rows, GB/s): 2^22 + 1
// streams 6968 unstaged (24 per thread) vs 6882 staged at best, so from 3.5 M
// streams the unstaged kernel stays; 3,000,017 streams 4411 unstaged vs 6762
// staged at 8 per thread; 1,000,003 streams 4204 vs 6297 at 2; 250,001
// streams 5642 at 4; 65,537 streams 4976 at 8 (banded).
uint32_t staged_vpt(uint64_t streams, uint32_t requested, int sms) {
  if (requested) return requested == 1 || requested == 2 || requested == 4 || requested == 6 || requested == 8
                            ? requested : 0;
  const uint64_t M = uint64_t(1) << 20;
  if (streams >= 7 * M / 2) return 0;
  if (streams >= 2 * M) return 8;
  if (streams >= M / 2) return 2;
  const uint64_t tiles8 = (streams + uint64_t(kGenBlock) * 8 - 1) / (uint64_t(kGenBlock) * 8);
  return tiles8 * 2 < static_cast<uint64_t>(sms) ? 8 : 4;  // 8 when the launch will be banded
}

// Row buffers of the bulk-copy row kernel for `vpt` values per thread (0 if
// that count has no bulk variant).
uint32_t bulk_buffers(uint32_t vpt) {
  switch (vpt) {
    case 4: return 8;
    case 8: return 12;
    case 16: return 4;
    default: return 0;
  }
}

// Bulk-copy row kernel (values per thread, row buffers) for one launch of
// `rows` rows over `streams` streams when the caller leaves the shape to the
// library, for rows on 128-byte lines (`lined`) and off them; nb == 0: keep
// the register or staged kernel.  Measured on GB300 (GB/s; the register-
// store or staged kernel in brackets):
//  - on the lines, 1024 rows: 2^22 streams 7517 at (8, 12) [7470]; below
//    3.5 M streams the register kernels stay ahead (2^20: 7211 [7247]; 2^16:
//    6574 [6858]);
//  - off the lines, 1024 rows, at (8, 12): 2^22 + 1 streams 7125 [6957], an
//    output one word off a line 7147 [6893], 3,000,017 streams 6983 [6713],
//    250,001 7078 [5629], 65,537 (banded) 6343 [4957]; at (16, 4): 1,000,003
//    streams 6769 [6333] (6565 at (8, 12));
//  - off the lines, 16-128 rows: 3,000,017 streams at (8, 12) 6215-7121
//    [6002-7107]; 250,001 streams 2917-6296 [2595-6250]; 65,537 streams
//    (33 tiles of 2048) at (4, 8) 877-2312 [585-1730]; 1,000,003 streams
//    staged stays level or ahead below 128 rows (6248-6494 at 64-96 rows
//    against 6155-6443); at 8 rows every form is within ~10 %.
// Each copy has a fixed cost: 4 KiB copies (two values per thread) stayed
// near 4.2 TB/s, so bulk tiles hold 8 KiB and more.  With one block per SM
// (the buffers take most of its shared memory) each tile's start -- loading
// its states -- is exposed, so lined launches of few rows keep the register
// kernels: 2^22 streams x 128 rows 7221 [7209], 2^24 x 32 rows 6574 [6580],
// 2^26 x 8 rows 4852 [5368], 2^28 x 2 rows 2233 [3503].
BulkChoice bulk_default(uint64_t streams, uint64_t rows, bool lined, uint32_t sms) {
  const uint64_t M = uint64_t(1) << 20;
  if (lined) return streams >= 7 * M / 2 && rows >= 128 ? BulkChoice{8, 12} : BulkChoice{};
  if (streams < 64 * 1024 || rows < 16) return BulkChoice{};
  if (streams >= M / 2 && streams < 2 * M) return rows >= 128 ? BulkChoice{16, 4} : BulkChoice{};
  if (streams < M / 2 && rows < 256) {
    // Unbanded (banding starts at 256 rows): when tiles of 2048 streams
    // would leave most SMs idle, tiles of 1024 give twice as many blocks.
    const uint64_t tiles8 = (streams + uint64_t(kGenBlock) * 8 - 1) / (uint64_t(kGenBlock) * 8);
    if (tiles8 * 2 < sms) return BulkChoice{4, 8};
  }
  return BulkChoice{8, 12};
}

LaunchShape rows_shape(uint64_t streams, uint32_t vpt, uint32_t block, int device, uint32_t max_grid,
                       uint32_t width, int policy) {
  LaunchShape sh;
  sh.block = block ? block : kGenBlock;
  const int sms = device_sm_count(device);
  if (policy == kStoreBulk) {
    // Every row written by bulk copies, whatever its alignment.
    sh.vpt = vpt ? vpt : 8;
    sh.bulk_forced = BulkChoice{sh.vpt, bulk_buffers(sh.vpt)};
    sh.width = 1;
    const uint64_t tiles = (streams + uint64_t(kGenBlock) * sh.vpt - 1) / (uint64_t(kGenBlock) * sh.vpt);
    uint64_t grid = max_grid && max_grid < tiles ? max_grid : tiles;
    if (grid > 0x7fffffffull) grid = 0x7fffffffull;
    sh.grid = sh.bulk_forced.nb && sh.block == kGenBlock ? static_cast<uint32_t>(grid ? grid : 1) : 0;
    return sh;
  }
  sh.bulk_auto = policy == kStoreStreaming && vpt == 0 && sh.block == kGenBlock && max_grid == 0 && width == 0;
  sh.sms = static_cast<uint32_t>(sms);
  if (sh.block == kGenBlock && streams % 16 != 0) {
    const uint32_t v = staged_vpt(streams, vpt, sms);
    if (v) {
      sh.staged = true;
      sh.vpt = v;
      sh.width = 1;
      const uint64_t tiles = (streams + uint64_t(kGenBlock) * v - 1) / (uint64_t(kGenBlock) * v);
      uint64_t grid = max_grid && max_grid < tiles ? max_grid : tiles;
      if (grid > 0x7fffffffull) grid = 0x7fffffffull;
      sh.grid = static_cast<uint32_t>(grid ? grid : 1);
      return sh;
    }
  }
  if (vpt == 0) vpt = sh.block == kGenBlock ? default_vpt(streams, sms) : 8;
  sh.vpt = vpt;
  // One 8-byte store per value measured fastest once a thread holds six or
  // more streams (see the shape sweep in the design notes); below that the
  // widest store the alignment allows.
  sh.width = width ? width : (vpt >= 6 ? 1 : 4);
  // Occupancy of the variant that will run (policy and store width change
  // the register count).
  const void *fn = rows_kernel_fn(vpt, static_cast<int>(sh.width), sh.block == kGenBlock ? policy : kStoreStreaming, sh.block);
  if (!fn) {
    sh.grid = 0;
    return sh;
  }
  const uint64_t tiles = (streams + static_cast<uint64_t>(sh.block) * vpt - 1) /
                         (static_cast<uint64_t>(sh.block) * vpt);
  // One block per tile by default: the hardware hands tiles out in order as
  // blocks finish, which measured ~10% faster than a persistent grid-stride
  // loop (tiles running at the same time stay adjacent in memory).  max_grid
  // asks for fewer blocks; then each block strides over the tiles.
  uint64_t grid = max_grid ? max_grid : tiles;
  if (grid > tiles) grid = tiles;
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  sh.grid = static_cast<uint32_t>(grid ? grid : 1);
  return sh;
}

LaunchShape resolve_shape(const LaunchShape &sh, const RowsLaunch &a) {
  LaunchShape r = sh;
  r.bulk_nb = 0;
  if (!a.out) return r;
  const bool lined = a.pitch % 16 == 0 && reinterpret_cast<uintptr_t>(a.out) % 128 == 0;
  const BulkChoice c = sh.bulk_forced.nb ? sh.bulk_forced
                       : sh.bulk_auto    ? bulk_default(a.s_end - a.s_begin, a.rows, lined, sh.sms)
                                         : BulkChoice{};
  if (!c.nb) return r;
  r.vpt = c.vpt;
  r.bulk_nb = c.nb;
  r.staged = false;
  r.width = 1;
  const uint64_t span = a.s_end - a.s_begin;
  const uint64_t tiles = (span + uint64_t(kGenBlock) * c.vpt - 1) / (uint64_t(kGenBlock) * c.vpt);
  uint64_t grid = tiles;
  if (sh.vpt == c.vpt && sh.grid && sh.grid < tiles) grid = sh.grid;  // a grid the caller asked for
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  r.grid = static_cast<uint32_t>(grid ? grid : 1);
  return r;
}

cudaError_t launch_rows(const RowsLaunch &a, const LaunchShape &sh, int store_policy, cudaStream_t st,
                        LaunchInfo *info) {
  if (a.band_rows && (a.ring_rows || !a.jump || (a.write_state && a.state_out == a.state)))
    return cudaErrorInvalidValue;
  // Widest store the output's alignment allows: every row must start on an
  // 8*W-byte boundary (pitch a multiple of W, base aligned to 8*W bytes).
  int width = 1;
  const uintptr_t base = reinterpret_cast<uintptr_t>(a.out);
  for (int w : {4, 2})
    if (a.out && a.pitch % w == 0 && base % (8 * w) == 0) {
      width = w;
      break;
    }
  if (width > static_cast<int>(sh.width)) width = static_cast<int>(sh.width);
  // Rows that do not start on 128-byte lines (a pitch that is not a multiple
  // of 16 values, or an output off a line): a warp's run of 8-byte stores
  // then touches nine 32-byte sectors instead of eight.  Shapes chosen for
  // such rows (sh.staged), and shapes of 1-8 values per thread whose output
  // starts off a line, run the staged row kernel, which stores line-aligned
  // pieces; the tiles are the same.
  const uint32_t vpt = sh.vpt;
  const bool small_vpt = vpt == 1 || vpt == 2 || vpt == 4 || vpt == 6 || vpt == 8;
  const bool bulk = a.out && sh.bulk_nb;
  const bool staged = !bulk && a.out && !a.ring_rows && sh.block == kGenBlock && small_vpt &&
                      (sh.staged || a.pitch % 16 != 0 || base % 128 != 0);
  const int policy = store_policy == kStoreBulk ? kStoreStreaming : store_policy;
  const void *fn = bulk     ? rows_bulk_kernel_fn(vpt, sh.bulk_nb, a.band_rows != 0, a.out_mode)
                   : staged ? rows_staged_kernel_fn(vpt, a.band_rows != 0, a.out_mode)
                            : rows_kernel_fn(vpt, width, policy, sh.block, a.band_rows != 0, a.out_mode);
  uint64_t grid = sh.grid;
  const uint64_t span = a.s_end - a.s_begin;
  if (!fn) return cudaErrorInvalidValue;
  size_t smem = 0;
  if (bulk) {
    smem = rows_bulk_smem_bytes(vpt, sh.bulk_nb);
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  RowsLaunch args = a;
  void *params[] = {&args};
  if (a.band_rows) {
    // One block per (tile, band) unit, unless the shape asked for fewer.
    const uint64_t tiles = (span + uint64_t(sh.block) * vpt - 1) / (uint64_t(sh.block) * vpt);
    const uint64_t units = tiles * ((a.rows + a.band_rows - 1) / a.band_rows);
    if (grid >= tiles) grid = units < 0x7fffffffull ? units : 0x7fffffffull;
  }
  if (grid > 0x7fffffffull) grid = 0x7fffffffull;
  cudaError_t e = cudaLaunchKernel(fn, dim3(static_cast<unsigned>(grid)), dim3(sh.block), params, smem, st);
  if (e == cudaSuccess) {
    count_launch();
    if (info) {
      info->kernel = bulk ? RNG_KERNEL_BULK : staged ? RNG_KERNEL_STAGED : RNG_KERNEL_REGISTER;
      info->vpt = vpt;
      info->block = sh.block;
      info->grid = static_cast<uint32_t>(grid);
      info->row_buffers = bulk ? sh.bulk_nb : 0;
      info->band_rows = a.band_rows;
    }
  }
  return e;
}

cudaError_t launch_init(uint64_t *state, uint64_t n, uint64_t id_base, uint32_t key,
                        cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t blocks_needed = (n + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(device_sm_count(dev)) * 8;
  const unsigned grid = static_cast<unsigned>(blocks_needed < cap ? blocks_needed : cap);
  void *params[] = {&state, &n, &id_base, &key};
  cudaError_t e = cudaLaunchKernel(init_kernel_fn(), dim3(grid ? grid : 1), dim3(256), params, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

cudaError_t launch_copy(uint64_t *dst, const uint64_t *src, uint64_t n, cudaStream_t st) {
  int dev = 0;
  cudaGetDevice(&dev);
  // One block per SM keeps enough stores in flight for the host link (1, 2,
  // 4, 8 and 16 blocks per SM measured within 5 % of each other) while the
  // generation kernel of the next chunk runs beside them.
  const uint64_t blocks_needed = (n + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(device_sm_count(dev));
  const unsigned grid = static_cast<unsigned>(blocks_needed < cap ? blocks_needed : cap);
  void *params[] = {&dst, &src, &n};
  cudaError_t e = cudaLaunchKernel(copy_kernel_fn(), dim3(grid ? grid : 1), dim3(256), params, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

namespace {

// 64x64 matrices over GF(2) as 64 column words (column j = image of bit j).
struct Gf2 {
  uint64_t col[64];
};

// a * b over GF(2) (apply b first).  Each column of b is multiplied through
// byte tables of a: tab[q][e] = XOR of a's columns 8q+i over the bits i of
// e, each entry one XOR from a smaller one, then 8 lookups per column.
Gf2 gf2_mul(const Gf2 &a, const Gf2 &b) {
  static thread_local uint64_t tab[8][256];
  for (int q = 0; q < 8; ++q) {
    tab[q][0] = 0;
    for (int e = 1; e < 256; ++e) tab[q][e] = tab[q][e & (e - 1)] ^ a.col[8 * q + __builtin_ctz(e)];
  }
  Gf2 r;
  for (int j = 0; j < 64; ++j) {
    uint64_t acc = 0;
    for (int q = 0; q < 8; ++q) acc ^= tab[q][(b.col[j] >> (8 * q)) & 255];
    r.col[j] = acc;
  }
  return r;
}

Gf2 gf2_identity() {
  Gf2 r;
  for (int j = 0; j < 64; ++j) r.col[j] = uint64_t(1) << j;
  return r;
}

// M^(2^i), i = 0 .. 63, for the xorshift update M (columns of M are the
// update of each unit vector), built once by repeated squaring.
const Gf2 *update_powers_of_two() {
  static const std::vector<Gf2> pw = [] {
    std::vector<Gf2> v(64);
    for (int j = 0; j < 64; ++j) v[0].col[j] = prng::xorshift_update(uint64_t(1) << j);
    for (int i = 1; i < 64; ++i) v[i] = gf2_mul(v[i - 1], v[i - 1]);
    return v;
  }();
  return pw.data();
}

// M^k: one product per set bit of k.
Gf2 update_power(uint64_t k) {
  const Gf2 *pw = update_powers_of_two();
  Gf2 result = gf2_identity();
  for (int i = 0; k; ++i, k >>= 1)
    if (k & 1) result = gf2_mul(pw[i], result);
  return result;
}

}  // namespace

void jump_table(uint64_t band_rows, uint32_t count, uint64_t *cols) {
  const Gf2 step = update_power(band_rows);
  Gf2 m = gf2_identity();  // band 0 starts at the launch's first row
  for (uint32_t b = 0; b < count; ++b) {
    for (int j = 0; j < 64; ++j) cols[64 * b + j] = m.col[j];
    m = gf2_mul(step, m);
  }
}

// Row kernel (bound by HBM writes): bands only when the tiles cannot cover
// half the SMs (128 unbanded tiles of 2^16 streams ran at 7.37 TB/s, three
// bands of them at 6.25); then about two (tile, band) units per SM (16 tiles
// of 4096 streams: 19 bands 6.6 TB/s, 10 bands 4.7 TB/s).
// Checksum kernel (bound by integer issue): bands whenever the tiles leave
// resident block slots empty, up to about four units per slot, so that the
// last wave of units is a small part of the launch.
// Bands hold at least 128 rows, which amortises each unit's jump.
uint64_t choose_band_rows(uint64_t streams, uint64_t rows, const LaunchShape &sh, int device, bool checksum,
                          uint32_t out) {
  const uint64_t sms = static_cast<uint64_t>(device_sm_count(device));
  const uint64_t tiles = (streams + uint64_t(sh.block) * sh.vpt - 1) / (uint64_t(sh.block) * sh.vpt);
  const uint64_t min_band = 128;
  const void *fn = checksum     ? checksum_kernel_fn(sh.vpt, true, out)
                   : sh.bulk_nb ? rows_bulk_kernel_fn(sh.vpt, sh.bulk_nb, true, out)
                   : sh.staged  ? rows_staged_kernel_fn(sh.vpt, true, out)
                                : rows_kernel_fn(sh.vpt, 1, kStoreStreaming, sh.block, true, out);
  if (!fn || rows < 2 * min_band) return 0;  // no banded variant of this shape, or too few rows
  uint64_t target;
  if (checksum) {
    const uint64_t slots = sms * static_cast<uint64_t>(std::max(1, occupancy(fn, sh.block)));
    if (tiles >= slots) return 0;
    target = 4 * slots;
  } else {
    if (tiles * 2 >= sms) return 0;
    target = 2 * sms;
  }
  uint64_t bands = (target + tiles - 1) / tiles;
  if (bands > rows / min_band) bands = rows / min_band;
  if (bands > kMaxBands) bands = kMaxBands;
  if (bands < 2) return 0;
  return (rows + bands - 1) / bands;
}

void jump_matrix(uint64_t k, uint64_t *cols) {
  const Gf2 m = update_power(k);
  for (int j = 0; j < 64; ++j) cols[j] = m.col[j];
}

cudaError_t launch_jump(uint64_t *state, uint64_t n, uint64_t id_base, uint32_t key, int from_hash,
                        const uint64_t *cols, cudaStream_t st) {
  Gf2 m;
  for (int j = 0; j < 64; ++j) m.col[j] = cols[j];
  int dev = 0;
  cudaGetDevice(&dev);
  const uint64_t blocks_needed = (n + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(device_sm_count(dev)) * 8;
  const unsigned grid = static_cast<unsigned>(blocks_needed < cap ? blocks_needed : cap);
  void *params[] = {&state, &n, &id_base, &key, &from_hash, &m};
  cudaError_t e = cudaLaunchKernel(jump_kernel_fn(), dim3(grid ? grid : 1), dim3(256), params, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

uint32_t checksum_vpt(uint64_t span, uint32_t vpt, int device, uint32_t out_mode) {
  (void)device;
  if (vpt) return vpt;
  // 16 values per thread amortise the per-row reductions best (2^22 and 2^26
  // streams: 1.72e12 values/s at 16, 1.38e12 at 8); runs with few tiles are
  // banded to fill the GPU (2^18 streams: 1.21e12 banded at 16 vs 0.83e12
  // unbanded at 8).  Up to 2^18 streams (banded launches) 32 are faster
  // still in output mode 0 (2^16 and 2^18 streams: 1.73e12 at 32, 1.64e12 at
  // 16; from 2^20 streams 16 is best: 1.55e12 vs 1.47e12 at 32).  Smaller
  // values only when one tile would be mostly empty.
  if (out_mode == 0 && span <= (uint64_t(1) << 18) && span >= uint64_t(kGenBlock) * 32) return 32;
  for (uint32_t v = 16; v >= 2; v /= 2)
    if (span >= uint64_t(kGenBlock) * v) return v;
  return 1;
}

cudaError_t launch_checksum(const RowsLaunch &a, uint32_t vpt, uint64_t *row_xor, uint64_t *row_sum,
                            cudaStream_t st) {
  const uint64_t span = a.s_end - a.s_begin;
  int dev = 0;
  cudaGetDevice(&dev);
  const int sms = device_sm_count(dev);
  if (a.band_rows && (!a.jump || (a.write_state && a.state_out == a.state))) return cudaErrorInvalidValue;
  const void *fn = checksum_kernel_fn(vpt, a.band_rows != 0, a.out_mode);
  if (!fn) return cudaErrorInvalidValue;
  const uint64_t tiles = (span + uint64_t(kGenBlock) * vpt - 1) / (uint64_t(kGenBlock) * vpt);
  const uint64_t units = a.band_rows ? tiles * ((a.rows + a.band_rows - 1) / a.band_rows) : tiles;
  const uint64_t resident = uint64_t(sms) * occupancy(fn, kGenBlock);
  const unsigned grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min(units, resident)));
  RowsLaunch args = a;
  unsigned long long *rx = reinterpret_cast<unsigned long long *>(row_xor);
  unsigned long long *rs = reinterpret_cast<unsigned long long *>(row_sum);
  void *params[] = {&args, &rx, &rs};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kGenBlock), params, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

bool rows_vpt_supported(uint32_t vpt) { return rows_kernel_fn(vpt, 1, kStoreDefault, kGenBlock) != nullptr; }
bool rows_shape_supported(uint32_t vpt, uint32_t block) {
  return rows_kernel_fn(vpt ? vpt : 8, 1, kStoreStreaming, block ? block : kGenBlock) != nullptr;
}

bool batch_vpt_supported(uint32_t vpt) { return worklist_kernel_fn(vpt) != nullptr; }

int batch_blocks_per_sm(uint32_t vpt, uint32_t block) {
  const void *fn = worklist_kernel_fn(vpt);
  return fn ? occupancy(fn, block) : 0;
}

int batch_work_blocks_per_sm(uint32_t vpt, uint32_t bulk_nb) {
  if (bulk_nb) {
    const void *fn = batch_work_bulk_kernel_fn(vpt, bulk_nb);
    if (!fn) return 0;
    const size_t smem = rows_bulk_smem_bytes(vpt, bulk_nb);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, static_cast<int>(kGenBlock), smem) != cudaSuccess || n < 1)
      n = 1;
    return n;
  }
  const void *fn = batch_work_kernel_fn(vpt);
  return fn ? occupancy(fn, kGenBlock) : 0;
}

cudaError_t launch_batch_work(const BatchWork *work, uint32_t n, uint32_t *counter, uint32_t vpt, uint32_t grid,
                              cudaStream_t st, uint32_t bulk_nb) {
  const void *fn = bulk_nb ? batch_work_bulk_kernel_fn(vpt, bulk_nb) : batch_work_kernel_fn(vpt);
  if (!fn) return cudaErrorInvalidValue;
  size_t smem = 0;
  if (bulk_nb) {
    smem = rows_bulk_smem_bytes(vpt, bulk_nb);
    const cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  void *params[] = {&work, &n, &counter};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(kGenBlock), params, smem, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

cudaError_t launch_batch(const BatchInstance *inst, const BatchUnit *units, uint32_t n_units,
                         uint32_t *counter, uint32_t vpt, uint32_t block, uint32_t grid,
                         cudaStream_t st) {
  const void *fn = worklist_kernel_fn(vpt);
  if (!fn || block != kGenBlock) return cudaErrorInvalidValue;
  void *params[] = {&inst, &units, &n_units, &counter};
  cudaError_t e = cudaLaunchKernel(fn, dim3(grid), dim3(block), params, 0, st);
  if (e == cudaSuccess) count_launch();
  return e;
}

}  // namespace rngi
