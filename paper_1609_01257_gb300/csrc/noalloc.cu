// Batched generation for callers that cannot allocate device memory.
//
// rng_batch_create (batch.cu) allocates its work records, a work counter and
// a CUDA graph with cudaMalloc.  Some callers cannot do that: code inside a
// framework whose memory pool owns the whole device and forbids allocations
// beside it, or latency-bound callers that must not pay for an allocation
// (and the device-wide synchronisation a cudaFree implies) on every call.
// This entry point produces the batched form's output with the served form's
// work-list kernel (worklist_kernel: an instance table, a unit table and a
// work counter), whose scratch -- the counter and the two tables, 48 bytes
// per instance and 16 per unit -- lives in one fixed-size array in device
// global memory declared at file scope below.  Every GPU that loads the
// library holds this array until the process exits.
//
// Host code cannot use the array's name as a device address (it names a
// host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress, once per device, the first time the entry point runs
// with that device current, and cached.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "internal.h"
#include "prng_math.cuh"

namespace {

constexpr uint32_t kVpt = 8;
constexpr uint32_t kBlock = 256;
constexpr uint64_t kTile = uint64_t(kBlock) * kVpt;
constexpr size_t kCounterBytes = 256;
constexpr size_t kInstBytes = size_t(RNG_NOALLOC_MAX_INSTANCES) * sizeof(rngi::BatchInstance);
constexpr size_t kUnitBytes = size_t(RNG_NOALLOC_MAX_UNITS) * sizeof(rngi::BatchUnit);
constexpr size_t kScratchBytes = kCounterBytes + kInstBytes + kUnitBytes;
constexpr int kMaxDevices = 64;

static_assert(sizeof(rngi::BatchInstance) == 48 && sizeof(rngi::BatchUnit) == 16, "table entry sizes");
static_assert(kInstBytes % 256 == 0, "unit table must stay 256-byte aligned");
static_assert(RNG_NOALLOC_SCRATCH_BYTES == kScratchBytes, "header and scratch size disagree");

// Scratch: [work counter | instance table | unit table].
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Host staging for the tables (no host allocation per call either).
rngi::BatchInstance g_host_inst[RNG_NOALLOC_MAX_INSTANCES];
rngi::BatchUnit g_host_units[RNG_NOALLOC_MAX_UNITS];

std::mutex g_mu;  // serialises the host side of calls (staging arrays, address cache)
unsigned char *g_scratch_addr[kMaxDevices];

}  // namespace

extern "C" int rng_batch_generate_noalloc(uint32_t count, const uint64_t *streams,
                                          const uint64_t *iterations, const uint64_t *seeds,
                                          uint64_t *const *outs, void *stream, rng_err **err) {
  if (count == 0 || !streams || !iterations || !seeds || !outs)
    return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: empty batch or NULL array");
  if (count > RNG_NOALLOC_MAX_INSTANCES)
    return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: %u instances, at most %u", count,
                      RNG_NOALLOC_MAX_INSTANCES);
  uint64_t n_units = 0;
  for (uint32_t k = 0; k < count; ++k) {
    if (streams[k] == 0 || streams[k] > (uint64_t(1) << 32) || iterations[k] == 0 || !outs[k])
      return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: instance %u has an invalid size or output", k);
    if (iterations[k] > (~uint64_t(0) / 8) / streams[k])
      return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: instance %u output size overflows", k);
    if (reinterpret_cast<uintptr_t>(outs[k]) % 8)
      return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: instance %u output not 8-byte aligned", k);
    n_units += (streams[k] + kTile - 1) / kTile;
  }
  if (n_units > RNG_NOALLOC_MAX_UNITS)
    return rngi::fail(err, RNG_EINVAL,
                      "rng_batch_generate_noalloc: %llu work units (tiles of %llu streams), at most %u",
                      (unsigned long long)n_units, (unsigned long long)kTile, RNG_NOALLOC_MAX_UNITS);

  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaError_t st = cudaGetDevice(&dev);
  if (st != cudaSuccess) return rngi::cuda_fail(err, st, "rng_batch_generate_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return rngi::fail(err, RNG_EINVAL, "rng_batch_generate_noalloc: device %d out of range", dev);
  if (!g_scratch_addr[dev]) {
    // Set-up for this device (the current one): the array's device address.
    void *p = nullptr;
    st = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (st != cudaSuccess) return rngi::cuda_fail(err, st, "rng_batch_generate_noalloc: cudaGetSymbolAddress");
    g_scratch_addr[dev] = static_cast<unsigned char *>(p);
  }
  unsigned char *base = g_scratch_addr[dev];
  uint32_t *d_counter = reinterpret_cast<uint32_t *>(base);
  rngi::BatchInstance *d_inst = reinterpret_cast<rngi::BatchInstance *>(base + kCounterBytes);
  rngi::BatchUnit *d_units = reinterpret_cast<rngi::BatchUnit *>(base + kCounterBytes + kInstBytes);

  uint32_t u = 0;
  for (uint32_t k = 0; k < count; ++k) {
    rngi::BatchInstance &in = g_host_inst[k];
    in.out = outs[k];
    in.state = nullptr;
    in.streams = streams[k];
    in.rows = iterations[k];
    in.key = prng::seed_key(seeds[k]);
    in.vec = (streams[k] % 2 == 0) && (reinterpret_cast<uintptr_t>(outs[k]) % 16 == 0);
    in.from_hash = 1;
    in.write_state = 0;
    for (uint64_t s = 0; s < streams[k]; s += kTile)
      g_host_units[u++] = {k, static_cast<uint32_t>(std::min(kTile, streams[k] - s)), s};
  }
  // Largest units first; ties in table order (std::sort works in place).
  std::sort(g_host_units, g_host_units + u, [](const rngi::BatchUnit &a, const rngi::BatchUnit &b) {
    const uint64_t wa = uint64_t(a.count) * g_host_inst[a.inst].rows;
    const uint64_t wb = uint64_t(b.count) * g_host_inst[b.inst].rows;
    if (wa != wb) return wa > wb;
    if (a.inst != b.inst) return a.inst < b.inst;
    return a.s_begin < b.s_begin;
  });
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // From pageable memory these copies return once the source has been read,
  // so the staging arrays can be refilled by the next call.
  st = cudaMemcpyAsync(d_inst, g_host_inst, count * sizeof(rngi::BatchInstance), cudaMemcpyHostToDevice, s);
  if (st == cudaSuccess)
    st = cudaMemcpyAsync(d_units, g_host_units, u * sizeof(rngi::BatchUnit), cudaMemcpyHostToDevice, s);
  if (st == cudaSuccess) st = cudaMemsetAsync(d_counter, 0, sizeof(uint32_t), s);  // must start at zero
  if (st != cudaSuccess) return rngi::cuda_fail(err, st, "rng_batch_generate_noalloc: table upload");
  const int per_sm = rngi::batch_blocks_per_sm(kVpt, kBlock);
  const uint64_t resident = uint64_t(rngi::device_sm_count(dev)) * (per_sm > 0 ? per_sm : 1);
  const uint32_t grid = static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(resident, u)));
  st = rngi::launch_batch(d_inst, d_units, u, d_counter, kVpt, kBlock, grid, s);
  return rngi::cuda_fail(err, st, "rng_batch_generate_noalloc: kernel launch");
}
