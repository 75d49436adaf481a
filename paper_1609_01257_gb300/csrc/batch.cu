// Batched form: many independent generator instances (each its own stream
// count, iteration count and seed, each starting at iteration 0) produced by
// one kernel launch captured in a CUDA graph.
//
// Work is cut into units of one tile (256 threads x values-per-thread
// streams) of one instance, with all of that instance's iterations; each
// unit is a self-contained 64-byte record.  Units run either one per block
// (the hardware dispatches blocks in table order) or on persistent blocks
// that take them from a device counter.  The autotuner times the graph for
// each values-per-thread and distribution candidate and keeps the fastest;
// every candidate writes the same bytes.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "internal.h"
#include "prng_math.cuh"

struct rng_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<rngi::BatchInstance> inst;
  rngi::BatchWork *d_work = nullptr;
  size_t units_cap = 0;
  uint32_t *d_counter = nullptr;
  uint32_t n_units = 0;
  uint32_t vpt = 0, block = 256, grid = 0;
  bool per_block = false;  // one unit per block (no counter) instead of a persistent grid
  uint32_t bulk_nb = 0;    // > 0: units of 16+ rows written by bulk copies from this many row buffers
  double tuned_ms = 0.0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

const uint32_t kBlock = 256;

void drop_graph(rng_batch *b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Row buffers of the bulk-copy batched kernel for `vpt` values per thread
// when the caller fixes the shape.
uint32_t default_bulk_buffers(uint32_t vpt) { return vpt == 4 ? 8u : vpt == 8 ? 12u : 0u; }

// Builds the unit table for `vpt`, uploads it and captures the graph
// (bulk_nb > 0: the bulk-copy variant).
int prepare(rng_batch *b, uint32_t vpt, bool per_block, uint32_t bulk_nb, rng_err **err) {
  const uint64_t tile = uint64_t(kBlock) * vpt;
  // One tile per unit.  (Grouping the tiles of few-row instances into units
  // of ~1 MiB was measured slower: 6.27 vs 6.61 TB/s on the 512-instance
  // batch -- a unit's tiles run one after another in one block.)  Instances
  // go largest first, each instance's tiles in stream order, so the units
  // running together write neighbouring parts of one output (measured 3 %
  // faster than sorting all units by size, which interleaves instances).
  std::vector<uint32_t> order(b->inst.size());
  for (uint32_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) {
    return b->inst[x].streams * b->inst[x].rows > b->inst[y].streams * b->inst[y].rows;
  });
  std::vector<rngi::BatchWork> units;
  for (uint32_t k : order) {
    const rngi::BatchInstance &in = b->inst[k];
    for (uint64_t s = 0; s < in.streams; s += tile) {
      rngi::BatchWork w{};
      w.out = in.out;
      w.streams = in.streams;
      w.rows = in.rows;
      w.s_begin = s;
      w.count = static_cast<uint32_t>(std::min<uint64_t>(tile, in.streams - s));
      w.key = in.key;
      w.vec = in.vec;
      units.push_back(w);
    }
  }
  if (units.size() > 0xffffffffull) return rngi::fail(err, RNG_EINVAL, "rng_batch: too many work units");
  if (units.size() > b->units_cap) {
    cudaFree(b->d_work);
    b->d_work = nullptr;
    int rc = rngi::cuda_fail(err, cudaMalloc(&b->d_work, units.size() * sizeof(rngi::BatchWork)),
                             "cudaMalloc(batch work table)");
    if (rc) return rc;
    b->units_cap = units.size();
  }
  int rc = rngi::cuda_fail(err,
                           cudaMemcpyAsync(b->d_work, units.data(), units.size() * sizeof(rngi::BatchWork),
                                           cudaMemcpyHostToDevice, b->stream),
                           "cudaMemcpy(batch work table)");
  if (rc) return rc;
  rc = rngi::cuda_fail(err, cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (rc) return rc;
  b->n_units = static_cast<uint32_t>(units.size());
  b->vpt = vpt;
  b->block = kBlock;
  b->bulk_nb = bulk_nb;
  const int per_sm = rngi::batch_work_blocks_per_sm(vpt, bulk_nb);
  const uint64_t resident = uint64_t(rngi::device_sm_count(b->device)) * (per_sm > 0 ? per_sm : 1);
  b->per_block = per_block;
  b->grid = per_block ? b->n_units
                      : static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(resident, b->n_units)));

  drop_graph(b);
  cudaError_t st = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (st == cudaSuccess) {
    cudaError_t s1 = per_block ? cudaSuccess : cudaMemsetAsync(b->d_counter, 0, sizeof(uint32_t), b->stream);
    cudaError_t s2 = rngi::launch_batch_work(b->d_work, b->n_units, per_block ? nullptr : b->d_counter, vpt,
                                             b->grid, b->stream, bulk_nb);
    st = cudaStreamEndCapture(b->stream, &b->graph);
    if (st == cudaSuccess) st = s1 != cudaSuccess ? s1 : s2;
  }
  if (st == cudaSuccess) st = cudaGraphInstantiate(&b->exec, b->graph, 0);
  return rngi::cuda_fail(err, st, "batch graph capture");
}

int replay(rng_batch *b, rng_err **err) {
  cudaError_t st = cudaGraphLaunch(b->exec, b->stream);
  if (st == cudaSuccess) rngi::count_launch();
  return rngi::cuda_fail(err, st, "cudaGraphLaunch");
}

}  // namespace

extern "C" {

void rng_batch_opts_default(rng_batch_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(rng_batch_opts);
  o->values_per_thread = 0;
  o->block_threads = 0;
  o->tune_reps = 3;
  o->stream = nullptr;
  o->device = -1;
  o->mode = 0;
  o->stores = 0;
}

int rng_batch_create(uint32_t count, const uint64_t *streams, const uint64_t *iterations,
                     const uint64_t *seeds, uint64_t *const *outs, const rng_batch_opts *opts,
                     rng_batch **out, rng_err **err) {
  if (!out) return rngi::fail(err, RNG_EINVAL, "rng_batch_create: NULL output pointer");
  *out = nullptr;
  if (count == 0 || !streams || !iterations || !seeds || !outs)
    return rngi::fail(err, RNG_EINVAL, "rng_batch_create: empty batch or NULL array");
  rng_batch_opts o;
  rng_batch_opts_default(&o);
  if (opts) {
    if (opts->struct_size != sizeof(rng_batch_opts))
      return rngi::fail(err, RNG_EINVAL, "rng_batch_create: opts.struct_size mismatch");
    o = *opts;
  }
  const uint32_t v = o.values_per_thread;
  if (v && !rngi::batch_vpt_supported(v))
    return rngi::fail(err, RNG_EINVAL,
                      "rng_batch_create: values_per_thread must be 0 or one of 1, 2, 4, 6, 8, 12, 16, 24, 32");
  if (o.mode > 2) return rngi::fail(err, RNG_EINVAL, "rng_batch_create: mode must be 0, 1 or 2");
  if (o.stores > 2) return rngi::fail(err, RNG_EINVAL, "rng_batch_create: stores must be 0, 1 or 2");
  if (o.stores == 2 && v && !default_bulk_buffers(v))
    return rngi::fail(err, RNG_EINVAL, "rng_batch_create: stores 2 (bulk copies) runs 0, 4 or 8 values per thread");
  if (o.block_threads && o.block_threads != kBlock)
    return rngi::fail(err, RNG_EINVAL, "rng_batch_create: block_threads must be 0 or 256");
  for (uint32_t k = 0; k < count; ++k) {
    if (streams[k] == 0 || streams[k] > (uint64_t(1) << 32) || iterations[k] == 0 || !outs[k])
      return rngi::fail(err, RNG_EINVAL, "rng_batch_create: instance %u has an invalid size or output", k);
    if (iterations[k] > (~uint64_t(0) / 8) / streams[k])
      return rngi::fail(err, RNG_EINVAL, "rng_batch_create: instance %u output size overflows", k);
    if (reinterpret_cast<uintptr_t>(outs[k]) % 8)
      return rngi::fail(err, RNG_EINVAL, "rng_batch_create: instance %u output not 8-byte aligned", k);
  }
  int dev = o.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return rngi::fail(err, RNG_ECUDA, "cudaGetDevice failed");
  cudaError_t st = cudaSetDevice(dev);
  if (st != cudaSuccess) return rngi::cuda_fail(err, st, "cudaSetDevice");

  rng_batch *b = new (std::nothrow) rng_batch();
  if (!b) return rngi::fail(err, RNG_ENOMEM, "rng_batch_create: host allocation failed");
  rngi::live_inc();
  b->device = dev;
  for (uint32_t k = 0; k < count; ++k) {
    rngi::BatchInstance in;
    in.out = outs[k];
    in.state = nullptr;
    in.streams = streams[k];
    in.rows = iterations[k];
    in.key = prng::seed_key(seeds[k]);
    in.vec = (streams[k] % 2 == 0) && (reinterpret_cast<uintptr_t>(outs[k]) % 16 == 0);
    in.from_hash = 1;
    in.write_state = 0;
    b->inst.push_back(in);
  }
  int rc = RNG_OK;
  if (o.stream) {
    b->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    rc = rngi::cuda_fail(err, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    b->own_stream = rc == RNG_OK;
  }
  if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&b->d_counter, sizeof(uint32_t)), "cudaMalloc(batch counter)");
  if (!rc && v) rc = prepare(b, v, o.mode == 1, o.stores == 2 ? default_bulk_buffers(v) : 0u, err);
  if (!rc && !v) {
    // Autotune: time each candidate's graph and keep the fastest.
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = rngi::cuda_fail(err, cudaEventCreate(&e0), "cudaEventCreate");
    if (!rc) rc = rngi::cuda_fail(err, cudaEventCreate(&e1), "cudaEventCreate");
    const uint32_t reps = o.tune_reps ? o.tune_reps : 3;
    uint32_t best_v = 0, best_nb = 0;
    bool best_pb = false;
    double best_ms = 0.0;
    // Register and staged stores at every compiled values-per-thread count,
    // then the bulk-copy variants, each with both work distributions.
    struct Cand {
      uint32_t vpt, nb;
    };
    static const Cand cands[] = {{1, 0}, {2, 0}, {4, 0}, {6, 0}, {8, 0}, {12, 0}, {16, 0}, {24, 0}, {32, 0},
                                 {4, 8}, {8, 6}, {8, 12}};
    const int n_cands = static_cast<int>(sizeof(cands) / sizeof(cands[0]));
    for (int k = 0; k < 2 * n_cands && !rc; ++k) {
      const uint32_t cand = cands[k % n_cands].vpt, nb = cands[k % n_cands].nb;
      const bool pb = k >= n_cands;
      if (o.mode == 1 && !pb) continue;
      if (o.mode == 2 && pb) continue;
      if ((o.stores == 1 && nb) || (o.stores == 2 && !nb)) continue;
      rc = prepare(b, cand, pb, nb, err);
      if (!rc) rc = replay(b, err);  // warm-up
      if (!rc) rc = rngi::cuda_fail(err, cudaEventRecord(e0, b->stream), "cudaEventRecord");
      for (uint32_t r = 0; r < reps && !rc; ++r) rc = replay(b, err);
      if (!rc) rc = rngi::cuda_fail(err, cudaEventRecord(e1, b->stream), "cudaEventRecord");
      if (!rc) rc = rngi::cuda_fail(err, cudaEventSynchronize(e1), "cudaEventSynchronize");
      float ms = 0.f;
      if (!rc) rc = rngi::cuda_fail(err, cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
      if (!rc && (best_v == 0 || ms / reps < best_ms)) {
        best_v = cand;
        best_nb = nb;
        best_pb = pb;
        best_ms = ms / reps;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (!rc) rc = prepare(b, best_v, best_pb, best_nb, err);
    if (!rc) b->tuned_ms = best_ms;
  }
  if (rc) {
    rng_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RNG_OK;
}

int rng_batch_run(rng_batch *b, rng_err **err) {
  if (!b) return rngi::fail(err, RNG_EINVAL, "rng_batch_run: NULL batch");
  if (cudaSetDevice(b->device) != cudaSuccess) return rngi::fail(err, RNG_ECUDA, "rng_batch_run: cudaSetDevice");
  return replay(b, err);
}

int rng_batch_sync(rng_batch *b, rng_err **err) {
  if (!b) return rngi::fail(err, RNG_EINVAL, "rng_batch_sync: NULL batch");
  return rngi::cuda_fail(err, cudaStreamSynchronize(b->stream), "rng_batch_sync");
}

int rng_batch_config(const rng_batch *b, uint32_t *vpt, uint32_t *block, uint32_t *grid, uint64_t *units,
                     uint32_t *mode, double *tuned_ms) {
  if (!b) return RNG_EINVAL;
  if (mode) *mode = b->per_block ? 1u : 2u;
  if (vpt) *vpt = b->vpt;
  if (block) *block = b->block;
  if (grid) *grid = b->grid;
  if (units) *units = b->n_units;
  if (tuned_ms) *tuned_ms = b->tuned_ms;
  return RNG_OK;
}

int rng_batch_stores(const rng_batch *b, uint32_t *stores, uint32_t *row_buffers) {
  if (!b) return RNG_EINVAL;
  if (stores) *stores = b->bulk_nb ? 2u : 1u;
  if (row_buffers) *row_buffers = b->bulk_nb;
  return RNG_OK;
}

void *rng_batch_stream(rng_batch *b) { return b ? static_cast<void *>(b->stream) : nullptr; }

void rng_batch_destroy(rng_batch *b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  drop_graph(b);
  cudaFree(b->d_work);
  cudaFree(b->d_counter);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  rngi::live_dec();
}

}  // extern "C"
