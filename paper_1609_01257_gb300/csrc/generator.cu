// Generator object: device state, launch shape, the device-side double
// buffer with its copy stream (Section 5 of the cf4ocl paper: generation into
// one buffer while the other is read to the host), the host consumer, and the
// CUDA-event profiler glue.
//
// The paper orders its two threads with two semaphores: the read of batch k
// must finish before the kernel that overwrites its buffer starts, and the
// kernel producing batch k must finish before its read starts.  Here the
// same two orders are CUDA events between the compute stream and the copy
// stream (`copied[b]` and `produced[b]`), so neither host thread blocks on
// the device between launches.
#include <cuda_runtime.h>
#include <errno.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "prng_math.cuh"

namespace rngi {
rng_prof *prof_create_owned();
void prof_destroy_owned(rng_prof *p);
void prof_clear(rng_prof *p);
void prof_add(rng_prof *p, const char *queue, const char *name, double s, double e);
}  // namespace rngi

namespace {

constexpr const char *kQueueMain = "Main";
constexpr const char *kQueueComms = "Comms";
constexpr size_t kMaxOps = size_t(1) << 20;

struct OpRec {
  const char *name;
  const char *queue;
  size_t ev0, ev1;
};

}  // namespace

struct rng_gen {
  uint64_t n = 0, seed = 0, g0 = 0, pos = 0;
  uint32_t key = 0;
  int device = 0;
  bool initialized = false;   // rng_init called and no failed run since
  bool materialized = false;  // state array holds s_pos (else: hash of the ids)
  rng_opts opts{};
  rngi::LaunchShape shape{};
  rngi::LaunchShape chunk_shape{};  // shape of the last streamed chunk width
  rngi::LaunchInfo last_launch{};   // what the last row-kernel launch ran
  uint64_t chunk_span = 0;
  uint64_t *d_state = nullptr;
  uint64_t *d_state2 = nullptr;      // second state array for banded launches
  uint64_t *d_jump = nullptr;        // GF(2) jump matrices for banded launches
  uint64_t jump_rows = 0;            // band_rows the table on the device is for
  uint32_t jump_count = 0;           // matrices in that table
  cudaStream_t compute = nullptr, copy = nullptr;
  bool own_compute = false;
  uint64_t *d_buf[2] = {nullptr, nullptr};
  size_t buf_bytes = 0;
  std::vector<void *> h_slots;
  std::vector<void *> h_slots_dev;  // the slots' device-side addresses
  std::vector<cudaEvent_t> slot_ready;
  cudaEvent_t produced[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
  // profiling
  std::vector<cudaEvent_t> evpool;
  size_t ev_used = 0;
  std::vector<OpRec> ops;
  cudaEvent_t origin = nullptr;
  std::chrono::steady_clock::time_point wall0;
  rng_prof *prof = nullptr;
  std::string summary;
  rng_host_stats host_stats{};  // of the last call through the staging slots
};

namespace {

cudaError_t next_event(rng_gen *g, size_t *idx) {
  if (g->ev_used == g->evpool.size()) {
    cudaEvent_t e;
    cudaError_t st = cudaEventCreate(&e);
    if (st != cudaSuccess) return st;
    g->evpool.push_back(e);
  }
  *idx = g->ev_used++;
  return cudaSuccess;
}

// Creates the events `ops` more profiled ops will need, so that no event is
// created inside a pipelined loop (creation blocks the enqueuing thread long
// enough to open gaps between copies).
void reserve_events(rng_gen *g, size_t ops) {
  if (!g->opts.profiling) return;
  const size_t room = kMaxOps > g->ops.size() ? kMaxOps - g->ops.size() : 0;
  const size_t want = g->ev_used + 2 * std::min(ops, room);
  while (g->evpool.size() < want) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    g->evpool.push_back(e);
  }
}

// Records the start event of an op on `s`; returns the op slot or -1 when
// profiling is off or the op log is full.
long op_begin(rng_gen *g, const char *name, const char *queue, cudaStream_t s) {
  if (!g->opts.profiling || g->ops.size() >= kMaxOps) return -1;
  size_t e0;
  if (next_event(g, &e0) != cudaSuccess) return -1;
  if (cudaEventRecord(g->evpool[e0], s) != cudaSuccess) return -1;
  g->ops.push_back({name, queue, e0, e0});
  return static_cast<long>(g->ops.size() - 1);
}

void op_end(rng_gen *g, long op, cudaStream_t s) {
  if (op < 0) return;
  size_t e1;
  if (next_event(g, &e1) != cudaSuccess || cudaEventRecord(g->evpool[e1], s) != cudaSuccess) {
    g->ops.pop_back();
    return;
  }
  g->ops[op].ev1 = e1;
}

int profile_restart(rng_gen *g, rng_err **err) {
  g->ops.clear();
  g->ev_used = 0;
  g->wall0 = std::chrono::steady_clock::now();
  if (!g->origin) {
    int rc = rngi::cuda_fail(err, cudaEventCreate(&g->origin), "cudaEventCreate");
    if (rc) return rc;
  }
  return rngi::cuda_fail(err, cudaEventRecord(g->origin, g->compute), "cudaEventRecord");
}

// Prepares a banded launch of `a` with `br` rows per band: the second state
// array (final states go there; the generator switches to it after the
// launch) and the GF(2) jump table on the device.
int setup_bands(rng_gen *g, rngi::RowsLaunch &a, uint64_t br, bool *swap, rng_err **err) {
  const uint64_t bands = (a.rows + br - 1) / br;
  if (bands > rngi::kMaxBands) return rngi::fail(err, RNG_EINVAL, "banded launch: %llu bands", (unsigned long long)bands);
  const uint32_t count = static_cast<uint32_t>(bands);  // one matrix per band
  int rc = RNG_OK;
  if (!g->d_state2)
    rc = rngi::cuda_fail(err, cudaMalloc(&g->d_state2, g->n * 8), "cudaMalloc(second state array)");
  if (!rc && !g->d_jump)
    rc = rngi::cuda_fail(err, cudaMalloc(&g->d_jump, size_t(rngi::kMaxBands) * 64 * 8), "cudaMalloc(jump table)");
  if (rc) return rc;
  if (g->jump_rows != br || g->jump_count < count) {
    std::vector<uint64_t> cols(size_t(count) * 64);
    rngi::jump_table(br, count, cols.data());
    // Pageable source: the call returns once the source has been read.
    rc = rngi::cuda_fail(err, cudaMemcpyAsync(g->d_jump, cols.data(), cols.size() * 8, cudaMemcpyHostToDevice,
                                              g->compute),
                         "jump table upload");
    if (rc) return rc;
    g->jump_rows = br;
    g->jump_count = count;
  }
  a.band_rows = br;
  a.jump = g->d_jump;
  if (a.write_state) {
    a.state_out = g->d_state2;
    *swap = true;
  }
  return RNG_OK;
}

// Launches the row kernel for `a`.  When the launch covers every stream but
// has too few tiles to fill the GPU, its rows are split into bands run by
// separate blocks: each band's blocks jump their states ahead over GF(2),
// and the final states are written to the second state array, which then
// becomes the current one.
// device_out: a.out is device memory (the bulk-copy kernel may write it);
// host destinations keep the register-store kernels.
int gen_launch_rows(rng_gen *g, rngi::RowsLaunch &a, const rngi::LaunchShape &shape, bool device_out,
                    rng_err **err) {
  a.band_rows = 0;
  a.jump = nullptr;
  a.state_out = a.state;
  a.out_mode = g->opts.output_mode;
  rngi::LaunchShape base = shape;
  if (!device_out) {
    base.bulk_auto = false;
    base.bulk_forced = rngi::BulkChoice{};
  }
  const rngi::LaunchShape sh = rngi::resolve_shape(base, a);
  bool swap = false;
  if (!a.ring_rows && a.out && a.s_begin == 0 && a.s_end == g->n) {
    const uint64_t br = rngi::choose_band_rows(g->n, a.rows, sh, g->device, false, a.out_mode);
    if (br) {
      int rc = setup_bands(g, a, br, &swap, err);
      if (rc) return rc;
    }
  }
  long op = op_begin(g, "RNG_KERNEL", kQueueMain, g->compute);
  cudaError_t st = rngi::launch_rows(a, sh, static_cast<int>(g->opts.store_policy), g->compute, &g->last_launch);
  op_end(g, op, g->compute);
  int rc = rngi::cuda_fail(err, st, "rows kernel launch");
  if (!rc && swap) std::swap(g->d_state, g->d_state2);
  return rc;
}

// Device buffers and events of the double buffer; with `slots` > 0, at least
// that many pinned staging slots (grown on demand, kept until rng_destroy).
int ensure_buffers(rng_gen *g, size_t slots, rng_err **err) {
  if (!g->d_buf[0]) {
    for (int b = 0; b < 2; ++b) {
      int rc = rngi::cuda_fail(err, cudaMalloc(&g->d_buf[b], g->buf_bytes), "cudaMalloc(device buffer)");
      if (rc) return rc;
      rc = rngi::cuda_fail(err, cudaEventCreateWithFlags(&g->produced[b], cudaEventDisableTiming),
                           "cudaEventCreate");
      if (rc) return rc;
      rc = rngi::cuda_fail(err, cudaEventCreateWithFlags(&g->copied[b], cudaEventDisableTiming),
                           "cudaEventCreate");
      if (rc) return rc;
    }
  }
  while (g->h_slots.size() < slots) {
    void *p = nullptr;
    int rc = rngi::cuda_fail(err, cudaHostAlloc(&p, g->buf_bytes, cudaHostAllocDefault),
                             "cudaHostAlloc(staging slot)");
    if (rc) return rc;
    cudaEvent_t e;
    rc = rngi::cuda_fail(err, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
    if (rc) {
      cudaFreeHost(p);
      return rc;
    }
    void *pd = nullptr;
    if (cudaHostGetDevicePointer(&pd, p, 0) != cudaSuccess) {
      cudaGetLastError();
      pd = p;  // unified addressing: the host address is valid on the device
    }
    g->h_slots.push_back(p);
    g->h_slots_dev.push_back(pd);
    g->slot_ready.push_back(e);
  }
  return RNG_OK;
}

struct Chunk {
  uint64_t r0, rows;     // iterations relative to the call's first one
  uint64_t s0, span;     // stream range
};

// Splits `T` iterations of `n` streams into chunks that fit one device buffer:
// whole rows when a row fits (as many rows as fit), else one row split into
// column slabs.  Chunks are computed from their index, so a call of any
// length needs no list of them.
struct ChunkPlan {
  uint64_t n = 0, T = 0;
  uint64_t rows_per = 0;  // rows per chunk (whole-row chunks), else 0
  uint64_t slab = 0;      // streams per column slab (one-row chunks)
  uint64_t per_row = 1;   // column slabs per row
  uint64_t count = 0;     // chunks

  ChunkPlan(uint64_t n_, uint64_t T_, size_t buf_bytes) : n(n_), T(T_) {
    const uint64_t cap_vals = buf_bytes / 8;
    if (n <= cap_vals) {
      rows_per = cap_vals / n;
      count = (T + rows_per - 1) / rows_per;
    } else {
      slab = cap_vals & ~uint64_t(1);
      per_row = (n + slab - 1) / slab;
      count = T * per_row;  // <= T * n, which the size check bounds
    }
  }

  Chunk at(uint64_t c) const {
    if (rows_per) {
      const uint64_t r = c * rows_per;
      return {r, (T - r) < rows_per ? (T - r) : rows_per, 0, n};
    }
    const uint64_t s = (c % per_row) * slab;
    return {c / per_row, 1, s, (n - s) < slab ? (n - s) : slab};
  }
};

int launch_chunk(rng_gen *g, const Chunk &c, bool from_hash, uint64_t *dst, rng_err **err) {
  rngi::RowsLaunch a{};
  a.state = g->d_state;
  a.out = dst;
  a.pitch = c.span;
  a.s_begin = c.s0;
  a.s_end = c.s0 + c.span;
  a.id_base = g->g0;
  a.rows = c.rows;
  a.key = g->key;
  a.from_hash = from_hash;
  a.write_state = 1;
  if (c.span != g->chunk_span) {
    // Chunks (which may be stored straight into host memory) run the
    // register-store kernels, in the caller's shape unless that is a
    // bulk-copy shape.
    const bool bulk = g->opts.store_policy == rngi::kStoreBulk;
    g->chunk_shape = rngi::rows_shape(c.span, bulk ? 0 : g->opts.values_per_thread, g->opts.block_threads,
                                      g->device, g->opts.grid_blocks, g->opts.store_width,
                                      bulk ? rngi::kStoreStreaming : static_cast<int>(g->opts.store_policy));
    g->chunk_span = c.span;
  }
  const rngi::LaunchShape sh = g->chunk_shape;
  return gen_launch_rows(g, a, sh, false, err);
}

// What the host consumers do with each finished staging slot.
struct Target {
  uint64_t *out_host = nullptr;  // pageable destination: copy the chunk there
  rng_sink_fn sink = nullptr;    // or hand it to a sink
  void *user = nullptr;
  uint64_t *row_xor = nullptr;   // or fold it into per-row XOR / sum
  uint64_t *row_sum = nullptr;
  unsigned consumers = 1;        // host threads draining the slots
  bool sm_copy = false;          // reads by a copy kernel instead of the copy engine
  bool direct = false;           // the kernel stores each chunk into its staging slot (no device buffer, no copy)
};

// XOR and wrapping sum of `n` values; four independent lanes so that the
// loop is bound by the memory reads, not by one dependency chain.
void xor_sum(const uint64_t *v, uint64_t n, uint64_t *x_out, uint64_t *s_out) {
  uint64_t x0 = 0, x1 = 0, x2 = 0, x3 = 0, s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  uint64_t k = 0;
  for (; k + 4 <= n; k += 4) {
    x0 ^= v[k];
    x1 ^= v[k + 1];
    x2 ^= v[k + 2];
    x3 ^= v[k + 3];
    s0 += v[k];
    s1 += v[k + 1];
    s2 += v[k + 2];
    s3 += v[k + 3];
  }
  for (; k < n; ++k) {
    x0 ^= v[k];
    s0 += v[k];
  }
  *x_out = x0 ^ x1 ^ x2 ^ x3;
  *s_out = s0 + s1 + s2 + s3;
}

// Host consumer threads for staged output (the "out" block of Section 5, with
// the host-side buffering the paper names as an improvement): each takes the
// next finished slot, waits for its copy, copies it to a pageable
// destination, hands it to a sink, or folds it into per-row checksums, and
// frees the slot.  With one thread, chunks are consumed in order.
struct Consumer {
  struct Job {
    Chunk c;
    size_t slot;
    bool stop;
  };
  rng_gen *g;
  Target t;
  uint64_t first_iteration;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Job> jobs;
  std::vector<bool> slot_free;
  int status = RNG_OK;
  std::string msg;
  std::vector<std::thread> th;
  double copy_wait_s = 0.0, consume_s = 0.0;  // summed over threads (under mu)

  int consume(const Job &j, std::string *m, double *wait_s, double *work_s) {
    const auto t0 = std::chrono::steady_clock::now();
    cudaError_t st = cudaEventSynchronize(g->slot_ready[j.slot]);
    const auto t1 = std::chrono::steady_clock::now();
    *wait_s = std::chrono::duration<double>(t1 - t0).count();
    if (st != cudaSuccess) {
      *m = std::string("cudaEventSynchronize: ") + cudaGetErrorString(st);
      return RNG_ECUDA;
    }
    const int rc = consume_ready(j, m);
    *work_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t1).count();
    return rc;
  }

  int consume_ready(const Job &j, std::string *m) {
    const uint64_t *vals = static_cast<const uint64_t *>(g->h_slots[j.slot]);
    if (t.out_host) {
      memcpy(t.out_host + j.c.r0 * g->n + j.c.s0, vals, j.c.rows * j.c.span * 8);
    } else if (t.sink) {
      int urc = t.sink(t.user, first_iteration + j.c.r0, j.c.rows, j.c.s0, j.c.span, j.c.span, vals);
      if (urc) {
        *m = "host consumer returned " + std::to_string(urc);
        return RNG_ESINK;
      }
    } else {
      // Column slabs of one row may be folded by different threads.
      for (uint64_t r = 0; r < j.c.rows; ++r) {
        uint64_t x, s;
        xor_sum(vals + r * j.c.span, j.c.span, &x, &s);
        __atomic_fetch_xor(&t.row_xor[j.c.r0 + r], x, __ATOMIC_RELAXED);
        __atomic_fetch_add(&t.row_sum[j.c.r0 + r], s, __ATOMIC_RELAXED);
      }
    }
    return RNG_OK;
  }

  void run() {
    for (;;) {
      Job j;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [&] { return !jobs.empty(); });
        j = jobs.front();
        jobs.pop_front();
      }
      if (j.stop) return;
      bool skip;
      {
        std::lock_guard<std::mutex> lk(mu);
        skip = status != RNG_OK;
      }
      std::string m;
      double wait_s = 0.0, work_s = 0.0;
      const int rc = skip ? RNG_OK : consume(j, &m, &wait_s, &work_s);
      {
        std::lock_guard<std::mutex> lk(mu);
        copy_wait_s += wait_s;
        consume_s += work_s;
        if (rc != RNG_OK && status == RNG_OK) {
          status = rc;
          msg = m;
        }
        slot_free[j.slot] = true;
      }
      cv.notify_all();
    }
  }
};

// Host consumer threads used when the caller does not choose: every host
// core but one (left to the thread issuing launches and copies), 1 to 16.
// Folding and copying a slot are bound by each core's memory bandwidth
// (about 18-20 GB/s per Grace core), so the link rate needs most cores.
unsigned auto_consumers() {
  const unsigned hw = std::thread::hardware_concurrency();
  return std::max(1u, std::min(16u, hw > 1 ? hw - 1 : 1u));
}

int double_buffer_host(rng_gen *g, uint64_t T, Target tgt, rng_err **err) {
  bool pinned = false;
  uint64_t *out_dev_addr = tgt.out_host;  // the destination as the device addresses it
  if (tgt.out_host) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, tgt.out_host) == cudaSuccess && attr.type == cudaMemoryTypeHost) {
      pinned = true;
      if (attr.devicePointer) out_dev_addr = static_cast<uint64_t *>(attr.devicePointer);
    }
    cudaGetLastError();
  }
  const bool staged = !pinned;
  const ChunkPlan chunks(g->n, T, g->buf_bytes);
  // No more consumers than chunks; two slots beyond the consumers keep the
  // copy engine busy while every consumer holds one.
  tgt.consumers = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(tgt.consumers, chunks.count)));
  size_t slots = 0;
  if (staged) slots = g->opts.host_slots ? std::max<uint32_t>(2, g->opts.host_slots) : tgt.consumers + 2;
  int rc = ensure_buffers(g, slots, err);
  if (rc) return rc;
  if (staged) slots = g->h_slots.size();
  reserve_events(g, 2 * std::min<uint64_t>(chunks.count, kMaxOps));  // one kernel and one read per chunk
  const bool hash_first_rows = !g->materialized;
  const uint64_t first_it = g->pos;
  g->initialized = false;  // re-armed only if the whole run succeeds

  Consumer cons;
  cons.g = g;
  cons.t = tgt;
  cons.first_iteration = first_it;
  if (staged) {
    cons.slot_free.assign(slots, true);
    for (unsigned k = 0; k < tgt.consumers; ++k) {
      try {
        cons.th.emplace_back([&cons] { cons.run(); });
      } catch (...) {
        break;  // run with the threads that could be started
      }
    }
    if (cons.th.empty()) {
      g->initialized = true;  // nothing was launched
      return rngi::fail(err, RNG_ENOMEM, "rng_generate: cannot start a host consumer thread");
    }
  }
  const auto wait_limit = std::chrono::milliseconds(g->opts.host_wait_ms ? g->opts.host_wait_ms : 600000);
  const auto call0 = std::chrono::steady_clock::now();
  double producer_wait_s = 0.0;

  int status = RNG_OK;
  std::string status_msg;
  for (uint64_t c = 0; c < chunks.count && status == RNG_OK; ++c) {
    const Chunk ck = chunks.at(c);
    const int b = static_cast<int>(c & 1);
    size_t slot = 0;
    if (staged) {
      const auto w0 = std::chrono::steady_clock::now();
      std::unique_lock<std::mutex> lk(cons.mu);
      const bool ok = cons.cv.wait_for(lk, wait_limit, [&] {
        return cons.status != RNG_OK ||
               std::find(cons.slot_free.begin(), cons.slot_free.end(), true) != cons.slot_free.end();
      });
      producer_wait_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - w0).count();
      if (cons.status != RNG_OK) break;
      if (!ok) {
        status = RNG_ETIMEOUT;
        status_msg = "no staging slot freed by the host consumer within the wait limit";
        cons.status = RNG_ETIMEOUT;
        break;
      }
      slot = static_cast<size_t>(std::find(cons.slot_free.begin(), cons.slot_free.end(), true) -
                                 cons.slot_free.begin());
      cons.slot_free[slot] = false;
    }
    cudaError_t st = cudaSuccess;
    if (tgt.direct && staged) {
      // The kernel writes the chunk straight into its staging slot over the
      // host link; the slot is ready once the kernel has finished.
      status = launch_chunk(g, ck, hash_first_rows && ck.r0 == 0, static_cast<uint64_t *>(g->h_slots_dev[slot]), err);
      if (status) break;
      st = cudaEventRecord(g->slot_ready[slot], g->compute);
      if (st != cudaSuccess) { status = rngi::cuda_fail(err, st, "event record"); break; }
      {
        std::lock_guard<std::mutex> lk(cons.mu);
        cons.jobs.push_back({ck, slot, false});
      }
      cons.cv.notify_all();
      continue;
    }
    if (c >= 2) st = cudaStreamWaitEvent(g->compute, g->copied[b], 0);
    if (st != cudaSuccess) { status = rngi::cuda_fail(err, st, "cudaStreamWaitEvent"); break; }
    status = launch_chunk(g, ck, hash_first_rows && ck.r0 == 0, g->d_buf[b], err);
    if (status) break;
    st = cudaEventRecord(g->produced[b], g->compute);
    if (st == cudaSuccess) st = cudaStreamWaitEvent(g->copy, g->produced[b], 0);
    if (st != cudaSuccess) { status = rngi::cuda_fail(err, st, "event ordering"); break; }
    long op = op_begin(g, "READ_BUFFER", kQueueComms, g->copy);
    if (tgt.sm_copy) {
      void *dst = staged ? g->h_slots_dev[slot] : static_cast<void *>(out_dev_addr + ck.r0 * g->n + ck.s0);
      st = rngi::launch_copy(static_cast<uint64_t *>(dst), g->d_buf[b], ck.rows * ck.span, g->copy);
    } else {
      void *dst = staged ? g->h_slots[slot] : static_cast<void *>(tgt.out_host + ck.r0 * g->n + ck.s0);
      st = cudaMemcpyAsync(dst, g->d_buf[b], ck.rows * ck.span * 8, cudaMemcpyDeviceToHost, g->copy);
    }
    op_end(g, op, g->copy);
    if (st == cudaSuccess) st = cudaEventRecord(g->copied[b], g->copy);
    if (st == cudaSuccess && staged) st = cudaEventRecord(g->slot_ready[slot], g->copy);
    if (st != cudaSuccess) { status = rngi::cuda_fail(err, st, "device-to-host copy"); break; }
    if (staged) {
      {
        std::lock_guard<std::mutex> lk(cons.mu);
        cons.jobs.push_back({ck, slot, false});
      }
      cons.cv.notify_all();
    }
  }
  if (staged) {
    {
      std::lock_guard<std::mutex> lk(cons.mu);
      for (size_t k = 0; k < cons.th.size(); ++k) cons.jobs.push_back({Chunk{}, 0, true});
    }
    cons.cv.notify_all();
    for (std::thread &th : cons.th) th.join();
    if (status == RNG_OK && cons.status != RNG_OK) {
      status = cons.status;
      status_msg = cons.msg;
    }
  }
  cudaError_t st = cudaStreamSynchronize(g->copy);
  cudaError_t st2 = cudaStreamSynchronize(g->compute);
  rng_host_stats &hs = g->host_stats;
  hs = rng_host_stats{};
  hs.chunks = chunks.count;
  hs.consumers = staged ? static_cast<uint32_t>(cons.th.size()) : 0;
  hs.slots = staged ? static_cast<uint32_t>(slots) : 0;
  hs.wall_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - call0).count();
  hs.producer_wait_s = producer_wait_s;
  hs.copy_wait_s = cons.copy_wait_s;
  hs.consume_s = cons.consume_s;
  if (status == RNG_OK && st != cudaSuccess) status = rngi::cuda_fail(err, st, "cudaStreamSynchronize(copy)");
  if (status == RNG_OK && st2 != cudaSuccess) status = rngi::cuda_fail(err, st2, "cudaStreamSynchronize(compute)");
  if (status != RNG_OK) {
    if (!status_msg.empty()) rngi::fail(err, status, "rng_generate: %s", status_msg.c_str());
    return status;  // streams partly advanced: rng_init required again
  }
  g->materialized = true;
  g->pos += T;
  g->initialized = true;
  return RNG_OK;
}

// Whether kernels on g's device can store into host memory at `p`: page-locked
// (registered) memory always can under unified addressing; pageable memory
// only where the device reads the host's page tables (e.g. Grace over
// NVLink-C2C).  *dev_ptr receives the address to use in kernels.
bool device_can_store(rng_gen *g, uint64_t *p, uint64_t **dev_ptr) {
  cudaPointerAttributes attr;
  cudaError_t st = cudaPointerGetAttributes(&attr, p);
  if (st != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (attr.type == cudaMemoryTypeHost) {
    *dev_ptr = static_cast<uint64_t *>(attr.devicePointer ? attr.devicePointer : p);
    return true;
  }
  if (attr.type == cudaMemoryTypeUnregistered) {
    int pageable = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, g->device) == cudaSuccess &&
        pageable) {
      *dev_ptr = p;
      return true;
    }
  }
  return false;
}

// Direct path: one launch stores all rows into host memory over the link.
int direct_host(rng_gen *g, uint64_t T, uint64_t *dst, rng_err **err) {
  rngi::RowsLaunch a{};
  a.state = g->d_state;
  a.out = dst;
  a.pitch = g->n;
  a.s_begin = 0;
  a.s_end = g->n;
  a.id_base = g->g0;
  a.rows = T;
  a.key = g->key;
  a.from_hash = !g->materialized;
  a.write_state = 1;
  int rc = gen_launch_rows(g, a, g->shape, false, err);
  if (rc) return rc;
  g->materialized = true;
  g->pos += T;
  return rngi::cuda_fail(err, cudaStreamSynchronize(g->compute), "cudaStreamSynchronize(direct to host)");
}

int check_gen(const rng_gen *g, rng_err **err, const char *fn) {
  if (!g) return rngi::fail(err, RNG_EINVAL, "%s: NULL generator", fn);
  if (cudaSetDevice(g->device) != cudaSuccess)
    return rngi::fail(err, RNG_ECUDA, "%s: cannot select device %d", fn, g->device);
  return RNG_OK;
}

int size_ok(uint64_t n, uint64_t T, rng_err **err) {
  if (T > (~uint64_t(0) / 8) / n) return rngi::fail(err, RNG_EINVAL, "output size 8*%llu*%llu overflows",
                                                    (unsigned long long)n, (unsigned long long)T);
  return RNG_OK;
}

}  // namespace

extern "C" {

void rng_opts_default(rng_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(rng_opts);
  o->values_per_thread = 0;
  o->block_threads = 0;
  o->fuse_init = 1;
  o->stream_offset = 0;
  o->device_buffer_bytes = size_t(32) << 20;
  o->host_slots = 0;
  o->profiling = 1;
  o->compute_stream = nullptr;
  o->device = -1;
  o->store_policy = 1;
  o->host_wait_ms = 0;
}

int rng_create(uint64_t streams, uint64_t seed, const rng_opts *opts, rng_gen **out, rng_err **err) {
  if (!out) return rngi::fail(err, RNG_EINVAL, "rng_create: NULL output pointer");
  *out = nullptr;
  if (streams == 0 || streams > (uint64_t(1) << 32))
    return rngi::fail(err, RNG_EINVAL, "rng_create: streams must be in [1, 2^32], got %llu",
                      (unsigned long long)streams);
  rng_opts o;
  rng_opts_default(&o);
  if (opts) {
    if (opts->struct_size != sizeof(rng_opts))
      return rngi::fail(err, RNG_EINVAL, "rng_create: opts.struct_size %u != %zu", opts->struct_size,
                        sizeof(rng_opts));
    o = *opts;
  }
  if (o.values_per_thread && !rngi::rows_vpt_supported(o.values_per_thread))
    return rngi::fail(err, RNG_EINVAL,
                      "rng_create: values_per_thread must be 0 or one of 1-8, 10, 12, 14, 16, 20, 24, 28, 32, 48, 64");
  if (o.block_threads && !rngi::rows_shape_supported(o.values_per_thread, o.block_threads))
    return rngi::fail(err, RNG_EINVAL,
                      "rng_create: block_threads must be 0 or 256, or 128/512/1024 with values_per_thread "
                      "2, 4, 6, 8, 12, 16 or 24");
  if (o.device_buffer_bytes == 0) o.device_buffer_bytes = size_t(32) << 20;
  if (o.device_buffer_bytes < 16 || o.device_buffer_bytes % 16)
    return rngi::fail(err, RNG_EINVAL, "rng_create: device_buffer_bytes must be a positive multiple of 16");
  if (o.store_policy > 2) return rngi::fail(err, RNG_EINVAL, "rng_create: store_policy must be 0, 1 or 2");
  if (o.store_policy == 2 && ((o.block_threads && o.block_threads != rngi::kGenBlock) ||
                              !(o.values_per_thread == 0 || o.values_per_thread == 4 ||
                                o.values_per_thread == 8 || o.values_per_thread == 16)))
    return rngi::fail(err, RNG_EINVAL,
                      "rng_create: store_policy 2 (bulk copies) runs 256-thread blocks with 0, 4, 8 or 16 "
                      "values per thread");
  if (o.host_path > 3) return rngi::fail(err, RNG_EINVAL, "rng_create: host_path must be 0, 1, 2 or 3");
  if (o.host_consumers > 64) return rngi::fail(err, RNG_EINVAL, "rng_create: host_consumers must be at most 64");
  if (o.output_mode > 1) return rngi::fail(err, RNG_EINVAL, "rng_create: output_mode must be 0 or 1");
  if (o.output_mode == 1) {
    const uint32_t v = o.values_per_thread;
    if ((o.block_threads && o.block_threads != rngi::kGenBlock) ||
        !(v == 0 || v == 1 || v == 2 || v == 4 || v == 8 || v == 16 || v == 24 || v == 32))
      return rngi::fail(err, RNG_EINVAL,
                        "rng_create: output_mode 1 runs 256-thread blocks with 0, 1, 2, 4, 8, 16, 24 or 32 "
                        "values per thread");
  }
  if (o.store_width != 0 && o.store_width != 1 && o.store_width != 2 && o.store_width != 4)
    return rngi::fail(err, RNG_EINVAL, "rng_create: store_width must be 0, 1, 2 or 4");
  if (o.stream_offset > (uint64_t(1) << 32) - streams)
    return rngi::fail(err, RNG_EINVAL, "rng_create: stream_offset + streams must not exceed 2^32");

  int dev = o.device;
  if (dev < 0) {
    cudaError_t st = cudaGetDevice(&dev);
    if (st != cudaSuccess) return rngi::cuda_fail(err, st, "cudaGetDevice");
  }
  cudaError_t st = cudaSetDevice(dev);
  if (st != cudaSuccess) return rngi::cuda_fail(err, st, "cudaSetDevice");

  rng_gen *g = new (std::nothrow) rng_gen();
  if (!g) return rngi::fail(err, RNG_ENOMEM, "rng_create: host allocation failed");
  g->n = streams;
  g->seed = seed;
  g->g0 = o.stream_offset;
  g->key = prng::seed_key(seed);
  g->device = dev;
  g->opts = o;
  g->buf_bytes = o.device_buffer_bytes;
  g->shape = rngi::rows_shape(streams, o.values_per_thread, o.block_threads, dev, o.grid_blocks, o.store_width,
                              static_cast<int>(o.store_policy));
  rngi::live_inc();
  int rc = RNG_OK;
  if (o.compute_stream) {
    g->compute = static_cast<cudaStream_t>(o.compute_stream);
  } else {
    rc = rngi::cuda_fail(err, cudaStreamCreateWithFlags(&g->compute, cudaStreamNonBlocking), "cudaStreamCreate");
    g->own_compute = rc == RNG_OK;
  }
  if (!rc) rc = rngi::cuda_fail(err, cudaStreamCreateWithFlags(&g->copy, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&g->d_state, streams * 8), "cudaMalloc(state)");
  if (!rc) rc = profile_restart(g, err);
  if (!rc) g->prof = rngi::prof_create_owned();
  if (!rc && !g->prof) rc = rngi::fail(err, RNG_ENOMEM, "rng_create: profiler allocation failed");
  if (rc) {
    rng_destroy(g);
    return rc;
  }
  *out = g;
  return RNG_OK;
}

void rng_destroy(rng_gen *g) {
  if (!g) return;
  cudaSetDevice(g->device);
  if (g->compute) cudaStreamSynchronize(g->compute);
  if (g->copy) cudaStreamSynchronize(g->copy);
  cudaFree(g->d_state);
  cudaFree(g->d_state2);
  cudaFree(g->d_jump);
  for (int b = 0; b < 2; ++b) {
    cudaFree(g->d_buf[b]);
    if (g->produced[b]) cudaEventDestroy(g->produced[b]);
    if (g->copied[b]) cudaEventDestroy(g->copied[b]);
  }
  for (void *p : g->h_slots) cudaFreeHost(p);
  for (cudaEvent_t e : g->slot_ready) cudaEventDestroy(e);
  for (cudaEvent_t e : g->evpool) cudaEventDestroy(e);
  if (g->origin) cudaEventDestroy(g->origin);
  if (g->copy) cudaStreamDestroy(g->copy);
  if (g->own_compute && g->compute) cudaStreamDestroy(g->compute);
  rngi::prof_destroy_owned(g->prof);
  delete g;
  rngi::live_dec();
}

int rng_init(rng_gen *g, rng_err **err) {
  int rc = check_gen(g, err, "rng_init");
  if (rc) return rc;
  g->pos = 0;
  g->materialized = false;
  if (!g->opts.fuse_init) {
    long op = op_begin(g, "INIT_KERNEL", kQueueMain, g->compute);
    cudaError_t st = rngi::launch_init(g->d_state, g->n, g->g0, g->key, g->compute);
    op_end(g, op, g->compute);
    rc = rngi::cuda_fail(err, st, "init kernel launch");
    if (rc) return rc;
    g->materialized = true;
  }
  g->initialized = true;
  return RNG_OK;
}

int rng_generate(rng_gen *g, uint64_t iterations, uint64_t *out_dev, uint64_t *out_host, rng_err **err) {
  int rc = check_gen(g, err, "rng_generate");
  if (rc) return rc;
  if ((out_dev == nullptr) == (out_host == nullptr))
    return rngi::fail(err, RNG_EINVAL, "rng_generate: exactly one of out_dev and out_host must be set");
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_generate: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, iterations, err);
  if (rc) return rc;
  if (out_host) {
    uint64_t *dptr = nullptr;
    const bool can = (g->opts.host_path == 0 || g->opts.host_path == 2) && device_can_store(g, out_host, &dptr);
    if (g->opts.host_path == 2 && !can)
      return rngi::fail(err, RNG_EINVAL, "rng_generate: the GPU cannot store into this host memory (host_path = 2)");
    if (can) return direct_host(g, iterations, dptr, err);
    Target tgt;
    tgt.out_host = out_host;
    tgt.consumers = g->opts.host_consumers ? g->opts.host_consumers : auto_consumers();
    tgt.sm_copy = g->opts.host_path == 3;
    return double_buffer_host(g, iterations, tgt, err);
  }
  if (reinterpret_cast<uintptr_t>(out_dev) % 8)
    return rngi::fail(err, RNG_EINVAL, "rng_generate: out_dev must be 8-byte aligned");
  rngi::RowsLaunch a{};
  a.state = g->d_state;
  a.out = out_dev;
  a.pitch = g->n;
  a.s_begin = 0;
  a.s_end = g->n;
  a.id_base = g->g0;
  a.rows = iterations;
  a.key = g->key;
  a.from_hash = !g->materialized;
  a.write_state = 1;
  rc = gen_launch_rows(g, a, g->shape, true, err);
  if (rc) return rc;
  g->materialized = true;
  g->pos += iterations;
  return RNG_OK;
}

int rng_generate_ring(rng_gen *g, uint64_t iterations, uint64_t *ring_dev, uint64_t ring_rows, rng_err **err) {
  int rc = check_gen(g, err, "rng_generate_ring");
  if (rc) return rc;
  if (!ring_dev || ring_rows == 0) return rngi::fail(err, RNG_EINVAL, "rng_generate_ring: NULL ring or zero rows");
  if (reinterpret_cast<uintptr_t>(ring_dev) % 8)
    return rngi::fail(err, RNG_EINVAL, "rng_generate_ring: ring must be 8-byte aligned");
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_generate_ring: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, ring_rows, err);
  if (rc) return rc;
  rngi::RowsLaunch a{};
  a.state = g->d_state;
  a.out = ring_dev;
  a.pitch = g->n;
  a.s_begin = 0;
  a.s_end = g->n;
  a.id_base = g->g0;
  a.rows = iterations;
  a.key = g->key;
  a.from_hash = !g->materialized;
  a.write_state = 1;
  a.ring_rows = ring_rows;
  rc = gen_launch_rows(g, a, g->shape, true, err);
  if (rc) return rc;
  g->materialized = true;
  g->pos += iterations;
  return RNG_OK;
}

int rng_generate_sink(rng_gen *g, uint64_t iterations, rng_sink_fn sink, void *user, rng_err **err) {
  int rc = check_gen(g, err, "rng_generate_sink");
  if (rc) return rc;
  if (!sink) return rngi::fail(err, RNG_EINVAL, "rng_generate_sink: NULL sink");
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_generate_sink: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, iterations, err);
  if (rc) return rc;
  Target tgt;
  tgt.sink = sink;
  tgt.user = user;
  tgt.consumers = g->opts.host_consumers ? g->opts.host_consumers : 1;
  tgt.sm_copy = g->opts.host_path == 3;
  tgt.direct = g->opts.host_path == 2;
  return double_buffer_host(g, iterations, tgt, err);
}

// Sink of rng_generate_fd: writes each chunk's bytes to the descriptor,
// retrying short writes and interrupted calls.
static int fd_sink(void *user, uint64_t, uint64_t rows, uint64_t, uint64_t n_streams, uint64_t,
                   const uint64_t *values) {
  const int fd = *static_cast<const int *>(user);
  const char *p = reinterpret_cast<const char *>(values);
  size_t left = rows * n_streams * 8;
  while (left) {
    const ssize_t w = write(fd, p, left);
    if (w < 0) {
      if (errno == EINTR) continue;
      return errno ? errno : 1;
    }
    p += w;
    left -= static_cast<size_t>(w);
  }
  return 0;
}

int rng_generate_fd(rng_gen *g, uint64_t iterations, int fd, rng_err **err) {
  int rc = check_gen(g, err, "rng_generate_fd");
  if (rc) return rc;
  if (fd < 0) return rngi::fail(err, RNG_EINVAL, "rng_generate_fd: bad file descriptor %d", fd);
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_generate_fd: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, iterations, err);
  if (rc) return rc;
  int user = fd;
  Target tgt;
  tgt.sink = fd_sink;
  tgt.user = &user;
  tgt.consumers = 1;  // the bytes must reach the descriptor in order
  tgt.sm_copy = g->opts.host_path == 3;
  tgt.direct = g->opts.host_path == 2;
  return double_buffer_host(g, iterations, tgt, err);
}

int rng_generate_host_checksum(rng_gen *g, uint64_t iterations, uint64_t *row_xor_host, uint64_t *row_sum_host,
                               rng_err **err) {
  int rc = check_gen(g, err, "rng_generate_host_checksum");
  if (rc) return rc;
  if (!row_xor_host || !row_sum_host)
    return rngi::fail(err, RNG_EINVAL, "rng_generate_host_checksum: NULL output");
  if (!g->initialized)
    return rngi::fail(err, RNG_ESTATE, "rng_generate_host_checksum: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, iterations, err);
  if (rc) return rc;
  memset(row_xor_host, 0, iterations * 8);
  memset(row_sum_host, 0, iterations * 8);
  Target tgt;
  tgt.row_xor = row_xor_host;
  tgt.row_sum = row_sum_host;
  tgt.consumers = g->opts.host_consumers ? g->opts.host_consumers : auto_consumers();
  tgt.sm_copy = g->opts.host_path == 3;
  tgt.direct = g->opts.host_path == 2;
  return double_buffer_host(g, iterations, tgt, err);
}

int rng_generate_checksum(rng_gen *g, uint64_t iterations, uint64_t *row_xor_dev, uint64_t *row_sum_dev,
                          rng_err **err) {
  int rc = check_gen(g, err, "rng_generate_checksum");
  if (rc) return rc;
  if (!row_xor_dev || !row_sum_dev) return rngi::fail(err, RNG_EINVAL, "rng_generate_checksum: NULL output");
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_generate_checksum: generator not initialised");
  if (iterations == 0) return RNG_OK;
  rc = size_ok(g->n, iterations, err);
  if (rc) return rc;
  cudaError_t st = cudaMemsetAsync(row_xor_dev, 0, iterations * 8, g->compute);
  if (st == cudaSuccess) st = cudaMemsetAsync(row_sum_dev, 0, iterations * 8, g->compute);
  rc = rngi::cuda_fail(err, st, "cudaMemsetAsync(checksums)");
  if (rc) return rc;
  rngi::RowsLaunch a{};
  a.state = g->d_state;
  a.out = nullptr;
  a.pitch = 0;
  a.s_begin = 0;
  a.s_end = g->n;
  a.id_base = g->g0;
  a.rows = iterations;
  a.key = g->key;
  a.from_hash = !g->materialized;
  a.write_state = 1;
  a.state_out = a.state;
  const uint32_t v = g->opts.values_per_thread;
  const uint32_t vpt = rngi::checksum_vpt(g->n, (v && (v & (v - 1)) == 0 && v <= 64) ? v : 0, g->device,
                                           g->opts.output_mode);
  // Few tiles, many rows: bands, as for the row kernel.
  rngi::LaunchShape sh{};
  sh.vpt = vpt;
  sh.block = rngi::kGenBlock;
  bool swap = false;
  a.out_mode = g->opts.output_mode;
  const uint64_t br = rngi::choose_band_rows(g->n, iterations, sh, g->device, true, a.out_mode);
  if (br) {
    rc = setup_bands(g, a, br, &swap, err);
    if (rc) return rc;
  }
  long op = op_begin(g, "CHECKSUM_KERNEL", kQueueMain, g->compute);
  st = rngi::launch_checksum(a, vpt, row_xor_dev, row_sum_dev, g->compute);
  op_end(g, op, g->compute);
  rc = rngi::cuda_fail(err, st, "checksum kernel launch");
  if (rc) return rc;
  if (swap) std::swap(g->d_state, g->d_state2);
  g->materialized = true;
  g->pos += iterations;
  return RNG_OK;
}

int rng_skip(rng_gen *g, uint64_t iterations, rng_err **err) {
  int rc = check_gen(g, err, "rng_skip");
  if (rc) return rc;
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_skip: generator not initialised (call rng_init)");
  if (iterations == 0) return RNG_OK;
  uint64_t cols[64];
  rngi::jump_matrix(iterations, cols);  // on the host, before the timed op
  long op = op_begin(g, "SKIP_KERNEL", kQueueMain, g->compute);
  cudaError_t st = rngi::launch_jump(g->d_state, g->n, g->g0, g->key, !g->materialized, cols, g->compute);
  op_end(g, op, g->compute);
  rc = rngi::cuda_fail(err, st, "jump kernel launch");
  if (rc) return rc;
  g->materialized = true;
  g->pos += iterations;  // wraps modulo 2^64 like the period of the update
  return RNG_OK;
}

int rng_host_stats_get(const rng_gen *g, rng_host_stats *out) {
  if (!g || !out) return RNG_EINVAL;
  *out = g->host_stats;
  return RNG_OK;
}

int rng_position(const rng_gen *g, uint64_t *position) {
  if (!g || !position) return RNG_EINVAL;
  *position = g->pos;
  return RNG_OK;
}

int rng_streams(const rng_gen *g, uint64_t *streams) {
  if (!g || !streams) return RNG_EINVAL;
  *streams = g->n;
  return RNG_OK;
}

int rng_get_state(rng_gen *g, uint64_t *host_states, rng_err **err) {
  int rc = check_gen(g, err, "rng_get_state");
  if (rc) return rc;
  if (!host_states) return rngi::fail(err, RNG_EINVAL, "rng_get_state: NULL output");
  if (!g->initialized) return rngi::fail(err, RNG_ESTATE, "rng_get_state: generator not initialised");
  if (!g->materialized) {
    rc = rngi::cuda_fail(err, rngi::launch_init(g->d_state, g->n, g->g0, g->key, g->compute), "init kernel launch");
    if (rc) return rc;
    g->materialized = true;
  }
  cudaError_t st = cudaMemcpyAsync(host_states, g->d_state, g->n * 8, cudaMemcpyDeviceToHost, g->compute);
  if (st == cudaSuccess) st = cudaStreamSynchronize(g->compute);
  return rngi::cuda_fail(err, st, "rng_get_state copy");
}

int rng_set_state(rng_gen *g, const uint64_t *host_states, uint64_t position, rng_err **err) {
  int rc = check_gen(g, err, "rng_set_state");
  if (rc) return rc;
  if (!host_states) return rngi::fail(err, RNG_EINVAL, "rng_set_state: NULL states");
  cudaError_t st = cudaMemcpyAsync(g->d_state, host_states, g->n * 8, cudaMemcpyHostToDevice, g->compute);
  if (st == cudaSuccess) st = cudaStreamSynchronize(g->compute);
  rc = rngi::cuda_fail(err, st, "rng_set_state copy");
  if (rc) return rc;
  g->materialized = true;
  g->initialized = true;
  g->pos = position;
  return RNG_OK;
}

int rng_sync(rng_gen *g, rng_err **err) {
  int rc = check_gen(g, err, "rng_sync");
  if (rc) return rc;
  cudaError_t st = cudaStreamSynchronize(g->compute);
  if (st == cudaSuccess) st = cudaStreamSynchronize(g->copy);
  return rngi::cuda_fail(err, st, "rng_sync");
}

void *rng_compute_stream(rng_gen *g) { return g ? static_cast<void *>(g->compute) : nullptr; }

int rng_launch_config(const rng_gen *g, uint32_t *vpt, uint32_t *block, uint32_t *grid) {
  if (!g) return RNG_EINVAL;
  if (vpt) *vpt = g->shape.vpt;
  if (block) *block = g->shape.block;
  if (grid) *grid = g->shape.grid;
  return RNG_OK;
}

int rng_last_launch(const rng_gen *g, rng_launch_info *info, rng_err **err) {
  if (!g || !info) return rngi::fail(err, RNG_EINVAL, "rng_last_launch: NULL generator or info");
  if (info->struct_size != sizeof(rng_launch_info))
    return rngi::fail(err, RNG_EINVAL, "rng_last_launch: info.struct_size %u != %zu", info->struct_size,
                      sizeof(rng_launch_info));
  const rngi::LaunchInfo &l = g->last_launch;
  if (l.block == 0) return rngi::fail(err, RNG_ESTATE, "rng_last_launch: no row-kernel launch yet");
  info->kernel = l.kernel;
  info->values_per_thread = l.vpt;
  info->block_threads = l.block;
  info->grid_blocks = l.grid;
  info->row_buffers = l.row_buffers;
  info->band_rows = l.band_rows;
  return RNG_OK;
}

rng_prof *rng_profiler(rng_gen *g, rng_err **err) {
  if (check_gen(g, err, "rng_profiler")) return nullptr;
  cudaError_t st = cudaStreamSynchronize(g->compute);
  if (st == cudaSuccess) st = cudaStreamSynchronize(g->copy);
  if (rngi::cuda_fail(err, st, "rng_profiler: synchronize")) return nullptr;
  const double elapsed =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - g->wall0).count();
  rngi::prof_clear(g->prof);
  for (const OpRec &op : g->ops) {
    float t0 = 0.f, t1 = 0.f;
    st = cudaEventElapsedTime(&t0, g->origin, g->evpool[op.ev0]);
    if (st == cudaSuccess) st = cudaEventElapsedTime(&t1, g->origin, g->evpool[op.ev1]);
    if (st != cudaSuccess) {
      rngi::cuda_fail(err, st, "cudaEventElapsedTime");
      return nullptr;
    }
    rngi::prof_add(g->prof, op.queue, op.name, t0 * 1e-3, t1 * 1e-3);
  }
  rng_prof_set_elapsed(g->prof, elapsed);
  if (rng_prof_calc(g->prof, err)) return nullptr;
  return g->prof;
}

const char *rng_profile_summary(rng_gen *g, int agg_sort, int ovl_sort, rng_err **err) {
  rng_prof *p = rng_profiler(g, err);
  if (!p) return nullptr;
  const char *s = rng_prof_summary(p, agg_sort, ovl_sort);
  g->summary = s ? s : "";
  return g->summary.c_str();
}

int rng_profile_export(rng_gen *g, const char *path, rng_err **err) {
  rng_prof *p = rng_profiler(g, err);
  if (!p) return err && *err ? (*err)->code : RNG_ECUDA;
  return rng_prof_export(p, path, err);
}

int rng_profile_reset(rng_gen *g, rng_err **err) {
  int rc = check_gen(g, err, "rng_profile_reset");
  if (rc) return rc;
  return profile_restart(g, err);
}

int rng_profile_stat(rng_gen *g, const char *name, uint64_t *count, double *total_s, rng_err **err) {
  int rc = check_gen(g, err, "rng_profile_stat");
  if (rc) return rc;
  if (!name) return rngi::fail(err, RNG_EINVAL, "rng_profile_stat: NULL name");
  uint64_t n = 0;
  double tot = 0.0;
  bool synced = false;
  for (const OpRec &op : g->ops) {
    if (strcmp(op.name, name) != 0) continue;
    if (!synced) {
      cudaError_t st = cudaEventSynchronize(g->evpool[g->ops.back().ev1]);
      if (st == cudaSuccess) st = cudaStreamSynchronize(g->compute);
      if (st == cudaSuccess) st = cudaStreamSynchronize(g->copy);
      rc = rngi::cuda_fail(err, st, "rng_profile_stat: synchronize");
      if (rc) return rc;
      synced = true;
    }
    float ms = 0.f;
    cudaError_t st = cudaEventElapsedTime(&ms, g->evpool[op.ev0], g->evpool[op.ev1]);
    rc = rngi::cuda_fail(err, st, "cudaEventElapsedTime");
    if (rc) return rc;
    ++n;
    tot += ms * 1e-3;
  }
  if (count) *count = n;
  if (total_s) *total_s = tot;
  return RNG_OK;
}

}  // extern "C"
