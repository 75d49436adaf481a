// Served form: continuous batching of generation requests on one GPU.
//
// A scheduler thread owns the device: it admits queued requests in arrival
// order against a device-memory arena (outputs + per-request states) and a
// slot limit, and launches "steps".  A step is one work-list kernel over the
// next rows of every admitted request (a fair share of the step's byte
// quantum each, at least one row), so a request that arrives while others are
// running joins the next step instead of waiting for them to finish, and a
// large request is spread over several steps, continuing each time from its
// state kept on the device.  Up to max_steps_in_flight steps are queued on
// the stream; a step's completion event marks the requests whose last rows it
// produced as done.  The arithmetic is the generator's own (hash init, then
// xorshift), so every output equals the same request served alone.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"
#include "prng_math.cuh"

namespace {

using Clock = std::chrono::steady_clock;
constexpr uint64_t kAlign = 256;
constexpr uint32_t kBlock = 256;

struct Request {
  uint64_t ticket = 0, seed = 0, streams = 0, iters = 0;
  uint32_t key = 0;
  uint64_t issued = 0;
  uint64_t out_off = 0, out_bytes = 0, state_off = 0, state_bytes = 0;
  Clock::time_point t_submit;
  double latency = 0.0;
  bool done = false;
  bool released = false;      // output returned; kept only for its state
  bool keep_state = false;    // final states stay resident for a continuation
  bool has_state = false;     // state_off/state_bytes hold an arena block
  bool state_is_hash = true;  // first chunk starts from the id hash
  uint64_t first_iteration = 0;
  uint64_t parent = 0;        // ticket continued from (0: fresh generator)
  uint64_t child = 0;         // ticket continuing this one
};

struct TableSlot {
  rngi::BatchInstance *h_inst = nullptr, *d_inst = nullptr;
  rngi::BatchUnit *h_units = nullptr, *d_units = nullptr;
  uint32_t *d_counter = nullptr;
  cudaEvent_t uploaded = nullptr;  // the slot's tables are on the device
  cudaEvent_t done = nullptr;      // the step using the slot has finished
};

struct Step {
  size_t slot;
  std::vector<uint64_t> finishing;
  uint64_t bytes;
};

// First-fit arena over one device allocation; blocks are kAlign-aligned.
class Arena {
 public:
  uint64_t size = 0, used = 0, peak = 0;
  std::map<uint64_t, uint64_t> free_;  // offset -> length
  void reset(uint64_t sz) {
    size = sz;
    used = 0;
    free_.clear();
    free_[0] = sz;
  }
  bool alloc(uint64_t bytes, uint64_t *off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      *off = it->first;
      const uint64_t rest = it->second - bytes;
      const uint64_t roff = it->first + bytes;
      free_.erase(it);
      if (rest) free_[roff] = rest;
      used += bytes;
      peak = std::max(peak, used);
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    used -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
};

}  // namespace

struct rng_server {
  rng_server_opts opts{};
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // Table uploads and counter resets run here, ordered before their step's
  // kernel by the slot's `uploaded` event, so that they overlap the step
  // already running instead of queueing behind it on `stream`.
  cudaStream_t upload = nullptr;
  uint8_t *base = nullptr;
  Arena arena;
  std::vector<TableSlot> slots;
  std::vector<size_t> free_slots;
  int grid_per_sm = 1, sms = 1;
  size_t rr = 0;  // rotating start of the next step's scan over active requests

  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Request *> pending;
  std::vector<Request *> active;
  std::deque<Step> inflight;
  std::unordered_map<uint64_t, Request *> tickets;
  std::deque<uint64_t> done_q;
  uint64_t next_ticket = 1;
  bool stop = false;
  int fatal = RNG_OK;
  std::string fatal_msg;
  rng_server_stats st{};
  std::thread th;

  uint64_t *addr(uint64_t off) { return reinterpret_cast<uint64_t *>(base + off); }

  void fail_locked(cudaError_t e, const char *what) {
    if (fatal == RNG_OK) {
      fatal = RNG_ECUDA;
      fatal_msg = std::string(what) + ": " + cudaGetErrorString(e);
    }
  }

  // Builds and launches one step; returns false if nothing was launched.
  bool launch_step_locked() {
    std::vector<Request *> want;
    const size_t na = active.size();
    for (size_t i = 0; i < na; ++i) {
      Request *r = active[(rr + i) % na];
      if (r->issued < r->iters) want.push_back(r);
    }
    ++rr;
    if (want.empty() || free_slots.empty()) return false;
    const size_t slot = free_slots.back();
    TableSlot &ts = slots[slot];
    const uint64_t tile = uint64_t(kBlock) * opts.values_per_thread;
    const uint64_t share = std::max<uint64_t>(1, opts.step_bytes / want.size());
    uint32_t n_inst = 0;
    uint64_t n_units = 0, bytes = 0;
    Step step{slot, {}, 0};
    for (Request *r : want) {
      const uint64_t row_bytes = 8 * r->streams;
      uint64_t rows = std::max<uint64_t>(1, share / row_bytes);
      rows = std::min(rows, r->iters - r->issued);
      const uint64_t units = (r->streams + tile - 1) / tile;
      if (n_units + units > opts.max_units_per_step || n_inst >= opts.max_active) break;
      rngi::BatchInstance &in = ts.h_inst[n_inst];
      in.out = addr(r->out_off) + r->issued * r->streams;
      in.state = addr(r->state_off);
      in.streams = r->streams;
      in.rows = rows;
      in.key = r->key;
      in.vec = (r->streams % 2 == 0) ? 1u : 0u;  // arena blocks are 256-byte aligned
      in.from_hash = (r->issued == 0 && r->state_is_hash) ? 1u : 0u;
      in.write_state = (r->issued + rows < r->iters || r->keep_state) ? 1u : 0u;
      for (uint64_t s0 = 0; s0 < r->streams; s0 += tile)
        ts.h_units[n_units++] = {n_inst, static_cast<uint32_t>(std::min(tile, r->streams - s0)), s0};
      ++n_inst;
      r->issued += rows;
      bytes += rows * row_bytes;
      if (r->issued == r->iters) step.finishing.push_back(r->ticket);
    }
    if (n_inst == 0) return false;  // a single request needs more units than a step holds
    // Units stay in request order, each request's tiles together: blocks
    // running at the same time write neighbouring parts of one output (as in
    // the batched form, where this beat sorting all units by size).
    // The slot is free, so no kernel reads its device tables any more and
    // its last upload from the host tables has finished.
    cudaError_t e = cudaMemcpyAsync(ts.d_inst, ts.h_inst, n_inst * sizeof(rngi::BatchInstance),
                                    cudaMemcpyHostToDevice, upload);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ts.d_units, ts.h_units, n_units * sizeof(rngi::BatchUnit), cudaMemcpyHostToDevice, upload);
    // Work distribution: one unit per block (hardware dispatch in table
    // order), or persistent blocks taking units from a counter.
    const bool per_block = opts.mode != 2;
    if (e == cudaSuccess && !per_block) e = cudaMemsetAsync(ts.d_counter, 0, sizeof(uint32_t), upload);
    if (e == cudaSuccess) e = cudaEventRecord(ts.uploaded, upload);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(stream, ts.uploaded, 0);
    const uint64_t resident = uint64_t(sms) * grid_per_sm;
    const uint32_t grid = per_block ? static_cast<uint32_t>(n_units)
                                    : static_cast<uint32_t>(std::max<uint64_t>(1, std::min<uint64_t>(resident, n_units)));
    if (e == cudaSuccess)
      e = rngi::launch_batch(ts.d_inst, ts.d_units, static_cast<uint32_t>(n_units), per_block ? nullptr : ts.d_counter,
                             opts.values_per_thread, kBlock, grid, stream);
    if (e == cudaSuccess) e = cudaEventRecord(ts.done, stream);
    if (e != cudaSuccess) {
      fail_locked(e, "server step launch");
      return false;
    }
    free_slots.pop_back();
    step.bytes = bytes;
    inflight.push_back(std::move(step));
    st.steps++;
    st.bytes_generated += bytes;
    return true;
  }

  void complete_steps_locked() {
    while (!inflight.empty()) {
      Step &s = inflight.front();
      cudaError_t e = cudaEventQuery(slots[s.slot].done);
      if (e == cudaErrorNotReady) return;
      if (e != cudaSuccess) {
        fail_locked(e, "server step");
        return;
      }
      const auto now = Clock::now();
      for (uint64_t t : s.finishing) {
        Request *r = tickets[t];
        r->latency = std::chrono::duration<double>(now - r->t_submit).count();
        r->done = true;
        if (!r->keep_state && r->has_state) {
          arena.release(r->state_off, r->state_bytes);
          r->has_state = false;
        }
        active.erase(std::find(active.begin(), active.end(), r));
        done_q.push_back(t);
        st.completed++;
      }
      free_slots.push_back(s.slot);
      inflight.pop_front();
      cv_done.notify_all();
    }
  }

  // A continuation can start once its parent has finished: it takes over the
  // parent's resident states instead of hashing the ids.
  void admit_locked() {
    while (!pending.empty() && active.size() < opts.max_active) {
      Request *r = pending.front();
      Request *parent = r->parent ? tickets[r->parent] : nullptr;
      if (parent && !parent->done) return;  // arrival order is kept
      uint64_t out_off, state_off = 0;
      if (!arena.alloc(r->out_bytes, &out_off)) return;
      if (parent) {
        r->state_off = parent->state_off;
        r->state_bytes = parent->state_bytes;
        r->has_state = true;
        r->state_is_hash = false;
        parent->has_state = false;
        if (parent->released) {
          tickets.erase(parent->ticket);
          delete parent;
        }
      } else {
        if (!arena.alloc(r->state_bytes, &state_off)) {
          arena.release(out_off, r->out_bytes);
          return;
        }
        r->state_off = state_off;
        r->has_state = true;
      }
      r->out_off = out_off;
      pending.pop_front();
      active.push_back(r);
      st.peak_active = std::max<uint64_t>(st.peak_active, active.size());
    }
  }

  void run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
      complete_steps_locked();
      if (fatal != RNG_OK) {
        cv_done.notify_all();
        // Keep draining completions so destroy can finish; launch nothing.
        if (stop && inflight.empty()) break;
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(200));
        lk.lock();
        continue;
      }
      if (!stop) admit_locked();
      bool launched = false;
      if (!stop)
        while (inflight.size() < opts.max_steps_in_flight && launch_step_locked()) launched = true;
      if (stop && inflight.empty()) break;
      if (launched) continue;
      if (inflight.empty()) {
        cv_sched.wait(lk);
      } else {
        // A step is running: poll its event at a short interval.
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(20));
        lk.lock();
      }
    }
  }
};

extern "C" {

void rng_server_opts_default(rng_server_opts *o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->struct_size = sizeof(rng_server_opts);
  o->max_active = 1024;
  o->hbm_budget_bytes = uint64_t(64) << 30;
  o->step_bytes = uint64_t(2) << 30;
  o->max_steps_in_flight = 2;
  o->values_per_thread = 4;
  o->max_units_per_step = 1u << 20;
  o->mode = 1;
  o->device = -1;
  o->stream = nullptr;
}

int rng_server_create(const rng_server_opts *opts, rng_server **out, rng_err **err) {
  if (!out) return rngi::fail(err, RNG_EINVAL, "rng_server_create: NULL output pointer");
  *out = nullptr;
  rng_server_opts o;
  rng_server_opts_default(&o);
  if (opts) {
    if (opts->struct_size != sizeof(rng_server_opts))
      return rngi::fail(err, RNG_EINVAL, "rng_server_create: opts.struct_size mismatch");
    o = *opts;
  }
  if (o.values_per_thread == 0) o.values_per_thread = 4;
  if (!rngi::batch_vpt_supported(o.values_per_thread))
    return rngi::fail(err, RNG_EINVAL,
                      "rng_server_create: values_per_thread must be one of 1, 2, 4, 6, 8, 12, 16, 24, 32");
  if (o.mode < 1 || o.mode > 2) return rngi::fail(err, RNG_EINVAL, "rng_server_create: mode must be 1 or 2");
  if (o.max_active == 0 || o.max_steps_in_flight == 0 || o.step_bytes == 0 || o.max_units_per_step == 0 ||
      o.hbm_budget_bytes < kAlign)
    return rngi::fail(err, RNG_EINVAL, "rng_server_create: zero limit in options");
  int dev = o.device;
  if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return rngi::fail(err, RNG_ECUDA, "cudaGetDevice failed");
  cudaError_t e = cudaSetDevice(dev);
  if (e != cudaSuccess) return rngi::cuda_fail(err, e, "cudaSetDevice");
  rng_server *s = new (std::nothrow) rng_server();
  if (!s) return rngi::fail(err, RNG_ENOMEM, "rng_server_create: host allocation failed");
  rngi::live_inc();
  s->opts = o;
  s->device = dev;
  s->sms = rngi::device_sm_count(dev);
  s->grid_per_sm = std::max(1, rngi::batch_blocks_per_sm(o.values_per_thread, kBlock));
  int rc = RNG_OK;
  if (o.stream) {
    s->stream = static_cast<cudaStream_t>(o.stream);
  } else {
    rc = rngi::cuda_fail(err, cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    s->own_stream = rc == RNG_OK;
  }
  if (!rc) rc = rngi::cuda_fail(err, cudaStreamCreateWithFlags(&s->upload, cudaStreamNonBlocking), "cudaStreamCreate");
  if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&s->base, o.hbm_budget_bytes), "cudaMalloc(server arena)");
  if (!rc) s->arena.reset(o.hbm_budget_bytes);
  const uint32_t n_slots = o.max_steps_in_flight + 1;
  for (uint32_t i = 0; i < n_slots && !rc; ++i) {
    TableSlot t;
    rc = rngi::cuda_fail(err, cudaHostAlloc(&t.h_inst, o.max_active * sizeof(rngi::BatchInstance), 0), "cudaHostAlloc");
    if (!rc) rc = rngi::cuda_fail(err, cudaHostAlloc(&t.h_units, size_t(o.max_units_per_step) * sizeof(rngi::BatchUnit), 0), "cudaHostAlloc");
    if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&t.d_inst, o.max_active * sizeof(rngi::BatchInstance)), "cudaMalloc");
    if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&t.d_units, size_t(o.max_units_per_step) * sizeof(rngi::BatchUnit)), "cudaMalloc");
    if (!rc) rc = rngi::cuda_fail(err, cudaMalloc(&t.d_counter, sizeof(uint32_t)), "cudaMalloc");
    if (!rc) rc = rngi::cuda_fail(err, cudaEventCreateWithFlags(&t.done, cudaEventDisableTiming), "cudaEventCreate");
    if (!rc) rc = rngi::cuda_fail(err, cudaEventCreateWithFlags(&t.uploaded, cudaEventDisableTiming), "cudaEventCreate");
    s->slots.push_back(t);
    s->free_slots.push_back(i);
  }
  if (rc) {
    rng_server_destroy(s);
    return rc;
  }
  s->th = std::thread([s] { s->run(); });
  *out = s;
  return RNG_OK;
}

int rng_server_submit_ex(rng_server *s, uint64_t seed, uint64_t streams, uint64_t iterations, uint32_t flags,
                         uint64_t continue_ticket, uint64_t *ticket, rng_err **err) {
  if (!s || !ticket) return rngi::fail(err, RNG_EINVAL, "rng_server_submit: NULL argument");
  if (flags & ~uint32_t(RNG_REQ_KEEP_STATE))
    return rngi::fail(err, RNG_EINVAL, "rng_server_submit: unknown flags 0x%x", flags);
  std::lock_guard<std::mutex> lk(s->mu);
  Request *parent = nullptr;
  if (continue_ticket) {
    auto it = s->tickets.find(continue_ticket);
    if (it == s->tickets.end() || !it->second->keep_state || it->second->child)
      return rngi::fail(err, RNG_ESTATE,
                        "rng_server_submit: ticket %llu is not a request kept for continuation (or already continued)",
                        (unsigned long long)continue_ticket);
    parent = it->second;
    seed = parent->seed;
    streams = parent->streams;
  }
  if (streams == 0 || streams > (uint64_t(1) << 32) || iterations == 0)
    return rngi::fail(err, RNG_EINVAL, "rng_server_submit: streams must be in [1, 2^32] and iterations >= 1");
  if (iterations > (~uint64_t(0) / 8) / streams - 1)
    return rngi::fail(err, RNG_EINVAL, "rng_server_submit: size overflows");
  const uint64_t tile = uint64_t(kBlock) * s->opts.values_per_thread;
  if ((streams + tile - 1) / tile > s->opts.max_units_per_step)
    return rngi::fail(err, RNG_EINVAL, "rng_server_submit: request wider than one step's work table");
  if (s->fatal != RNG_OK)
    return rngi::fail(err, s->fatal, "rng_server_submit: server failed: %s", s->fatal_msg.c_str());
  const uint64_t out_bytes = 8 * streams * iterations, state_bytes = 8 * streams;
  const uint64_t need = (out_bytes + kAlign - 1) / kAlign * kAlign + (state_bytes + kAlign - 1) / kAlign * kAlign;
  if (need > s->opts.hbm_budget_bytes) {
    s->st.rejected++;
    return rngi::fail(err, RNG_EBUDGET, "rng_server_submit: request needs %llu bytes, budget is %llu",
                      (unsigned long long)need, (unsigned long long)s->opts.hbm_budget_bytes);
  }
  Request *r = new (std::nothrow) Request();
  if (!r) return rngi::fail(err, RNG_ENOMEM, "rng_server_submit: host allocation failed");
  r->seed = seed;
  r->streams = streams;
  r->iters = iterations;
  r->key = prng::seed_key(seed);
  r->out_bytes = out_bytes;
  r->state_bytes = state_bytes;
  r->keep_state = (flags & RNG_REQ_KEEP_STATE) != 0;
  r->ticket = s->next_ticket++;
  if (parent) {
    r->parent = parent->ticket;
    r->first_iteration = parent->first_iteration + parent->iters;
    parent->child = r->ticket;
  }
  r->t_submit = Clock::now();
  s->tickets[r->ticket] = r;
  s->pending.push_back(r);
  s->st.submitted++;
  *ticket = r->ticket;
  s->cv_sched.notify_one();
  return RNG_OK;
}

int rng_server_submit(rng_server *s, uint64_t seed, uint64_t streams, uint64_t iterations, uint64_t *ticket,
                      rng_err **err) {
  return rng_server_submit_ex(s, seed, streams, iterations, 0, 0, ticket, err);
}

int rng_server_poll(rng_server *s, uint32_t max, uint64_t *tickets, uint64_t **outs, double *latency_s,
                    uint32_t *n_done, uint32_t timeout_ms, rng_err **err) {
  if (!s || !n_done || (max && !tickets)) return rngi::fail(err, RNG_EINVAL, "rng_server_poll: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                      [&] { return !s->done_q.empty() || s->fatal != RNG_OK; });
  uint32_t n = 0;
  while (n < max && !s->done_q.empty()) {
    const uint64_t t = s->done_q.front();
    s->done_q.pop_front();
    Request *r = s->tickets[t];
    tickets[n] = t;
    if (outs) outs[n] = s->addr(r->out_off);
    if (latency_s) latency_s[n] = r->latency;
    ++n;
  }
  *n_done = n;
  if (n == 0 && s->fatal != RNG_OK)
    return rngi::fail(err, s->fatal, "rng_server_poll: server failed: %s", s->fatal_msg.c_str());
  return RNG_OK;
}

int rng_server_read(rng_server *s, uint64_t ticket, uint64_t first, uint64_t count, uint64_t *host_dst,
                    rng_err **err) {
  if (!s || (count && !host_dst)) return rngi::fail(err, RNG_EINVAL, "rng_server_read: NULL argument");
  uint64_t *src;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end() || !it->second->done || it->second->released)
      return rngi::fail(err, RNG_ESTATE, "rng_server_read: ticket %llu is not a completed, unreleased request",
                        (unsigned long long)ticket);
    Request *r = it->second;
    if (first > r->streams * r->iters || count > r->streams * r->iters - first)
      return rngi::fail(err, RNG_EINVAL, "rng_server_read: range outside the output");
    src = s->addr(r->out_off) + first;
  }
  cudaSetDevice(s->device);
  return rngi::cuda_fail(err, cudaMemcpy(host_dst, src, count * 8, cudaMemcpyDeviceToHost), "rng_server_read");
}

int rng_server_release(rng_server *s, uint64_t ticket, rng_err **err) {
  if (!s) return rngi::fail(err, RNG_EINVAL, "rng_server_release: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->tickets.find(ticket);
  if (it == s->tickets.end() || !it->second->done || it->second->released)
    return rngi::fail(err, RNG_ESTATE, "rng_server_release: ticket %llu is not a completed, unreleased request",
                      (unsigned long long)ticket);
  Request *r = it->second;
  if (r->released)
    return rngi::fail(err, RNG_ESTATE, "rng_server_release: ticket %llu already released", (unsigned long long)ticket);
  s->arena.release(r->out_off, r->out_bytes);
  r->released = true;
  s->st.released++;
  if (r->has_state && !r->child) {  // kept states nobody continues: free them too
    s->arena.release(r->state_off, r->state_bytes);
    r->has_state = false;
  }
  if (!r->has_state) {
    s->tickets.erase(it);
    delete r;
  }
  s->cv_sched.notify_one();
  return RNG_OK;
}

int rng_server_get_stats(rng_server *s, rng_server_stats *out) {
  if (!s || !out) return RNG_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  out->pending = s->pending.size();
  out->active = s->active.size();
  out->bytes_in_use = s->arena.used;
  out->peak_bytes_in_use = s->arena.peak;
  return RNG_OK;
}

void rng_server_destroy(rng_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_sched.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  if (s->upload) cudaStreamSynchronize(s->upload);
  for (auto &kv : s->tickets) delete kv.second;
  for (TableSlot &t : s->slots) {
    cudaFreeHost(t.h_inst);
    cudaFreeHost(t.h_units);
    cudaFree(t.d_inst);
    cudaFree(t.d_units);
    cudaFree(t.d_counter);
    if (t.done) cudaEventDestroy(t.done);
    if (t.uploaded) cudaEventDestroy(t.uploaded);
  }
  cudaFree(s->base);
  if (s->upload) cudaStreamDestroy(s->upload);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
  delete s;
  rngi::live_dec();
}

}  // extern "C"
