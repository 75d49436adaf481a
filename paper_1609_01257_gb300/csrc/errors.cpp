// Error objects, status strings and the live-object / launch counters.
// Errors follow the two-route convention of the cf4ocl paper (Section 3.1):
// a status code as the return value and an optional error object passed as
// the last argument.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>

#include "internal.h"

namespace {
std::atomic<long> g_live{0};
std::atomic<uint64_t> g_launches{0};
}  // namespace

namespace rngi {

int fail(rng_err **err, int code, const char *fmt, ...) {
  if (err && !*err) {
    rng_err *e = static_cast<rng_err *>(calloc(1, sizeof(rng_err)));
    if (e) {
      e->code = code;
      va_list ap;
      va_start(ap, fmt);
      vsnprintf(e->msg, sizeof(e->msg), fmt, ap);
      va_end(ap);
      *err = e;
    }
  }
  return code;
}

int cuda_fail(rng_err **err, cudaError_t st, const char *what) {
  if (st == cudaSuccess) return RNG_OK;
  const int code = (st == cudaErrorMemoryAllocation) ? RNG_ENOMEM : RNG_ECUDA;
  return fail(err, code, "%s: %s (%s)", what, cudaGetErrorString(st), cudaGetErrorName(st));
}

void live_inc() { g_live.fetch_add(1); }
void live_dec() { g_live.fetch_sub(1); }
void count_launch(uint64_t n) { g_launches.fetch_add(n); }

}  // namespace rngi

extern "C" {

void rng_err_clear(rng_err **err) {
  if (err && *err) {
    free(*err);
    *err = nullptr;
  }
}

const char *rng_strerror(int code) {
  switch (code) {
    case RNG_OK: return "success";
    case RNG_EINVAL: return "invalid argument";
    case RNG_ENOMEM: return "out of memory";
    case RNG_ECUDA: return "CUDA error";
    case RNG_ESTATE: return "call out of order";
    case RNG_ETIMEOUT: return "wait timed out";
    case RNG_EBUDGET: return "memory budget exceeded";
    case RNG_ESINK: return "host consumer failed";
    default: return "unknown status";
  }
}

long rng_live_objects(void) { return g_live.load(); }
uint64_t rng_launch_count(void) { return g_launches.load(); }

}  // extern "C"
