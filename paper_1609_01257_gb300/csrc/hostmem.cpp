// Page-locked host memory for host output (rng_host_alloc / rng_host_free).
//
// Section 5 reads every generated batch into host memory.  On Grace-Blackwell
// the rate at which the GPU writes a large destination over NVLink-C2C depends
// on the pages behind it: into 64 KiB pages (what cudaHostAlloc returns) copies
// stall intermittently, for every engine that moves the bytes; into 512 MiB
// transparent huge pages they run at the link rate throughout.  This
// allocator maps anonymous memory aligned to the huge-page size, asks for
// huge pages (MADV_HUGEPAGE), faults every page in from a few threads and
// page-locks the range with cudaHostRegister.
#include <cuda_runtime.h>
#include <errno.h>
#include <stdio.h>
#include <string.h>
#include <sys/mman.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

struct Mapping {
  size_t len;
};

std::mutex g_mu;
std::map<void *, Mapping> g_maps;  // page-locked ranges handed out, by start address

size_t base_page() {
  const long p = sysconf(_SC_PAGESIZE);
  return p > 0 ? static_cast<size_t>(p) : 4096;
}

// Transparent huge-page size of this kernel (PMD size), 2 MiB when unknown.
size_t huge_page() {
  size_t v = 0;
  if (FILE *f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long x = 0;
    if (fscanf(f, "%llu", &x) == 1) v = static_cast<size_t>(x);
    fclose(f);
  }
  return v >= base_page() && (v & (v - 1)) == 0 ? v : (size_t(2) << 20);
}

// Faults every page of [p, p + len) in, writing one zero byte per base page
// (the kernel zero-fills new pages, so the contents stay zero), from up to
// 16 threads of at least 256 MiB each.
void touch(char *p, size_t len) {
  const size_t page = base_page();
  const size_t per_min = size_t(256) << 20;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t n = std::max<size_t>(1, std::min<size_t>({hw, 16, (len + per_min - 1) / per_min}));
  const size_t per = ((len / n + page - 1) / page) * page;
  auto work = [p, len, page](size_t a, size_t b) {
    for (size_t o = a; o < b && o < len; o += page) *reinterpret_cast<volatile char *>(p + o) = 0;
  };
  std::vector<std::thread> th;
  for (size_t k = 1; k < n; ++k) {
    try {
      th.emplace_back(work, k * per, (k + 1) * per);
    } catch (...) {
      work(k * per, (k + 1) * per);  // no thread: touch it here
    }
  }
  work(0, per);
  for (std::thread &t : th) t.join();
}

}  // namespace

extern "C" {

int rng_host_alloc(size_t bytes, uint32_t flags, void **out, rng_err **err) {
  if (!out) return rngi::fail(err, RNG_EINVAL, "rng_host_alloc: NULL output pointer");
  *out = nullptr;
  if (bytes == 0) return rngi::fail(err, RNG_EINVAL, "rng_host_alloc: zero bytes");
  if (flags & ~uint32_t(RNG_HOST_HUGE_PAGES))
    return rngi::fail(err, RNG_EINVAL, "rng_host_alloc: unknown flags 0x%x", flags);
  const bool huge = flags & RNG_HOST_HUGE_PAGES;
  const size_t align = huge ? huge_page() : base_page();
  if (bytes > (~size_t(0) >> 1) - align)
    return rngi::fail(err, RNG_EINVAL, "rng_host_alloc: %zu bytes is too large", bytes);
  const size_t len = (bytes + align - 1) / align * align;
  // Over-map by one alignment unit and trim, so the range starts on a
  // huge-page boundary (huge pages back only aligned ranges).
  void *raw = mmap(nullptr, len + align, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED)
    return rngi::fail(err, RNG_ENOMEM, "rng_host_alloc: mmap of %zu bytes failed: %s", len + align, strerror(errno));
  char *r = static_cast<char *>(raw);
  char *p = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(r) + align - 1) / align * align);
  if (p > r) munmap(r, static_cast<size_t>(p - r));
  const size_t tail = static_cast<size_t>((r + len + align) - (p + len));
  if (tail) munmap(p + len, tail);
  // Without transparent huge pages (disabled in the kernel) the advice fails
  // and the range keeps base pages; the memory is still usable.
  madvise(p, len, huge ? MADV_HUGEPAGE : MADV_NOHUGEPAGE);
  touch(p, len);
  cudaError_t st = cudaHostRegister(p, len, cudaHostRegisterPortable);
  if (st != cudaSuccess) {
    munmap(p, len);
    return rngi::cuda_fail(err, st, "rng_host_alloc: cudaHostRegister");
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_maps[p] = Mapping{len};
  }
  rngi::live_inc();
  *out = p;
  return RNG_OK;
}

int rng_host_free(void *p) {
  if (!p) return RNG_OK;
  size_t len = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_maps.find(p);
    if (it == g_maps.end()) return RNG_EINVAL;
    len = it->second.len;
    g_maps.erase(it);
  }
  const cudaError_t st = cudaHostUnregister(p);
  munmap(p, len);
  rngi::live_dec();
  return st == cudaSuccess ? RNG_OK : RNG_ECUDA;
}

}  // extern "C"
