/*
 * rng.h -- C ABI of the GB300 massive pseudo-random number generator.
 *
 * The generator is the example application of the cf4ocl paper (Fachada,
 * Lopes, Martins, Rosa, "cf4ocl: a C framework for OpenCL", Section 5,
 * "Example: massive pseudo-random number generator", kernels in Listings
 * S4 and S5).  n streams ("work-items") each hold a 64-bit state.  The
 * initial state of stream g is a hash of its 32-bit id (Listing S4) and is
 * also the stream's first output; every later output is the previous state
 * advanced by the xorshift update s ^= s << 21; s ^= s >> 35; s ^= s << 4
 * (Listing S5).  One call produces i iterations of n values in the
 * iteration-major layout of Section 5: value[it * n + g], 8 * n * i bytes
 * in total (Eq. 1).
 *
 * Run seed (the paper has none): the 32-bit id is XORed with
 * key(seed) = lo32(mix64(seed)) ^ hi32(mix64(seed)) before hashing, mix64
 * being the splitmix64 output finaliser.  key(0) = 0, so seed 0 gives the
 * paper's numbers exactly.
 *
 * Conventions (Section 3.1 of the paper):
 *  - every constructor (*_create, *_new) has a matching destructor;
 *    destructors accept NULL; rng_live_objects() counts live objects;
 *  - an error is reported twice: as the return value (an rng_status code)
 *    and, when the caller passes a non-NULL `rng_err **err` whose *err is
 *    NULL, as a newly allocated rng_err that the caller frees with
 *    rng_err_clear().  An *err that is already set is left as it is.
 *  - no function calls exit() or aborts the process.
 *  - strings returned by the library are owned by the object they came from
 *    and stay valid until the next call on that object or its destruction.
 */
#ifndef PRNG_GB300_RNG_H
#define PRNG_GB300_RNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ */
/* Errors                                                              */
/* ------------------------------------------------------------------ */
enum rng_status {
    RNG_OK = 0,
    RNG_EINVAL = 1,   /* bad argument (NULL object, size out of range, ...) */
    RNG_ENOMEM = 2,   /* device or pinned host allocation failed */
    RNG_ECUDA = 3,    /* a CUDA runtime call failed; message names it */
    RNG_ESTATE = 4,   /* call out of order (e.g. generate before init) */
    RNG_ETIMEOUT = 5, /* a bounded wait gave up */
    RNG_EBUDGET = 6,  /* request does not fit the memory budget */
    RNG_ESINK = 7     /* a host consumer callback returned non-zero */
};

typedef struct rng_err {
    int code;       /* one of rng_status */
    char msg[256];  /* human-readable description */
} rng_err;

/* Frees *err (if any) and sets it to NULL.  NULL-safe. */
void rng_err_clear(rng_err **err);
/* Static string naming a status code. */
const char *rng_strerror(int code);
/* Number of library objects (generators, profilers, batches, servers)
 * created and not yet destroyed -- the memcheck of Section 3.1. */
long rng_live_objects(void);
/* Number of CUDA kernels this library has launched in this process. */
uint64_t rng_launch_count(void);

/* ------------------------------------------------------------------ */
/* Options                                                             */
/* ------------------------------------------------------------------ */
typedef struct rng_opts {
    uint32_t struct_size;         /* sizeof(rng_opts), set by rng_opts_default */
    uint32_t values_per_thread;   /* streams per GPU thread: 1-8, 10, 12, ... 28
                                     (even), 32, 36, 40, 48 or 64; 0 = choose */
    uint32_t block_threads;       /* threads per block: 256 (0 = 256), or 128, 512,
                                     1024 with values_per_thread 2, 4, 6, 8, 12,
                                     16 or 24 (one 8-byte streaming store per value) */
    uint32_t fuse_init;           /* 1 (default): rng_init launches nothing and the
                                     first rng_generate hashes the ids itself;
                                     0: rng_init runs the separate init kernel */
    uint64_t stream_offset;       /* id of this object's first stream (a shard of
                                     a larger generator); ids g0 .. g0+n-1 */
    uint64_t device_buffer_bytes; /* host output: size of each of the two device
                                     buffers (ping-pong, Section 5); default 32 MiB */
    uint32_t host_slots;          /* pinned staging slots (device_buffer_bytes
                                     each) for pageable host output, sinks and
                                     host checksums; 0 (default) = the host
                                     consumers + 2, else at least 2 */
    uint32_t profiling;           /* 1 (default): time every kernel and copy with
                                     CUDA events for the profiler */
    void *compute_stream;         /* cudaStream_t for kernels; NULL = own stream */
    int32_t device;               /* CUDA device ordinal; -1 = current device */
    uint32_t store_policy;        /* 0 = default stores, 1 (default) = streaming
                                     stores (st.global.cs, evict-first), with
                                     the bulk-copy kernel where it measured
                                     faster (device outputs of at least 128
                                     rows per call) when the shape is left to
                                     the library (values_per_thread,
                                     block_threads, grid_blocks and
                                     store_width all 0); 2 =
                                     every device-output row staged in shared
                                     memory and written by TMA bulk copies
                                     (cp.async.bulk), 256-thread blocks, 0
                                     (= 8), 4, 8 or 16 values per thread.
                                     Host destinations always use register
                                     stores */
    uint32_t host_wait_ms;        /* longest wait for a free staging slot while a
                                     host consumer holds them all; 0 = 600000 */
    uint32_t store_width;         /* widest store in values: 1, 2 or 4 (the
                                     output's alignment may force narrower);
                                     0 = per shape (1 for >= 6 values per
                                     thread, else 4) */
    uint32_t grid_blocks;         /* blocks of the row kernel's grid; 0 = one per
                                     tile of block_threads x values_per_thread
                                     streams; fewer: blocks stride over tiles */
    uint32_t host_path;           /* host output: 0 = direct when the GPU can
                                     store into the destination (page-locked
                                     memory, or pageable memory on systems with
                                     pageable access such as Grace over
                                     NVLink-C2C), else double buffer;
                                     1 = always the double buffer of Section 5;
                                     2 = always direct (RNG_EINVAL if the GPU
                                     cannot store into the destination);
                                     3 = the double buffer with its reads done
                                     by a copy kernel on the copy stream (SMs
                                     storing into page-locked memory or the
                                     staging slots) instead of the copy engine.
                                     Sinks, file descriptors and host checksums
                                     go through page-locked staging slots: in
                                     modes 0 and 1 by the double buffer with
                                     copy-engine reads, in mode 3 with
                                     copy-kernel reads, and in mode 2 the
                                     kernel stores each chunk straight into
                                     its slot (no device buffer, no copy) */
    uint32_t host_consumers;      /* host threads draining the staging slots
                                     (at most 64).  0 (default): one for sinks
                                     (in order); for pageable copies and host
                                     checksums, the host's cores but one (1-16).
                                     Above 1, a sink is called concurrently
                                     from several threads, chunks in any
                                     order; rng_generate_fd always uses one */
    uint32_t output_mode;         /* value emitted for each state: 0 (default)
                                     the state itself, as in Section 5; 1 the
                                     xorshift64* scrambled value (state times
                                     0x2545F4914F6CDD1D modulo 2^64; Vigna,
                                     ACM TOMS 42(4), 2016), the stronger
                                     generator the paper says could replace
                                     plain xorshift.  The state sequence,
                                     rng_skip and the checkpoints are the same
                                     in both modes; the checksums are over
                                     the emitted values.  Mode 1 needs
                                     block_threads 0 or 256 and
                                     values_per_thread 0, 1, 2, 4, 8, 16, 24
                                     or 32, and always uses streaming stores */
} rng_opts;

void rng_opts_default(rng_opts *opts);

/* ------------------------------------------------------------------ */
/* Generator (Section 5: init kernel, rng kernel, device->host reads)  */
/* ------------------------------------------------------------------ */
typedef struct rng_gen rng_gen;  /* use one generator from one host thread at a time */

/* Creates a generator of `streams` streams (1 <= streams <= 2^32; ids
 * are reduced to 32 bits before hashing, as in Listing S4) with run seed
 * `seed`.  Allocates the state array (8 bytes per stream) on the device.
 * `opts` may be NULL (defaults).  The generator must be initialised with
 * rng_init before the first rng_generate. */
int rng_create(uint64_t streams, uint64_t seed, const rng_opts *opts,
               rng_gen **out, rng_err **err);

/* Section 5, init kernel (Listing S4): state of stream g := hash of
 * (g0 + g) and the seed; position := 0.  With fuse_init (the default) no
 * kernel runs here: the next generation launch hashes the ids in registers
 * (the init values are iteration 0, so nothing is stored twice).  Otherwise
 * the separate init kernel runs, ordered on the compute stream; the call
 * returns before the device work completes.  Calling it again restarts the
 * streams. */
int rng_init(rng_gen *g, rng_err **err);

/* Section 5, rng kernel (Listing S5) plus the device-side double buffer:
 * emits iterations p .. p+iterations-1 (p = current position, iteration 0
 * being the init value) and then advances p by `iterations`.
 * Exactly one of the two outputs is non-NULL:
 *  - out_dev: caller-owned device memory of at least 8*streams*iterations
 *    bytes, 8-byte aligned (shapes with few values per thread use 16- or
 *    32-byte stores when rows are aligned to them);
 *    value (it - p) * streams + g.  Ordered on the compute stream; returns
 *    before the kernel completes.
 *  - out_host: caller-owned host memory of 8*streams*iterations bytes in
 *    the same layout.  Double-buffer path (Section 5): values are produced
 *    in two device buffers that alternate (generation into one while the
 *    other is copied to the host on a separate copy stream, ordered by CUDA
 *    events); page-locked memory is written directly by the copy engine,
 *    pageable memory goes through the library's pinned staging slots.
 *    Direct path: the kernel stores the values into the host memory itself
 *    over the host link, with no device buffer and no copy (see
 *    rng_opts.host_path).  Blocks until every value is in out_host (the
 *    paper's blocking read).
 * iterations == 0 is a no-op.  Errors: RNG_EINVAL (both or neither output,
 * size overflow), RNG_ESTATE (not initialised), RNG_ENOMEM (device buffers
 * or staging slots could not be allocated), RNG_ECUDA.  A host-output call
 * that fails part-way leaves the streams partly advanced: the generator
 * then refuses further generation with RNG_ESTATE until rng_init. */
int rng_generate(rng_gen *g, uint64_t iterations, uint64_t *out_dev,
                 uint64_t *out_host, rng_err **err);

/* Like rng_generate with device output, but into a ring of `ring_rows`
 * rows (ring_dev: caller-owned device memory of 8*streams*ring_rows bytes):
 * iteration p+i goes to row i mod ring_rows, so rows are overwritten within
 * the call and the ring ends up holding the last min(iterations, ring_rows)
 * iterations.  For consumers that only need the most recent rows, and for
 * measuring generation over more iterations than fit in memory.  One kernel
 * launch; ordered on the compute stream. */
int rng_generate_ring(rng_gen *g, uint64_t iterations, uint64_t *ring_dev,
                      uint64_t ring_rows, rng_err **err);

/* Host consumer ("out" block of Section 5).  Called on a library thread
 * once per chunk of finished values, in order unless rng_opts.host_consumers
 * is above 1 (then concurrently from that many threads, in any order):
 * `values` holds `rows`
 * consecutive iterations starting at absolute iteration `first_iteration`,
 * each row covering streams first_stream .. first_stream+n_streams-1
 * (relative to this generator), rows `row_pitch` values apart.  The
 * memory is a pinned staging slot, valid only during the call.  A
 * non-zero return stops the run with RNG_ESINK. */
typedef int (*rng_sink_fn)(void *user, uint64_t first_iteration, uint64_t rows,
                           uint64_t first_stream, uint64_t n_streams,
                           uint64_t row_pitch, const uint64_t *values);

/* Like rng_generate with host output, but hands each chunk to `sink`
 * instead of a caller buffer (streams of any length, e.g. to a pipe).
 * Blocks until the last chunk has been consumed. */
int rng_generate_sink(rng_gen *g, uint64_t iterations, rng_sink_fn sink,
                      void *user, rng_err **err);

/* The paper's program output (Section 5: raw binary values to stdout, for
 * piping to a consumer such as a statistical test suite): streams
 * `iterations` rows, in order, to the file descriptor `fd` (e.g. 1 for
 * stdout) as native-endian uint64 values, through the double buffer and the
 * pinned staging slots, a library thread writing one slot while the next is
 * filled (the host-side dual buffer the paper names as an improvement).
 * Blocks until everything is written; RNG_ESINK if a write fails. */
int rng_generate_fd(rng_gen *g, uint64_t iterations, int fd, rng_err **err);

/* Timing of the host side of the last call that went through the double
 * buffer (rng_generate with host output on the double-buffer path,
 * rng_generate_sink, rng_generate_fd, rng_generate_host_checksum): which
 * stage bounds the pipeline.  A large producer_wait_s means the consumers
 * are behind (every slot held); a large copy_wait_s means the consumers
 * wait for the link.  Zero consumers and slots: the destination was
 * page-locked and the copies went straight into it. */
typedef struct rng_host_stats {
    uint64_t chunks;          /* device-buffer chunks streamed */
    uint32_t consumers;       /* host consumer threads */
    uint32_t slots;           /* pinned staging slots */
    double wall_s;            /* the call, from its first launch to its end */
    double producer_wait_s;   /* issuing thread waiting for a free slot */
    double copy_wait_s;       /* consumers waiting for their slot's copy,
                                 summed over the consumer threads */
    double consume_s;         /* consumers copying, folding or in the sink,
                                 summed over the consumer threads */
} rng_host_stats;

/* Copies the host-side timing of g's last double-buffer call into *out.
 * RNG_EINVAL for NULL arguments. */
int rng_host_stats_get(const rng_gen *g, rng_host_stats *out);

/* Host-side check of streamed output (the consumer of the paper's streaming
 * program, Section 5, "out" block): streams iterations p .. p+iterations-1
 * over the host link through the double buffer and the pinned staging slots,
 * and the host consumer threads (rng_opts.host_consumers) fold every row
 * into its XOR (row_xor_host[it-p]) and wrapping sum modulo 2^64
 * (row_sum_host[it-p]) over all streams, releasing each slot as soon as it
 * is folded; the values themselves are not kept.  Both arrays are
 * caller-owned host memory of `iterations` uint64 words; the call clears
 * them first and blocks until every row is folded.  Same values as
 * rng_generate_checksum, computed on the host after the link instead of on
 * the device.  Errors as rng_generate with host output. */
int rng_generate_host_checksum(rng_gen *g, uint64_t iterations, uint64_t *row_xor_host,
                               uint64_t *row_sum_host, rng_err **err);

/* Generate-and-checksum mode: advances the streams through iterations
 * p .. p+iterations-1 without storing the values and writes, for each
 * iteration, the XOR (row_xor_dev[it-p]) and the wrapping sum modulo 2^64
 * (row_sum_dev[it-p]) of that iteration's values over all streams.  Both
 * arrays are caller-owned device memory of `iterations` uint64 words; the
 * call clears them first.  Ordered on the compute stream. */
int rng_generate_checksum(rng_gen *g, uint64_t iterations, uint64_t *row_xor_dev,
                          uint64_t *row_sum_dev, rng_err **err);

/* Jump-ahead: advances every stream by `iterations` iterations without
 * producing them (position p += iterations, modulo 2^64).  The update of
 * Listing S5 is linear over GF(2), so k iterations are one multiplication by
 * the k-th power of its 64x64 bit matrix, computed on the host by repeated
 * squaring and applied by one kernel (64 conditional XORs per stream).  The
 * update has period 2^64 - 1: skipping that many returns every stream to its
 * current state.  For resuming a run, checkpoints, and splitting a run by
 * iterations across callers.  Ordered on the compute stream. */
int rng_skip(rng_gen *g, uint64_t iterations, rng_err **err);

/* Current position p (next iteration to be emitted) and stream count. */
int rng_position(const rng_gen *g, uint64_t *position);
int rng_streams(const rng_gen *g, uint64_t *streams);
/* Copies the current states (s_p of each stream) to host memory. Blocks. */
int rng_get_state(rng_gen *g, uint64_t *host_states, rng_err **err);
/* Checkpoint restore: loads one state per stream from host memory and sets
 * the position to `position` (the iteration those states emit next), e.g.
 * states saved with rng_get_state.  Leaves the generator initialised.
 * Blocks until the copy is done. */
int rng_set_state(rng_gen *g, const uint64_t *host_states, uint64_t position, rng_err **err);
/* Waits for all work the generator has queued. */
int rng_sync(rng_gen *g, rng_err **err);
/* The compute stream (cudaStream_t) the generator launches on. */
void *rng_compute_stream(rng_gen *g);
/* Register-store launch configuration chosen for `streams` at creation:
 * values per thread, threads per block and blocks of the grid.  A device
 * output may run the bulk-copy row kernel in another shape instead (see
 * store_policy); rng_last_launch reports what a launch ran. */
int rng_launch_config(const rng_gen *g, uint32_t *values_per_thread,
                      uint32_t *block_threads, uint32_t *grid_blocks);

/* What the generator's last row-kernel launch ran (introspection; the paper
 * has no counterpart).  kernel: RNG_KERNEL_REGISTER (each thread stores its
 * values from registers), RNG_KERNEL_STAGED (rows staged in shared memory and
 * stored as line-aligned 16-byte pieces) or RNG_KERNEL_BULK (rows staged in
 * shared memory and written by TMA bulk copies, row_buffers buffers in turn).
 * band_rows: rows per band of a banded launch, else 0.  Set info->struct_size
 * = sizeof(rng_launch_info) first.  RNG_ESTATE before the first launch. */
enum { RNG_KERNEL_REGISTER = 0, RNG_KERNEL_STAGED = 1, RNG_KERNEL_BULK = 2 };
typedef struct rng_launch_info {
    uint32_t struct_size;
    uint32_t kernel;
    uint32_t values_per_thread;
    uint32_t block_threads;
    uint32_t grid_blocks;
    uint32_t row_buffers;
    uint64_t band_rows;
} rng_launch_info;
int rng_last_launch(const rng_gen *g, rng_launch_info *info, rng_err **err);

/* Releases the device state, buffers, streams and events.  NULL-safe. */
void rng_destroy(rng_gen *g);

/* ------------------------------------------------------------------ */
/* Page-locked host memory for host output (Section 5)                 */
/* ------------------------------------------------------------------ */
/* Section 5 reads every generated batch into host memory.  This allocates
 * `bytes` of zero-filled, page-locked host memory (registered with CUDA, so
 * rng_generate's double buffer copies into it directly and its direct path
 * stores into it over the host link) and returns its address in *out.
 * With RNG_HOST_HUGE_PAGES in `flags` the range is aligned to the kernel's
 * transparent huge-page size and asks the kernel for huge pages
 * (MADV_HUGEPAGE); without it, base pages only.  On Grace-Blackwell the
 * GPU's write rate into a large destination depends on these pages: into
 * 64 KiB pages (as cudaHostAlloc returns them) copies of 32 MiB stall
 * intermittently for whichever engine moves the bytes, into 512 MiB huge
 * pages they run at the link rate.  Where the kernel has transparent huge
 * pages disabled the range keeps base pages.  The memory is owned by the
 * caller and released with rng_host_free; every page is faulted in before
 * the call returns, so it blocks for about a second per 32 GiB.  Errors:
 * RNG_EINVAL (NULL out, zero bytes, unknown flags), RNG_ENOMEM (the mapping
 * failed), RNG_ECUDA / RNG_ENOMEM (page-locking failed; nothing is kept). */
#define RNG_HOST_HUGE_PAGES 1u
int rng_host_alloc(size_t bytes, uint32_t flags, void **out, rng_err **err);

/* Releases memory from rng_host_alloc (unregisters and unmaps it).  NULL is
 * a no-op; any other address not returned by rng_host_alloc is RNG_EINVAL. */
int rng_host_free(void *p);

/* ------------------------------------------------------------------ */
/* Profiler (Section 3.3 and the profiling summary of Section 4.1)     */
/* ------------------------------------------------------------------ */
typedef struct rng_prof rng_prof;

/* Sort flags for summaries: by name or by time/duration, optionally
 * descending. */
enum {
    RNG_PROF_SORT_NAME = 0,
    RNG_PROF_SORT_TIME = 1,
    RNG_PROF_SORT_DESC = 0x10
};

/* A stand-alone profiler fed with explicit event intervals (seconds).
 * Host-only: usable without a GPU. */
rng_prof *rng_prof_new(void);
int rng_prof_add(rng_prof *p, const char *queue, const char *name,
                 double start_s, double end_s);
/* Wall time of the profiled region ("Total elapsed time"). */
int rng_prof_set_elapsed(rng_prof *p, double elapsed_s);
/* Aggregates per event name, pairwise overlaps of events on different
 * queues (summed per ordered pair: event that started later, event
 * already running), effective time = total - overlaps, device share =
 * effective / elapsed. */
int rng_prof_calc(rng_prof *p, rng_err **err);
size_t rng_prof_num_aggregates(const rng_prof *p);
int rng_prof_aggregate(const rng_prof *p, size_t index, const char **name,
                       double *abs_s, double *rel_pct);
size_t rng_prof_num_overlaps(const rng_prof *p);
int rng_prof_overlap(const rng_prof *p, size_t index, const char **name1,
                     const char **name2, double *duration_s);
double rng_prof_total(const rng_prof *p);
double rng_prof_effective(const rng_prof *p);
double rng_prof_elapsed(const rng_prof *p);
/* Text summary in the layout of the paper's figure (aggregate table,
 * overlap table, effective/elapsed/device/host lines).  Owned by p. */
const char *rng_prof_summary(rng_prof *p, int agg_sort, int ovl_sort);
/* Table of all events: one line "queue<TAB>start<TAB>end<TAB>name" per
 * event, times in nanoseconds from the first event, ordered by start. */
int rng_prof_export(rng_prof *p, const char *path, rng_err **err);
void rng_prof_destroy(rng_prof *p);

/* The generator's own profiler: every kernel ("INIT_KERNEL",
 * "RNG_KERNEL", "CHECKSUM_KERNEL") on queue "Main" and every device-to-host
 * copy ("READ_BUFFER") on queue "Comms" since creation or the last reset,
 * timed with CUDA events recorded on the stream the work ran on.  Waits for
 * that work.  Owned by g.  NULL on error. */
rng_prof *rng_profiler(rng_gen *g, rng_err **err);
const char *rng_profile_summary(rng_gen *g, int agg_sort, int ovl_sort, rng_err **err);
int rng_profile_export(rng_gen *g, const char *path, rng_err **err);
/* Drops recorded events and restarts the wall clock. */
int rng_profile_reset(rng_gen *g, rng_err **err);
/* Count and summed device time (seconds) of the recorded events with this
 * name.  Waits for them. */
int rng_profile_stat(rng_gen *g, const char *name, uint64_t *count,
                     double *total_s, rng_err **err);

/* ------------------------------------------------------------------ */
/* Batched form: many independent generators in one graph launch       */
/* ------------------------------------------------------------------ */
typedef struct rng_batch rng_batch;

typedef struct rng_batch_opts {
    uint32_t struct_size;
    uint32_t values_per_thread;  /* 1, 2, 4, 6, 8, 12, 16, 24 or 32; 0 = autotune */
    uint32_t block_threads;      /* 0 = 256 */
    uint32_t tune_reps;          /* timed replays per candidate (default 3) */
    void *stream;                /* cudaStream_t; NULL = own stream */
    int32_t device;              /* -1 = current */
    uint32_t mode;               /* work distribution: 0 = autotune (both),
                                    1 = one work unit per block (the hardware
                                    hands units out in order), 2 = persistent
                                    blocks taking units from a device counter */
    uint32_t stores;             /* 0 = autotune (both), 1 = register and
                                    staged stores, 2 = units of at least 16
                                    rows staged in shared memory and written
                                    by TMA bulk copies (shorter units keep the
                                    stores of 1; 0, 4 or 8 values per thread) */
} rng_batch_opts;

void rng_batch_opts_default(rng_batch_opts *opts);

/* `count` independent instances; instance k has streams[k] streams
 * (1 .. 2^32), iterations[k] iterations (>= 1), run seed seeds[k] and
 * writes its iterations 0 .. iterations[k]-1 to outs[k], caller-owned
 * device memory of 8*streams[k]*iterations[k] bytes, in its own
 * iteration-major layout.  Builds the work table, picks the launch shape
 * (autotuned unless fixed in opts) and captures one persistent launch in a
 * CUDA graph.  Output arrays are written during tuning. */
int rng_batch_create(uint32_t count, const uint64_t *streams,
                     const uint64_t *iterations, const uint64_t *seeds,
                     uint64_t *const *outs, const rng_batch_opts *opts,
                     rng_batch **out, rng_err **err);
/* Replays the captured graph on the batch's stream; asynchronous. */
int rng_batch_run(rng_batch *b, rng_err **err);
int rng_batch_sync(rng_batch *b, rng_err **err);
/* Chosen shape -- values per thread, block size, grid, work units, work
 * distribution (1 = one unit per block, 2 = persistent blocks with a
 * counter) -- and the tuned time of one replay (ms; 0 if not tuned). */
int rng_batch_config(const rng_batch *b, uint32_t *values_per_thread,
                     uint32_t *block_threads, uint32_t *grid_blocks,
                     uint64_t *work_units, uint32_t *mode, double *tuned_ms);
/* Store path the batch runs: *stores = 1 (register and staged stores) or 2
 * (bulk copies for units of at least 16 rows, from *row_buffers shared row
 * buffers per block). */
int rng_batch_stores(const rng_batch *b, uint32_t *stores, uint32_t *row_buffers);
void *rng_batch_stream(rng_batch *b);
void rng_batch_destroy(rng_batch *b);

/* ------------------------------------------------------------------ */
/* Batched generation without allocation                               */
/* ------------------------------------------------------------------ */
/* The paper has no counterpart to this entry point.  It is for callers that
 * cannot call cudaMalloc: code inside a framework whose memory pool owns the
 * whole device and forbids allocations beside it, or latency-bound code that
 * cannot pay for an allocation (or the device-wide synchronisation of a
 * cudaFree) on every call.
 *
 * It produces exactly what rng_batch_create + rng_batch_run produce for the
 * same instances (iterations 0 .. iterations[k]-1 of instance k into outs[k],
 * iteration-major), with one launch of the served form's work-list kernel
 * (an instance table, a unit table and a work counter), but it allocates
 * nothing: no cudaMalloc, cudaFree, pinned or host heap memory and no CUDA
 * graph.  Its scratch -- the counter and the two tables -- is one fixed array
 * of RNG_NOALLOC_SCRATCH_BYTES in device global memory that every GPU loading
 * this library holds until the process exits.
 *
 * Limits: at most RNG_NOALLOC_MAX_INSTANCES instances and
 * RNG_NOALLOC_MAX_UNITS work units, one unit per started group of 2048
 * streams of an instance (sum over k of ceil(streams[k] / 2048)); larger
 * batches are rejected with RNG_EINVAL and a message naming the limit,
 * before anything is queued.
 *
 * Arguments are those of rng_batch_create (host arrays of `count` entries;
 * outs[k] caller-owned device memory of 8*streams[k]*iterations[k] bytes,
 * 8-byte aligned); `stream` is the cudaStream_t to launch on (NULL = the
 * legacy default stream).  The call queues a table upload, a reset of the
 * counter and the kernel on `stream` and returns without waiting for the
 * kernel.  The tables are uploaded from pageable host memory, so the call
 * may wait for work already queued on `stream` before it returns.
 *
 * The first call on a device, with that device current, looks up the
 * scratch array's device address (cudaGetSymbolAddress) and caches it; this
 * may make the driver load the library's device code.  Make that first call
 * before any stream capture begins.  A cudaDeviceReset destroys the array with
 * the context, so do not call this entry point again on a device after
 * resetting it in the same process.  All calls share the one array and each
 * call overwrites it, so calls whose work overlaps on the GPU (launched on
 * different streams without ordering between them) race and produce wrong
 * output; calls on one stream are ordered and safe.  The host side of
 * concurrent calls is serialised by a lock. */
#define RNG_NOALLOC_MAX_INSTANCES 4096u
#define RNG_NOALLOC_MAX_UNITS 262144u
#define RNG_NOALLOC_SCRATCH_BYTES \
    (256u + RNG_NOALLOC_MAX_INSTANCES * 48u + RNG_NOALLOC_MAX_UNITS * 16u)
int rng_batch_generate_noalloc(uint32_t count, const uint64_t *streams,
                               const uint64_t *iterations, const uint64_t *seeds,
                               uint64_t *const *outs, void *stream, rng_err **err);

/* ------------------------------------------------------------------ */
/* Served form: continuous batching of generation requests             */
/* ------------------------------------------------------------------ */
/* A request asks for iterations 0 .. iterations-1 (iteration-major, the
 * layout of Section 5) of a generator with `streams` streams and run seed
 * `seed`.  A scheduler thread admits queued requests in arrival order while
 * the device-memory budget (outputs plus states) and the slot count allow,
 * and launches steps: one work-list kernel per step covering the next rows
 * of every admitted request, so requests that arrive while others run join
 * the next step.  Requests larger than one step's quantum continue over
 * several steps from their device-resident states.  Every result is
 * identical to the same request served alone. */
typedef struct rng_server rng_server;

typedef struct rng_server_opts {
    uint32_t struct_size;
    uint32_t max_active;          /* requests admitted at once; default 1024 */
    uint64_t hbm_budget_bytes;    /* device arena for outputs and states; default 64 GiB */
    uint64_t step_bytes;          /* output bytes one step aims to produce; default 2 GiB */
    uint32_t max_steps_in_flight; /* launched, unfinished steps; default 2 */
    uint32_t values_per_thread;   /* 1, 2, 4, 6, 8, 12, 16, 24 or 32; 0 = 4 */
    uint32_t max_units_per_step;  /* work-table capacity per step; default 1<<20 */
    int32_t device;               /* -1 = current */
    void *stream;                 /* cudaStream_t; NULL = own stream */
    uint32_t mode;                /* 1 (default) = one work unit per block,
                                     2 = persistent blocks with a counter.
                                     The defaults (4 values per thread, one
                                     unit per block) gave the lowest p99 over
                                     20 s of the Poisson workload: 1.09 ms,
                                     against 1.24 at 8 per thread with
                                     persistent blocks: a step's kernel must
                                     drain before the next one starts, and
                                     smaller units shorten that tail */
} rng_server_opts;

typedef struct rng_server_stats {
    uint64_t submitted, completed, rejected, released;
    uint64_t steps, bytes_generated;
    uint64_t pending, active, bytes_in_use, peak_bytes_in_use, peak_active;
} rng_server_stats;

void rng_server_opts_default(rng_server_opts *opts);
/* Allocates the arena (one device allocation of hbm_budget_bytes) and
 * starts the scheduler thread. */
int rng_server_create(const rng_server_opts *opts, rng_server **out, rng_err **err);
/* Queues a request; non-blocking.  *ticket identifies it (>= 1).
 * RNG_EBUDGET if 8*streams*(iterations+1) bytes exceed the whole budget,
 * RNG_EINVAL for sizes out of range (1 <= streams <= 2^32, iterations >= 1),
 * or the scheduler's error if it has failed. */
int rng_server_submit(rng_server *s, uint64_t seed, uint64_t streams, uint64_t iterations,
                      uint64_t *ticket, rng_err **err);
/* Request flags. */
enum {
    RNG_REQ_KEEP_STATE = 1  /* keep the final states resident on the device
                               after completion, for a continuation */
};
/* Like rng_server_submit, with flags and continuation: when
 * continue_ticket != 0 it names a request submitted with
 * RNG_REQ_KEEP_STATE (and not continued before); the new request continues
 * that generator -- same seed and streams (the seed and streams arguments
 * are ignored), iterations starting where it stopped -- from its states
 * kept on the device, so nothing is recomputed or copied.  The continuation
 * is admitted once its parent has completed.  Kept states are freed when the
 * continuation takes them over, or when a request that nobody continues is
 * released. */
int rng_server_submit_ex(rng_server *s, uint64_t seed, uint64_t streams, uint64_t iterations,
                         uint32_t flags, uint64_t continue_ticket, uint64_t *ticket,
                         rng_err **err);
/* Returns up to `max` completed requests not returned before: ticket,
 * device address of its output (8*streams*iterations bytes, owned by the
 * server until released) and latency in seconds (submission to completion
 * seen by the scheduler).  Waits up to timeout_ms for the first one;
 * *n_done = 0 on timeout. */
int rng_server_poll(rng_server *s, uint32_t max, uint64_t *tickets, uint64_t **outs,
                    double *latency_s, uint32_t *n_done, uint32_t timeout_ms, rng_err **err);
/* Copies `count` values starting at value `first` of a completed request's
 * output to host memory (blocking). */
int rng_server_read(rng_server *s, uint64_t ticket, uint64_t first, uint64_t count,
                    uint64_t *host_dst, rng_err **err);
/* Returns a completed request's output memory to the budget. */
int rng_server_release(rng_server *s, uint64_t ticket, rng_err **err);
int rng_server_get_stats(rng_server *s, rng_server_stats *stats);
/* Finishes the steps in flight, drops queued requests, frees the arena.
 * NULL-safe. */
void rng_server_destroy(rng_server *s);

#ifdef __cplusplus
}
#endif

#endif /* PRNG_GB300_RNG_H */
