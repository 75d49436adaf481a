"""Python face of the generator object (Section 5 of the cf4ocl paper).

PyTorch supplies device memory and streams; every value is produced by the
CUDA library behind ``include/rng.h``.
"""
from __future__ import annotations

import ctypes
from typing import Callable, Optional

import numpy as np
import torch

from . import _capi as C


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


class Generator:
    """``streams`` independent xorshift streams seeded by the id hash.

    ``generate(T)`` returns the next ``T`` iterations as a ``(T, streams)``
    uint64 CUDA tensor (iteration-major, value ``[i, g]``); iteration 0 is the
    init value.  ``generate_to_host`` writes the same values into host memory:
    by default the kernel stores them there directly; ``host_path=1`` uses the
    paper's double buffer with copy-engine reads, ``host_path=3`` the double
    buffer with copy-kernel reads, ``host_path=2`` insists on direct stores.
    The keyword options mirror ``rng_opts`` in ``include/rng.h``
    (``output_mode=1``: xorshift64* values of the same states;
    ``host_consumers``: host threads draining the staging slots).
    """

    def __init__(self, streams: int, seed: int = 0, *, values_per_thread: int = 0,
                 fuse_init: bool = True, stream_offset: int = 0,
                 device_buffer_bytes: int = 32 << 20, host_slots: int = 0, host_consumers: int = 0,
                 profiling: bool = True, compute_stream=None, device: Optional[int] = None,
                 store_policy: int = 1, host_wait_ms: int = 0, store_width: int = 0,
                 block_threads: int = 0, grid_blocks: int = 0, host_path: int = 0, output_mode: int = 0,
                 init: bool = True):
        lib = C.load()
        o = C.RngOpts()
        lib.rng_opts_default(ctypes.byref(o))
        o.values_per_thread = values_per_thread
        o.fuse_init = 1 if fuse_init else 0
        o.stream_offset = stream_offset
        o.device_buffer_bytes = device_buffer_bytes
        o.host_slots = host_slots
        o.host_consumers = host_consumers
        o.profiling = 1 if profiling else 0
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if compute_stream is None:
            # A stream from torch's pool: it outlives this object, so tensors
            # that recorded it stay safe to free after close().
            compute_stream = torch.cuda.Stream(device=self.device)
        self._torch_stream = compute_stream
        o.compute_stream = _stream_handle(compute_stream)
        o.device = -1 if device is None else device
        o.store_policy = store_policy
        o.host_wait_ms = host_wait_ms
        o.store_width = store_width
        o.block_threads = block_threads
        o.grid_blocks = grid_blocks
        o.host_path = host_path
        o.output_mode = output_mode
        self._lib = lib
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            C.check(lib.rng_create, streams, seed & ((1 << 64) - 1), ctypes.byref(o), ctypes.byref(self._h))
        self.streams = streams
        self.seed = seed
        if init:
            self.init()

    # -- lifecycle -----------------------------------------------------------
    def close(self):
        if self._h:
            self._lib.rng_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- generation ------------------------------------------------------------
    def init(self):
        C.check(self._lib.rng_init, self._h)

    def skip(self, iterations: int):
        """Advance every stream by ``iterations`` (jump-ahead over GF(2))."""
        C.check(self._lib.rng_skip, self._h, iterations & ((1 << 64) - 1))

    @property
    def position(self) -> int:
        p = ctypes.c_uint64()
        self._lib.rng_position(self._h, ctypes.byref(p))
        return p.value

    @property
    def stream(self):
        """The compute stream the library launches on."""
        if isinstance(self._torch_stream, torch.cuda.Stream):
            return self._torch_stream
        return torch.cuda.ExternalStream(self._lib.rng_compute_stream(self._h), device=self.device)

    def launch_config(self):
        """Register-store shape chosen at creation (values per thread, block,
        grid); ``last_launch()`` reports the kernel a launch actually ran."""
        v, b, g = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        self._lib.rng_launch_config(self._h, ctypes.byref(v), ctypes.byref(b), ctypes.byref(g))
        return v.value, b.value, g.value

    def last_launch(self) -> dict:
        """What the last row-kernel launch ran: kernel ("register", "staged"
        or "bulk"), values per thread, block, grid, bulk row buffers and band
        rows (0 = unbanded)."""
        info = C.RngLaunchInfo()
        info.struct_size = ctypes.sizeof(C.RngLaunchInfo)
        C.check(self._lib.rng_last_launch, self._h, ctypes.byref(info))
        return {"kernel": C.KERNEL_NAMES.get(info.kernel, str(info.kernel)),
                "values_per_thread": info.values_per_thread, "block": info.block_threads,
                "grid": info.grid_blocks, "row_buffers": info.row_buffers, "band_rows": info.band_rows}

    def _after_current(self):
        # The library's work follows what torch's current stream has queued
        # (e.g. the output's allocation) ...
        ev = torch.cuda.Event()
        ev.record(torch.cuda.current_stream(self.device))
        self.stream.wait_event(ev)

    def _before_current(self):
        # ... and torch's current stream waits for it, so that a tensor handed
        # back is ready for whatever the caller queues next (``.cpu()``, ...).
        ev = torch.cuda.Event()
        ev.record(self.stream)
        torch.cuda.current_stream(self.device).wait_event(ev)

    def generate(self, iterations: int, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Next ``iterations`` rows on the device.  Asynchronous for the host:
        the kernel runs on the generator's compute stream, and torch's current
        stream is made to wait for it before the tensor is returned."""
        if out is None:
            out = torch.empty((iterations, self.streams), dtype=torch.uint64, device=self.device)
        assert out.is_cuda and out.is_contiguous() and out.element_size() == 8
        assert out.numel() >= iterations * self.streams
        self._after_current()
        C.check(self._lib.rng_generate, self._h, iterations, ctypes.c_void_p(out.data_ptr()), None)
        out.record_stream(self.stream)
        self._before_current()
        return out

    def generate_to(self, iterations: int, out_ptr: int):
        """Raw form: ``out_ptr`` is a device address of 8*streams*iterations bytes."""
        C.check(self._lib.rng_generate, self._h, iterations, ctypes.c_void_p(out_ptr), None)

    def generate_ring(self, iterations: int, ring: torch.Tensor) -> torch.Tensor:
        """Next ``iterations`` rows into ``ring`` (``(R, streams)`` uint64 CUDA
        tensor), row ``i mod R`` for iteration ``i``; asynchronous."""
        assert ring.is_cuda and ring.is_contiguous() and ring.element_size() == 8
        assert ring.numel() % self.streams == 0 and ring.numel() >= self.streams
        self._after_current()
        C.check(self._lib.rng_generate_ring, self._h, iterations, ctypes.c_void_p(ring.data_ptr()),
                ring.numel() // self.streams)
        ring.record_stream(self.stream)
        self._before_current()
        return ring

    def generate_to_host(self, iterations: int, out=None):
        """Next ``iterations`` rows into host memory (blocks until done).

        ``out`` may be a numpy uint64 array or a CPU tensor (pinned memory is
        written directly by the copy engine)."""
        if out is None:
            out = np.empty((iterations, self.streams), dtype=np.uint64)
        if isinstance(out, torch.Tensor):
            assert out.device.type == "cpu" and out.is_contiguous() and out.element_size() == 8
            ptr = out.data_ptr()
            n = out.numel()
        else:
            assert out.dtype == np.uint64 and out.flags.c_contiguous
            ptr = out.ctypes.data
            n = out.size
        assert n >= iterations * self.streams
        C.check(self._lib.rng_generate, self._h, iterations, None, ctypes.c_void_p(ptr))
        return out

    def generate_sink(self, iterations: int, sink: Callable[[int, np.ndarray, int], Optional[int]]):
        """Streams ``iterations`` rows through the pinned staging slots and
        calls ``sink(first_iteration, block, first_stream)`` per chunk, where
        ``block`` is a ``(rows, n_streams)`` uint64 view valid only during the
        call.  A truthy return value stops the run.  In order, unless the
        generator was made with ``host_consumers`` above 1 (then from that
        many threads, in any order)."""
        failure = []

        def _cb(_user, first_it, rows, first_stream, n_streams, pitch, values):
            try:
                buf = np.ctypeslib.as_array(values, shape=(rows * pitch,))
                block = buf.reshape(rows, pitch)[:, :n_streams]
                r = sink(int(first_it), block, int(first_stream))
                return int(r) if r else 0
            except Exception as e:  # surface Python errors as a sink failure
                failure.append(e)
                return 1

        cb = C.SINK_FN(_cb)
        try:
            C.check(self._lib.rng_generate_sink, self._h, iterations, cb, None)
        except C.RngError:
            if failure:
                raise failure[0]
            raise

    def generate_host_checksum(self, iterations: int):
        """Streams ``iterations`` rows over the host link and folds each row
        on the host into its XOR and wrapping sum (two uint64 numpy arrays);
        the values are not kept."""
        row_xor = np.empty(iterations, dtype=np.uint64)
        row_sum = np.empty(iterations, dtype=np.uint64)
        if iterations:
            C.check(self._lib.rng_generate_host_checksum, self._h, iterations,
                    ctypes.c_void_p(row_xor.ctypes.data), ctypes.c_void_p(row_sum.ctypes.data))
        return row_xor, row_sum

    def host_stats(self) -> dict:
        """Host-side timing of the last double-buffer call: chunks, consumer
        threads, slots, wall time, the issuing thread's wait for free slots,
        the consumers' wait for copies and their consuming time (seconds)."""
        s = C.RngHostStats()
        self._lib.rng_host_stats_get(self._h, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in C.RngHostStats._fields_}

    def generate_fd(self, iterations: int, fd: int):
        """Stream ``iterations`` rows as raw uint64 values to file descriptor ``fd``."""
        C.check(self._lib.rng_generate_fd, self._h, iterations, fd)

    def generate_checksum(self, iterations: int, row_xor: Optional[torch.Tensor] = None,
                          row_sum: Optional[torch.Tensor] = None):
        """Per-iteration XOR and wrapping sum over all streams, without
        storing the values (two uint64 CUDA tensors of length ``iterations``)."""
        if row_xor is None:
            row_xor = torch.empty(iterations, dtype=torch.uint64, device=self.device)
        if row_sum is None:
            row_sum = torch.empty(iterations, dtype=torch.uint64, device=self.device)
        self._after_current()
        C.check(self._lib.rng_generate_checksum, self._h, iterations,
                ctypes.c_void_p(row_xor.data_ptr()), ctypes.c_void_p(row_sum.data_ptr()))
        row_xor.record_stream(self.stream)
        row_sum.record_stream(self.stream)
        self._before_current()
        return row_xor, row_sum

    def state(self) -> np.ndarray:
        out = np.empty(self.streams, dtype=np.uint64)
        C.check(self._lib.rng_get_state, self._h, ctypes.c_void_p(out.ctypes.data))
        return out

    def set_state(self, states: np.ndarray, position: int):
        """Restore a checkpoint: per-stream states (as from ``state()``) and
        the iteration they emit next."""
        states = np.ascontiguousarray(states, dtype=np.uint64)
        assert states.size == self.streams
        C.check(self._lib.rng_set_state, self._h, ctypes.c_void_p(states.ctypes.data), position)

    def sync(self):
        C.check(self._lib.rng_sync, self._h)

    # -- profiling -------------------------------------------------------------
    def profile_summary(self, agg_sort=C.RNG_PROF_SORT_TIME | C.RNG_PROF_SORT_DESC,
                        ovl_sort=C.RNG_PROF_SORT_TIME | C.RNG_PROF_SORT_DESC) -> str:
        err = ctypes.POINTER(C.RngErr)()
        s = self._lib.rng_profile_summary(self._h, agg_sort, ovl_sort, ctypes.byref(err))
        if not s:
            msg = err.contents.msg.decode() if err else "rng_profile_summary failed"
            self._lib.rng_err_clear(ctypes.byref(err))
            raise C.RngError(C.RNG_ECUDA, msg)
        return s.decode()

    def profile_export(self, path: str):
        C.check(self._lib.rng_profile_export, self._h, path.encode())

    def profile_reset(self):
        C.check(self._lib.rng_profile_reset, self._h)

    def profile_stat(self, name: str):
        """(count, summed device seconds) of the recorded events ``name``."""
        n, t = ctypes.c_uint64(), ctypes.c_double()
        C.check(self._lib.rng_profile_stat, self._h, name.encode(), ctypes.byref(n), ctypes.byref(t))
        return n.value, t.value

    def profile(self):
        """Analysed profile: dict with aggregates, overlaps, totals."""
        err = ctypes.POINTER(C.RngErr)()
        p = self._lib.rng_profiler(self._h, ctypes.byref(err))
        if not p:
            msg = err.contents.msg.decode() if err else "rng_profiler failed"
            self._lib.rng_err_clear(ctypes.byref(err))
            raise C.RngError(C.RNG_ECUDA, msg)
        return Profiler._read(self._lib, p)


class Profiler:
    """Stand-alone profiler over explicit intervals (host only)."""

    def __init__(self):
        self._lib = C.load()
        self._h = self._lib.rng_prof_new()
        if not self._h:
            raise MemoryError("rng_prof_new failed")

    def add(self, queue: str, name: str, start_s: float, end_s: float):
        rc = self._lib.rng_prof_add(self._h, queue.encode(), name.encode(), start_s, end_s)
        if rc != C.RNG_OK:
            raise C.RngError(rc, "rng_prof_add rejected the event")

    def set_elapsed(self, s: float):
        self._lib.rng_prof_set_elapsed(self._h, s)

    def calc(self):
        C.check(self._lib.rng_prof_calc, self._h)
        return Profiler._read(self._lib, self._h)

    def summary(self, agg_sort=C.RNG_PROF_SORT_TIME | C.RNG_PROF_SORT_DESC,
                ovl_sort=C.RNG_PROF_SORT_TIME | C.RNG_PROF_SORT_DESC) -> str:
        return self._lib.rng_prof_summary(self._h, agg_sort, ovl_sort).decode()

    def export(self, path: str):
        C.check(self._lib.rng_prof_export, self._h, path.encode())

    def close(self):
        if self._h:
            self._lib.rng_prof_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _read(lib, h):
        aggs = {}
        for i in range(lib.rng_prof_num_aggregates(h)):
            nm, a, r = C.c_cp(), C.c_dbl(), C.c_dbl()
            lib.rng_prof_aggregate(h, i, ctypes.byref(nm), ctypes.byref(a), ctypes.byref(r))
            aggs[nm.value.decode()] = (a.value, r.value)
        ovl = {}
        for i in range(lib.rng_prof_num_overlaps(h)):
            n1, n2, d = C.c_cp(), C.c_cp(), C.c_dbl()
            lib.rng_prof_overlap(h, i, ctypes.byref(n1), ctypes.byref(n2), ctypes.byref(d))
            ovl[(n1.value.decode(), n2.value.decode())] = d.value
        return {
            "aggregate": aggs,
            "overlaps": ovl,
            "total": lib.rng_prof_total(h),
            "effective": lib.rng_prof_effective(h),
            "elapsed": lib.rng_prof_elapsed(h),
        }
