"""Batched form: many independent generators in one CUDA-graph launch."""
from __future__ import annotations

import ctypes
from typing import List, Optional, Sequence

import torch

from . import _capi as C


class Batch:
    """Instances ``(streams[k], iterations[k], seeds[k])``; ``outputs[k]`` is a
    ``(iterations[k], streams[k])`` uint64 CUDA tensor (iteration-major) that
    every ``run()`` fills with iterations 0 .. iterations[k]-1.  Launch shape
    is autotuned over values-per-thread, work distribution (``mode``) and
    store path (``stores``: 1 register and staged stores, 2 TMA bulk copies
    for units of 16+ rows) unless fixed."""

    def __init__(self, streams: Sequence[int], iterations: Sequence[int], seeds: Sequence[int], *,
                 outputs: Optional[List[torch.Tensor]] = None, values_per_thread: int = 0,
                 tune_reps: int = 3, mode: int = 0, stores: int = 0, stream=None,
                 device: Optional[int] = None):
        lib = C.load()
        k = len(streams)
        assert len(iterations) == k and len(seeds) == k and k > 0
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        if outputs is None:
            outputs = [torch.empty((int(t), int(n)), dtype=torch.uint64, device=self.device)
                       for n, t in zip(streams, iterations)]
        self.outputs = outputs
        arr = ctypes.c_uint64 * k
        ptrs = (ctypes.c_void_p * k)(*[o.data_ptr() for o in outputs])
        o = C.RngBatchOpts()
        lib.rng_batch_opts_default(ctypes.byref(o))
        o.values_per_thread = values_per_thread
        o.tune_reps = tune_reps
        o.mode = mode
        o.stores = stores
        if stream is None:
            stream = torch.cuda.Stream(device=self.device)  # pooled by torch, never destroyed
        self._torch_stream = stream
        o.stream = stream.cuda_stream if isinstance(stream, torch.cuda.Stream) else int(stream)
        o.device = -1 if device is None else device
        self._lib = lib
        self._h = ctypes.c_void_p()
        torch.cuda.current_stream(self.device).synchronize()  # outputs allocated before use
        with torch.cuda.device(self.device):
            C.check(lib.rng_batch_create, k, arr(*[int(x) for x in streams]), arr(*[int(x) for x in iterations]),
                    arr(*[int(x) & ((1 << 64) - 1) for x in seeds]), ptrs, ctypes.byref(o), ctypes.byref(self._h))

    def run(self):
        C.check(self._lib.rng_batch_run, self._h)

    def sync(self):
        C.check(self._lib.rng_batch_sync, self._h)

    @property
    def stream(self):
        if isinstance(self._torch_stream, torch.cuda.Stream):
            return self._torch_stream
        return torch.cuda.ExternalStream(self._lib.rng_batch_stream(self._h), device=self.device)

    def config(self):
        v, b, g = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        u, ms, m = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_uint32()
        self._lib.rng_batch_config(self._h, ctypes.byref(v), ctypes.byref(b), ctypes.byref(g), ctypes.byref(u),
                                   ctypes.byref(m), ctypes.byref(ms))
        st, nb = ctypes.c_uint32(), ctypes.c_uint32()
        self._lib.rng_batch_stores(self._h, ctypes.byref(st), ctypes.byref(nb))
        return {"values_per_thread": v.value, "block_threads": b.value, "grid_blocks": g.value,
                "work_units": u.value, "tuned_ms": ms.value, "one_unit_per_block": m.value == 1,
                "stores": "bulk" if st.value == 2 else "register", "row_buffers": nb.value}

    def close(self):
        if self._h:
            self._lib.rng_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
