"""GB300-native massive pseudo-random number generator.

A from-scratch CUDA (sm_103a) implementation of the example application of
"cf4ocl: a C framework for OpenCL" (Section 5): per-stream states seeded by
an integer hash of the stream id, advanced by a 64-bit xorshift, emitted in
the iteration-major layout, either kept on the device or streamed to host
memory through a device-side double buffer, with CUDA-event profiling
(Section 3.3).  The C ABI is ``include/rng.h``; this package only marshals
arguments to it.
"""
from ._capi import RngError, load, library_path  # noqa: F401
from .builder import build  # noqa: F401
from .generator import Generator, Profiler  # noqa: F401
from .batch import Batch  # noqa: F401
from .serve import Server, run_load  # noqa: F401
from .hostmem import host_empty  # noqa: F401


def launch_count() -> int:
    """Kernels (and graph launches) issued by the library in this process."""
    return int(load().rng_launch_count())


def live_objects() -> int:
    return int(load().rng_live_objects())


def shard_range(total_streams: int, rank: int, world_size: int):
    """Contiguous block of stream ids for ``rank`` of ``world_size`` (the
    streams are independent, so ranks generate disjoint column blocks of one
    larger generator with no data exchange).  Returns (first_id, count)."""
    base, extra = divmod(total_streams, world_size)
    first = rank * base + min(rank, extra)
    return first, base + (1 if rank < extra else 0)
