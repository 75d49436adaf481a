"""Page-locked host memory from the library's allocator (rng_host_alloc)."""
from __future__ import annotations

import ctypes
from typing import Sequence, Union

import numpy as np

from . import _capi as C


class _HostBlock:
    """Owns one rng_host_alloc range; numpy views keep it alive through their
    ``base`` and it is released with rng_host_free when the last view dies."""

    def __init__(self, nbytes: int, huge_pages: bool):
        self._lib = C.load()
        p = ctypes.c_void_p()
        C.check(self._lib.rng_host_alloc, ctypes.c_size_t(nbytes),
                C.RNG_HOST_HUGE_PAGES if huge_pages else 0, ctypes.byref(p))
        self.ptr = p.value
        self.nbytes = nbytes
        self.__array_interface__ = {"shape": (nbytes // 8,), "typestr": "<u8", "data": (self.ptr, False),
                                    "version": 3}

    def __del__(self):
        if getattr(self, "ptr", None):
            self._lib.rng_host_free(ctypes.c_void_p(self.ptr))
            self.ptr = None


def host_empty(shape: Union[int, Sequence[int]], huge_pages: bool = True) -> np.ndarray:
    """A uint64 array of ``shape`` in zero-filled, page-locked host memory
    (``rng_host_alloc``), backed by transparent huge pages unless
    ``huge_pages`` is False; a destination for ``Generator.generate_to_host``.
    The memory is released when the array and every view of it are gone."""
    shape = (int(shape),) if np.isscalar(shape) else tuple(int(x) for x in shape)
    n = int(np.prod(shape))
    if n <= 0:
        raise ValueError("host_empty: the array must hold at least one value")
    return np.asarray(_HostBlock(8 * n, huge_pages)).reshape(shape)
