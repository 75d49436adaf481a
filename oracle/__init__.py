"""CPU oracle for the cf4ocl massive-PRNG example (Section 5, Listings S4/S5).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The GPU library never
imports, links or executes anything in this package, and this package imports
nothing from the library.

``prng_oracle.c`` is the plain definition (hash, xorshift, iteration-major
output, row checksums), compiled with gcc and loaded through ctypes.
``gf2`` is an independent second formulation of the xorshift update as a
64x64 matrix over GF(2).  ``profile`` is the plain profiler arithmetic
(aggregates, overlaps, effective time) of Section 3.3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCE = os.path.join(_HERE, "prng_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

U64 = ctypes.c_uint64
U32 = ctypes.c_uint32
_P64 = ctypes.POINTER(ctypes.c_uint64)


def compile_source(src: str, out: str) -> str:
    """gcc a C oracle source into a shared library at ``out``."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".{os.getpid()}.tmp"
    subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp], check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``prng_oracle.c`` into ``oracle/_build/liboracle.so``."""
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(SOURCE)
    if force or not fresh:
        compile_source(SOURCE, _LIB_PATH)
    return _LIB_PATH


def _ptr(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P64)


class OracleLib:
    """ctypes view of one compiled oracle library (the real one, or a copy
    with a planted mistake in the mutation tests)."""

    def __init__(self, path: str):
        l = ctypes.CDLL(path)
        sig = {
            "oracle_hash_low": ([U32], U32),
            "oracle_hash_high": ([U32], U32),
            "oracle_mix64": ([U64], U64),
            "oracle_seed_key": ([U64], U32),
            "oracle_initial_state": ([U64, U64], U64),
            "oracle_step": ([U64], U64),
            "oracle_step_k": ([U64, U64], U64),
            "oracle_value": ([U64, U64, U64], U64),
            "oracle_generate": ([U64, U64, U64, U64, U64, _P64], ctypes.c_int),
            "oracle_row_checksums": ([U64, U64, U64, U64, U64, _P64, _P64, U64, _P64], ctypes.c_int),
            "oracle_output": ([U64, ctypes.c_int], U64),
            "oracle_value_mode": ([U64, U64, U64, ctypes.c_int], U64),
            "oracle_generate_mode": ([U64, U64, U64, U64, U64, ctypes.c_int, _P64], ctypes.c_int),
            "oracle_row_checksums_mode": ([U64, U64, U64, U64, U64, ctypes.c_int, _P64, _P64, U64, _P64],
                                          ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = res
        self._l = l
        self.path = path

    def hash_low(self, a: int) -> int:
        return int(self._l.oracle_hash_low(a))

    def hash_high(self, a: int) -> int:
        return int(self._l.oracle_hash_high(a))

    def mix64(self, z: int) -> int:
        return int(self._l.oracle_mix64(z))

    def seed_key(self, seed: int) -> int:
        return int(self._l.oracle_seed_key(seed))

    def initial_state(self, g: int, seed: int) -> int:
        return int(self._l.oracle_initial_state(g, seed))

    def step(self, s: int) -> int:
        return int(self._l.oracle_step(s))

    def step_k(self, s: int, k: int) -> int:
        return int(self._l.oracle_step_k(s, k))

    def output(self, s: int, mode: int) -> int:
        """Value emitted for state ``s`` in output mode ``mode`` (0: the state, 1: xorshift64*)."""
        return int(self._l.oracle_output(s, mode))

    def value(self, g: int, seed: int, i: int, output_mode: int = 0) -> int:
        """Output of stream ``g`` at iteration ``i``, computed on its own."""
        if output_mode:
            return int(self._l.oracle_value_mode(g, seed, i, output_mode))
        return int(self._l.oracle_value(g, seed, i))

    def generate(self, n_streams: int, seed: int, iterations: int, *, p0: int = 0,
                 g0: int = 0, output_mode: int = 0) -> np.ndarray:
        """Iterations ``p0 .. p0+T-1`` as a ``(T, N)`` uint64 array (iteration-major)."""
        out = np.empty((iterations, n_streams), dtype=np.uint64)
        if out.size:
            if output_mode:
                rc = self._l.oracle_generate_mode(n_streams, g0, seed, p0, iterations, output_mode, _ptr(out))
            else:
                rc = self._l.oracle_generate(n_streams, g0, seed, p0, iterations, _ptr(out))
            if rc != 0:
                raise MemoryError("oracle_generate: allocation failed")
        return out

    def row_checksums(self, n_streams: int, seed: int, iterations: int, *, p0: int = 0,
                      g0: int = 0, sample_every: int = 0, output_mode: int = 0):
        """Per-iteration (xor, wrapping sum) over all streams, plus every
        ``sample_every``-th row in full (``None`` when ``sample_every`` is 0)."""
        rx = np.zeros(iterations, dtype=np.uint64)
        rs = np.zeros(iterations, dtype=np.uint64)
        samples = None
        sp = None
        if sample_every:
            n_s = (iterations + sample_every - 1) // sample_every
            samples = np.empty((n_s, n_streams), dtype=np.uint64)
            sp = _ptr(samples)
        if iterations:
            if output_mode:
                rc = self._l.oracle_row_checksums_mode(n_streams, g0, seed, p0, iterations, output_mode,
                                                       _ptr(rx), _ptr(rs), sample_every, sp)
            else:
                rc = self._l.oracle_row_checksums(n_streams, g0, seed, p0, iterations, _ptr(rx),
                                                  _ptr(rs), sample_every, sp)
            if rc != 0:
                raise MemoryError("oracle_row_checksums: allocation failed")
        return rx, rs, samples


_default: OracleLib | None = None


def lib() -> OracleLib:
    global _default
    if _default is None:
        _default = OracleLib(build())
    return _default


def hash_low(a): return lib().hash_low(a)
def hash_high(a): return lib().hash_high(a)
def mix64(z): return lib().mix64(z)
def seed_key(seed): return lib().seed_key(seed)
def initial_state(g, seed): return lib().initial_state(g, seed)
def step(s): return lib().step(s)
def step_k(s, k): return lib().step_k(s, k)
def output(s, mode): return lib().output(s, mode)
def value(g, seed, i, output_mode=0): return lib().value(g, seed, i, output_mode)
def generate(n_streams, seed, iterations, **kw): return lib().generate(n_streams, seed, iterations, **kw)
def row_checksums(n_streams, seed, iterations, **kw): return lib().row_checksums(n_streams, seed, iterations, **kw)
