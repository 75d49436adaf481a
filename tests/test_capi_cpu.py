"""The C-ABI library on a machine without a GPU: it loads, exports every
declared symbol, rejects bad arguments with status codes (no exit, no
crash), and its host-only profiler reproduces the paper's summary."""
import ctypes
import os
import random
import re

import pytest

import paper_1609_01257_gb300 as lib
from paper_1609_01257_gb300 import _capi as C
from oracle import profile as oprof
from tests import golden_profile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "rng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(rng_[a-z_0-9]+)\s*\(", src))
    names.discard("rng_sink_fn")
    return names


@pytest.fixture(scope="module")
def L():
    lib.build()
    return lib.load()


def test_every_declared_symbol_is_exported(L):
    declared = _declared_functions()
    assert len(declared) >= 40
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(C.SIGNATURES), declared ^ set(C.SIGNATURES)


def test_strerror_and_counters(L):
    for code in range(8):
        assert L.rng_strerror(code)
    assert L.rng_strerror(99) == b"unknown status"
    assert L.rng_live_objects() >= 0


def test_bad_arguments_return_status_not_crash(L):
    err = ctypes.POINTER(C.RngErr)()
    h = ctypes.c_void_p()
    rc = L.rng_create(0, 1, None, ctypes.byref(h), ctypes.byref(err))
    assert rc == C.RNG_EINVAL and err and b"streams" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))
    assert not err
    rc = L.rng_create((1 << 32) + 1, 1, None, ctypes.byref(h), None)
    assert rc == C.RNG_EINVAL
    o = C.RngOpts()
    L.rng_opts_default(ctypes.byref(o))
    o.values_per_thread = 9  # not a compiled shape
    assert L.rng_create(16, 1, ctypes.byref(o), ctypes.byref(h), None) == C.RNG_EINVAL
    o.values_per_thread = 0
    o.struct_size = 4
    assert L.rng_create(16, 1, ctypes.byref(o), ctypes.byref(h), None) == C.RNG_EINVAL
    assert L.rng_init(None, None) == C.RNG_EINVAL
    assert L.rng_generate(None, 1, None, None, None) == C.RNG_EINVAL
    L.rng_destroy(None)
    L.rng_batch_destroy(None)
    L.rng_prof_destroy(None)
    assert L.rng_batch_create(0, None, None, None, None, None, ctypes.byref(h), None) == C.RNG_EINVAL


def test_option_structs_match_the_header(L):
    # Each *_opts_default writes sizeof() of the C struct into struct_size; the
    # binding's ctypes layout must have the same size and defaults.
    for cls, fn in [(C.RngOpts, L.rng_opts_default), (C.RngBatchOpts, L.rng_batch_opts_default),
                    (C.RngServerOpts, L.rng_server_opts_default)]:
        o = cls()
        fn(ctypes.byref(o))
        assert o.struct_size == ctypes.sizeof(cls), cls.__name__
    o = C.RngOpts()
    L.rng_opts_default(ctypes.byref(o))
    assert (o.host_slots, o.host_consumers, o.host_path, o.store_policy, o.fuse_init) == (0, 0, 0, 1, 1)
    assert o.output_mode == 0
    assert o.device_buffer_bytes == 32 << 20 and o.profiling == 1 and o.device == -1


def test_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("has a GPU")
    h = ctypes.c_void_p()
    err = ctypes.POINTER(C.RngErr)()
    before = L.rng_live_objects()
    rc = L.rng_create(16, 1, None, ctypes.byref(h), ctypes.byref(err))
    assert rc in (C.RNG_ECUDA, C.RNG_ENOMEM)
    assert not h
    assert L.rng_live_objects() == before
    L.rng_err_clear(ctypes.byref(err))


def test_library_profiler_reproduces_paper_summary(L):
    fx = golden_profile.load()
    p = lib.Profiler()
    for q, n, s, e in golden_profile.synthetic_events(fx):
        p.add(q, n, s, e)
    p.set_elapsed(fx["elapsed"])
    a = p.calc()
    for name, (rel, abs_s) in fx["agg"].items():
        assert a["aggregate"][name][0] == pytest.approx(abs_s, rel=1e-9)
        assert a["aggregate"][name][1] == pytest.approx(rel, abs=2e-3)
    assert a["overlaps"] == {("RNG_KERNEL", "READ_BUFFER"): pytest.approx(fx["overlap_total"], rel=1e-9)}
    assert a["effective"] == pytest.approx(fx["effective"], abs=5e-5)
    s = p.summary()
    # Lines of the printed figure, at its precision.
    assert re.search(r"\| READ_BUFFER\s+\|\s+89\.08\d\d \|\s+6\.6521e\+00 \|", s), s
    assert re.search(r"\| RNG_KERNEL\s+\|\s+10\.918\d \|\s+8\.1531e-01 \|", s), s
    assert re.search(r"\| INIT_KERNEL\s+\|\s+0\.0008 \|\s+6\.2464e-05 \|", s), s
    assert re.search(r"\| RNG_KERNEL\s+\| READ_BUFFER\s+\|\s+1\.5790e-02 \|", s), s
    assert "Time spent in device      : 82.30%" in s
    assert "Time spent in host        : 17.70%" in s
    # Sorted by time, descending: READ first.
    assert s.index("READ_BUFFER") < s.index("RNG_KERNEL") < s.index("INIT_KERNEL")
    p.close()


def test_library_profiler_matches_oracle_on_random_events(L, tmp_path):
    rng = random.Random(5)
    for trial in range(30):
        evs = []
        for q in ("Main", "Comms", "Aux")[: rng.randint(1, 3)]:
            t = rng.random()
            for _ in range(rng.randint(0, 12)):
                d = rng.random() * 0.3
                evs.append((q, rng.choice(["RNG_KERNEL", "READ_BUFFER", "INIT_KERNEL"]), t, t + d))
                t += d + rng.random() * 0.1
        rng.shuffle(evs)
        p = lib.Profiler()
        for e in evs:
            p.add(*e)
        p.set_elapsed(10.0)
        got = p.calc()
        want = oprof.analyse([oprof.Event(*e) for e in evs], 10.0)
        assert set(got["aggregate"]) == set(want.aggregate)
        for k, (a, r) in got["aggregate"].items():
            assert a == pytest.approx(want.aggregate[k], abs=1e-12)
            assert r == pytest.approx(want.relative[k], abs=1e-9)
        assert set(got["overlaps"]) == set(want.overlaps)
        for k, v in got["overlaps"].items():
            assert v == pytest.approx(want.overlaps[k], abs=1e-12)
        assert got["effective"] == pytest.approx(want.effective, abs=1e-12)
        if trial == 0:
            path = tmp_path / "ev.tsv"
            p.export(str(path))
            rows = [l.split("\t") for l in path.read_text().splitlines()]
            assert len(rows) == len(evs)
            starts = [float(r[1]) for r in rows]
            assert starts == sorted(starts)
        p.close()


def test_profiler_rejects_inverted_interval(L):
    p = lib.Profiler()
    with pytest.raises(C.RngError):
        p.add("Main", "X", 2.0, 1.0)
    p.close()


@pytest.mark.parametrize("total,world", [(10, 3), (1 << 22, 2), (7, 7), (5, 8)])
def test_shard_range_partitions(total, world):
    seen = []
    for r in range(world):
        first, count = lib.shard_range(total, r, world)
        seen.extend(range(first, first + count))
    assert seen == list(range(total))


def test_noalloc_rejects_bad_batches_before_any_cuda_call(L):
    # Every check of the allocation-free entry point runs on the host before
    # it looks at a device, so each bad batch fails the same way without a GPU.
    U64 = ctypes.c_uint64

    def call(streams, iterations, outs, count=None):
        k = len(streams) if count is None else count
        n = max(len(streams), 1)
        err = ctypes.POINTER(C.RngErr)()
        rc = L.rng_batch_generate_noalloc(k, (U64 * n)(*streams), (U64 * n)(*iterations), (U64 * n)(*([1] * n)),
                                          (ctypes.c_void_p * n)(*outs), None, ctypes.byref(err))
        msg = err.contents.msg if err else b""
        L.rng_err_clear(ctypes.byref(err))
        return rc, msg

    fake = 1 << 20  # a pointer value that is only range- and alignment-checked, never used
    assert call([], [], [], count=0)[0] == C.RNG_EINVAL
    assert call([16] * 4097, [1] * 4097, [fake] * 4097)[1].find(b"at most 4096") > 0
    assert call([0], [1], [fake])[0] == C.RNG_EINVAL
    assert call([(1 << 32) + 1], [1], [fake])[0] == C.RNG_EINVAL
    assert call([16], [0], [fake])[0] == C.RNG_EINVAL
    assert call([16], [1], [0])[0] == C.RNG_EINVAL                       # NULL output
    assert b"aligned" in call([16], [1], [fake + 4])[1]
    assert b"overflows" in call([1 << 32], [1 << 40], [fake])[1]
    rc, msg = call([1 << 32], [1], [fake])                                # 2^21 units of 2048 streams
    assert rc == C.RNG_EINVAL and b"work units" in msg
    assert L.rng_batch_generate_noalloc(1, None, None, None, None, None, None) == C.RNG_EINVAL


def test_batch_and_server_options_are_checked_on_the_host(L):
    # Option and size checks of the batched and served constructors run
    # before they look at a device: each bad value fails without a GPU and
    # creates no object.
    U64 = ctypes.c_uint64
    before = L.rng_live_objects()
    h = ctypes.c_void_p()
    fake = 1 << 20

    def batch(opts=None, streams=16, iterations=1, out=fake):
        err = ctypes.POINTER(C.RngErr)()
        rc = L.rng_batch_create(1, (U64 * 1)(streams), (U64 * 1)(iterations), (U64 * 1)(1),
                                (ctypes.c_void_p * 1)(out), ctypes.byref(opts) if opts else None,
                                ctypes.byref(h), ctypes.byref(err))
        msg = err.contents.msg if err else b""
        L.rng_err_clear(ctypes.byref(err))
        return rc, msg

    o = C.RngBatchOpts()
    L.rng_batch_opts_default(ctypes.byref(o))
    for field, bad in [("values_per_thread", 3), ("mode", 3), ("block_threads", 128), ("struct_size", 8),
                       ("stores", 3)]:
        b = C.RngBatchOpts()
        ctypes.memmove(ctypes.byref(b), ctypes.byref(o), ctypes.sizeof(o))
        setattr(b, field, bad)
        assert batch(b)[0] == C.RNG_EINVAL, field
    for vpt in (1, 2, 6, 12, 16, 32):  # bulk copies run 4 or 8 values per thread
        b = C.RngBatchOpts()
        ctypes.memmove(ctypes.byref(b), ctypes.byref(o), ctypes.sizeof(o))
        b.stores, b.values_per_thread = 2, vpt
        rc, msg = batch(b)
        assert rc == C.RNG_EINVAL and b"stores" in msg, vpt
    assert batch(streams=0)[0] == C.RNG_EINVAL
    assert batch(streams=(1 << 32) + 1)[0] == C.RNG_EINVAL
    assert batch(iterations=0)[0] == C.RNG_EINVAL
    assert b"aligned" in batch(out=fake + 4)[1]
    assert b"overflows" in batch(streams=1 << 32, iterations=1 << 40)[1]
    assert L.rng_batch_create(1, None, None, None, None, None, None, None) == C.RNG_EINVAL

    s = C.RngServerOpts()
    L.rng_server_opts_default(ctypes.byref(s))
    for field, bad in [("values_per_thread", 3), ("mode", 0), ("mode", 3), ("max_active", 0),
                       ("max_steps_in_flight", 0), ("step_bytes", 0), ("max_units_per_step", 0),
                       ("hbm_budget_bytes", 255), ("struct_size", 8)]:
        b = C.RngServerOpts()
        ctypes.memmove(ctypes.byref(b), ctypes.byref(s), ctypes.sizeof(s))
        setattr(b, field, bad)
        assert L.rng_server_create(ctypes.byref(b), ctypes.byref(h), None) == C.RNG_EINVAL, field
    assert L.rng_server_create(None, None, None) == C.RNG_EINVAL
    assert not h and L.rng_live_objects() == before


@pytest.mark.parametrize("field,bad", [
    ("values_per_thread", 9), ("block_threads", 384), ("device_buffer_bytes", 24), ("device_buffer_bytes", 8),
    ("store_policy", 3), ("host_path", 4), ("host_consumers", 65), ("output_mode", 2), ("store_width", 3),
    ("stream_offset", (1 << 32) - 15),
])
def test_generator_options_are_checked_on_the_host(L, field, bad):
    # rng_create checks every option before it looks at a device.
    o = C.RngOpts()
    L.rng_opts_default(ctypes.byref(o))
    setattr(o, field, bad)
    h = ctypes.c_void_p()
    err = ctypes.POINTER(C.RngErr)()
    before = L.rng_live_objects()
    assert L.rng_create(16, 1, ctypes.byref(o), ctypes.byref(h), ctypes.byref(err)) == C.RNG_EINVAL
    assert err and err.contents.code == C.RNG_EINVAL and b"rng_create" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))
    assert not h and L.rng_live_objects() == before


def test_alternative_output_mode_shapes_are_checked_on_the_host(L):
    o = C.RngOpts()
    L.rng_opts_default(ctypes.byref(o))
    o.output_mode = 1
    h = ctypes.c_void_p()
    for vpt, block in [(6, 0), (12, 0), (8, 128)]:
        o.values_per_thread, o.block_threads = vpt, block
        assert L.rng_create(4096, 1, ctypes.byref(o), ctypes.byref(h), None) == C.RNG_EINVAL, (vpt, block)


def test_bulk_copy_shapes_are_checked_on_the_host(L):
    # store_policy 2 (rows written by TMA bulk copies) is compiled for
    # 256-thread blocks with 4, 8 or 16 values per thread.
    o = C.RngOpts()
    L.rng_opts_default(ctypes.byref(o))
    o.store_policy = 2
    h = ctypes.c_void_p()
    for vpt, block in [(1, 0), (2, 0), (6, 0), (24, 0), (8, 128), (8, 512)]:
        o.values_per_thread, o.block_threads = vpt, block
        assert L.rng_create(4096, 1, ctypes.byref(o), ctypes.byref(h), None) == C.RNG_EINVAL, (vpt, block)
    assert not h


def test_last_launch_rejects_bad_arguments_without_a_gpu(L):
    info = C.RngLaunchInfo()
    info.struct_size = ctypes.sizeof(C.RngLaunchInfo)
    assert L.rng_last_launch(None, ctypes.byref(info), None) == C.RNG_EINVAL
    assert ctypes.sizeof(C.RngLaunchInfo) == 32


def test_host_alloc_rejects_bad_arguments_without_a_gpu(L):
    # Argument checks of the page-locked host allocator come before any
    # mapping or CUDA call; freeing NULL is a no-op and an address the
    # allocator did not return is refused.
    err = ctypes.POINTER(C.RngErr)()
    p = ctypes.c_void_p()
    assert L.rng_host_alloc(16, C.RNG_HOST_HUGE_PAGES, None, ctypes.byref(err)) == C.RNG_EINVAL
    L.rng_err_clear(ctypes.byref(err))
    assert L.rng_host_alloc(0, C.RNG_HOST_HUGE_PAGES, ctypes.byref(p), ctypes.byref(err)) == C.RNG_EINVAL
    assert b"zero bytes" in err.contents.msg and not p
    L.rng_err_clear(ctypes.byref(err))
    assert L.rng_host_alloc(16, 6, ctypes.byref(p), ctypes.byref(err)) == C.RNG_EINVAL
    assert b"flags" in err.contents.msg
    L.rng_err_clear(ctypes.byref(err))
    assert L.rng_host_free(None) == C.RNG_OK
    buf = ctypes.create_string_buffer(64)
    assert L.rng_host_free(ctypes.cast(buf, ctypes.c_void_p)) == C.RNG_EINVAL
