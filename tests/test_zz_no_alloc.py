"""The allocation-free run, tp_run_histories_noalloc, called through the C ABI.

It serves callers that cannot call cudaMalloc (their device memory belongs
to another allocator, or new allocations are not allowed where they run): it
takes the scene as a description and keeps its scratch in a fixed device
array inside the library.  Its sums must equal those of the regular entry
point (tp_create_scene + tp_run_histories) on the same histories, call after
call, since each call reuses the array the previous one left behind.

This file is named so that pytest collects it last."""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as G
    G.build()
    from paper_2304_06226_gb300 import engine, native
    return engine, native


def marshal(engine, desc):
    """The workload description as the C structures of include/tp.h."""
    d, keep = engine.scene_struct(desc)
    mats, mkeep = engine.material_structs(desc["materials"])
    bias = np.ascontiguousarray(desc["bias"], dtype=np.float64).reshape(-1)
    return d, mats, len(desc["materials"]), bias, keep + mkeep + [bias]


def call_noalloc(engine, N, desc, n, seed, counters=True, kernel=0, stage=0):
    """One call; returns (status, sums, squares, counters or None)."""
    d, mats, nm, bias, keep = marshal(engine, desc)
    tb = sum(t["bins"][0] * t["bins"][1] for t in desc["tallies"])
    out_sum = torch.zeros(tb, dtype=torch.float64, device="cuda")
    out_sq = torch.zeros(tb, dtype=torch.float64, device="cuda")
    counts = np.array([n], dtype=np.uint64)
    run = N.tp_run(seed, counts.ctypes.data_as(C.POINTER(C.c_uint64)), None, 0,
                   torch.cuda.current_stream().cuda_stream, 0, 0, None, 0, kernel, 0, 0, 0, stage)
    cnt = (C.c_int64 * 8)() if counters else None
    st = N.lib.tp_run_histories_noalloc(C.byref(d), mats, nm, bias.ctypes.data_as(N.DP) if bias.size else None,
                                        C.byref(run), out_sum.data_ptr(), out_sq.data_ptr(), cnt)
    return st, out_sum.cpu().numpy(), out_sq.cpu().numpy(), (list(cnt) if counters else None)


def run_noalloc(engine, N, desc, n, seed, counters=True):
    st, s, s2, c = call_noalloc(engine, N, desc, n, seed, counters)
    assert st == N.TP_OK, N.tp_last_error()
    return s, s2, c


def run_regular(engine, desc, n, seed):
    sc = engine.Scene(desc)
    sc.run(n, seed=seed)
    torch.cuda.synchronize()
    raw = sc.raw(0)
    c = sc.counters()
    sc.close()
    return raw["sum"], raw["sumsq"], c


@pytest.mark.parametrize("name", ["slab_f64", "powder_f32"])
def test_noalloc_matches_regular_entry_point_on_two_calls_in_a_row(env, name):
    engine, N = env
    if name == "slab_f64":
        n, desc = 40_000, W.slab(g=3.0, n_histories=40_000, precision="f64")
    else:
        n, desc = 400_000, W.powder(n_histories=400_000)
    ref_sum, ref_sq, ref_c = run_regular(engine, desc, n, seed=4096)
    for call in range(2):
        s, s2, c = run_noalloc(engine, N, desc, n, seed=4096)
        assert c[0] == n and c[1] == ref_c["events"], (call, c, ref_c)
        assert np.allclose(s, ref_sum, rtol=1e-9, atol=1e-12), call
        assert np.allclose(s2, ref_sq, rtol=1e-9, atol=1e-12), call


def test_noalloc_without_counters_matches_regular_entry_point(env):
    engine, N = env
    n, desc = 200_000, W.powder(n_histories=200_000)
    ref_sum, ref_sq, _ = run_regular(engine, desc, n, seed=77)
    s, s2, c = run_noalloc(engine, N, desc, n, seed=77, counters=False)
    assert c is None
    assert np.allclose(s, ref_sum, rtol=1e-9, atol=1e-12)
    assert np.allclose(s2, ref_sq, rtol=1e-9, atol=1e-12)


def test_noalloc_reports_a_device_wait_that_gave_up_without_counters(env):
    """The status word is read whether or not counters are asked for."""
    engine, N = env
    desc = W.powder(n_histories=100_000)
    N.tp_set_test_flags(None, N.TP_TEST_SKIP_TABLE_COPY)
    try:
        st, s, _, _ = call_noalloc(engine, N, desc, 100_000, seed=5, counters=False)
    finally:
        N.tp_set_test_flags(None, 0)
    assert st == N.TP_ERR_TIMEOUT, (st, N.tp_last_error())
    assert s.sum() == 0.0
    # and the next call is a normal one
    st, s, _, c = call_noalloc(engine, N, desc, 100_000, seed=5)
    assert st == N.TP_OK and c[0] == 100_000


def test_noalloc_rejects_other_kernels_and_large_tables(env):
    engine, N = env
    desc = W.powder(n_histories=1000)
    st, *_ = call_noalloc(engine, N, desc, 1000, seed=1, kernel=N.TP_KERNEL_EVENT)
    assert st == N.TP_ERR_INVALID_ARG and "history kernel" in N.tp_last_error()
    st, *_ = call_noalloc(engine, N, desc, 1000, seed=1, stage=2)   # tables read from device memory
    assert st == N.TP_ERR_INVALID_ARG and "unstaged" in N.tp_last_error()
    big = W.imaging(n_histories=1000)      # 1000 primitives: tables above 64 KiB
    st, *_ = call_noalloc(engine, N, big, 1000, seed=1)
    assert st == N.TP_ERR_INVALID_ARG, N.tp_last_error()
    assert "at most 65536" in N.tp_last_error()


def test_noalloc_rejects_sizes_beyond_its_limits(env):
    engine, N = env
    desc = W.slab(n_histories=10, precision="f64")
    d, mats, nm, bias, keep = marshal(engine, desc)
    d.n_instances = 65   # TP_NOALLOC_MAX_INSTANCES + 1
    counts = np.ones(d.n_instances, dtype=np.uint64)
    run = N.tp_run(1, counts.ctypes.data_as(C.POINTER(C.c_uint64)), None, 0, None, 0, 0, None, 0, 0, 0)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = N.lib.tp_run_histories_noalloc(C.byref(d), mats, nm, None, C.byref(run), buf.data_ptr(), buf.data_ptr(), None)
    assert st == N.TP_ERR_INVALID_ARG
    assert "64" in N.tp_last_error()
