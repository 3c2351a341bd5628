"""Failure detection on the GPU, in forms that fault and hang nothing.

* A bounded device wait that runs out: the test hook TP_TEST_SKIP_TABLE_COPY
  makes every block arm its wait for the bulk copy of the scene tables into
  shared memory without issuing the copy.  Each wait gives up after about half
  a second, the block records TP_ERR_TIMEOUT and returns with nothing in
  flight; tp_get_counters reports the status, no history ran, and the scene
  runs normally again after the flag is cleared and the tallies reset.
* A host-requested stop: tp_abort sets a flag in mapped host memory that the
  kernels poll whenever they claim histories; the run ends early with
  TP_ERR_ABORTED, and tp_reset_tallies makes the scene usable again."""
import time

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


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_table_copy_wait_runs_out_and_is_reported(env, kernel):
    engine, N = env
    sc = engine.Scene(W.powder(n_histories=200_000))
    try:
        sc.set_test_flags(N.TP_TEST_SKIP_TABLE_COPY)
        t0 = time.perf_counter()
        sc.run(200_000, kernel=kernel)
        cnt, st = sc.status()
        waited = time.perf_counter() - t0
        assert st == N.TP_ERR_TIMEOUT, (st, N.tp_last_error())
        assert "scene tables" in N.tp_last_error()
        assert cnt["histories"] == 0 and cnt["events"] == 0, cnt
        assert waited < 30.0
        # the context is usable: clear the hook, reset and run again
        sc.set_test_flags(0)
        sc.reset()
        sc.run(200_000, kernel=kernel)
        cnt, st = sc.status()
        assert st == N.TP_OK, N.tp_last_error()
        assert cnt["histories"] == 200_000
    finally:
        sc.close()


def test_abort_stops_a_running_launch(env):
    engine, N = env
    n = 4_000_000_000        # about a second of work on one GPU
    sc = engine.Scene(W.powder(n_histories=n))
    try:
        stream = torch.cuda.Stream()
        sc.run(n, kernel=3, stream=stream)   # explicit kernel: no autotuning before the launch
        time.sleep(0.05)
        sc.abort()
        stream.synchronize()
        cnt, st = sc.status()
        assert st == N.TP_ERR_ABORTED, (st, N.tp_last_error())
        assert cnt["histories"] < n // 2, cnt
        # aborted scenes stop at once until reset
        sc.run(1_000_000, kernel=3)
        cnt2, st2 = sc.status()
        assert st2 == N.TP_ERR_ABORTED
        assert cnt2["histories"] == cnt["histories"]
        sc.reset()
        sc.run(1_000_000, kernel=3)
        cnt3, st3 = sc.status()
        assert st3 == N.TP_OK and cnt3["histories"] == 1_000_000, (cnt3, N.tp_last_error())
    finally:
        sc.close()


@pytest.mark.parametrize("kernel", [1, 2, 3])
def test_abort_before_the_run_claims_nothing(env, kernel):
    engine, N = env
    sc = engine.Scene(W.slab(g=3.0, n_histories=100_000, precision="f64"))
    try:
        sc.abort()
        sc.run(100_000, kernel=kernel)
        cnt, st = sc.status()
        assert st == N.TP_ERR_ABORTED
        assert cnt["histories"] == 0, cnt
        sc.reset()
        sc.run(100_000, kernel=kernel)
        cnt, st = sc.status()
        assert st == N.TP_OK and cnt["histories"] == 100_000
    finally:
        sc.close()


def test_abort_stops_a_gradient_run_with_queued_secondaries(env):
    engine, N = env
    desc = W.batched()
    sc = engine.Scene(desc)
    try:
        sc.abort()
        sc.run(want_grad=True, kernel=2, secondaries=2)
        cnt, st = sc.status()
        assert st == N.TP_ERR_ABORTED
        assert cnt["histories"] == 0 and cnt["secondaries"] == 0, cnt
        sc.reset()
        small = np.full(sc.n_inst, 2000)
        sc.run(small, want_grad=True, kernel=2, secondaries=2)
        cnt, st = sc.status()
        assert st == N.TP_OK and cnt["histories"] == int(small.sum())
    finally:
        sc.close()
