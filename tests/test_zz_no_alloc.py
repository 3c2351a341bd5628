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


def marshal(N, desc):
    """The workload description as the C structures of include/tp.h."""
    keep = []
    shapes = {"box": N.TP_BOX, "tube": N.TP_TUBE, "sphere": N.TP_SPHERE}
    roles = {"bulk": 0, "detector": 1, "black": 2}
    kinds = {"count": 0, "angular": 1, "psd": 2, "wlx": 3, "multiscat": 4, "dq": 5}
    prims, mirrors = desc["prims"], []
    P = (N.tp_prim * max(1, len(prims)))()
    for i, p in enumerate(prims):
        mi = -1
        if p.get("mirror"):
            mi = len(mirrors)
            mirrors.append(p["mirror"])
        P[i] = N.tp_prim(shapes[p["shape"]], p["axis"], p["material"], roles[p["role"]], mi,
                         int(p["bind_rmin"]), int(p["bind_rmax"]), N.D3(*p["centre"]), N.D3(*p["params"]))
    M = (N.tp_mirror * max(1, len(mirrors)))(*[N.tp_mirror(m["m"], m["R0"], m["Qc"], m["alpha"], m["W"])
                                                for m in mirrors])
    s = desc["source"]
    ap = s.get("aperture")
    src = N.tp_source({"pencil": 0, "rect": 1, "moderator": 2}[s["kind"]], N.D3(*s["centre"]), N.D2(*s["half"]),
                      s["lambda"][0], s["lambda"][1], N.D2(*s["div"]), 1 if ap else 0, N.D2(*(ap or (0.0, 0.0))),
                      float(s.get("slit_z", 0.0)), N.D2(*s.get("slit_half", (0.0, 0.0))),
                      float(s.get("temperature", 0.0)))
    T = (N.tp_tally_desc * max(1, len(desc["tallies"])))()
    for i, t in enumerate(desc["tallies"]):
        T[i] = N.tp_tally_desc(kinds[t["kind"]], 0 if t["trigger"] == "entry" else 1, t["volume"], t["face"],
                               t["scat"], N.I2(*t["bins"]), N.D2(*t["lo"]), N.D2(*t["hi"]),
                               N.D3(*t["origin"]), N.D3(*t["axis"]))
    w = desc["world"]
    d = N.tp_scene_desc(shapes[w["shape"]], N.D3(*w["centre"]), N.D3(*w["params"]), len(prims), P, len(mirrors),
                        M, src, len(desc["tallies"]), T, 1, None, 0, None, 0.0,
                        N.TP_FP64 if desc["precision"] == "f64" else N.TP_FP32, 0)
    mats = (N.tp_material * max(1, len(desc["materials"])))()
    for i, m in enumerate(desc["materials"]):
        br = m.get("bragg")
        if br:
            arrs = [np.ascontiguousarray(br[k], dtype=np.float64) for k in ("d", "mult", "F2")]
            keep += arrs
            mats[i] = N.tp_material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"], len(arrs[0]),
                                    br["V0"], *[a.ctypes.data_as(N.DP) for a in arrs], -1, -1)
        else:
            mats[i] = N.tp_material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"], 0, 1.0,
                                    None, None, None, -1, -1)
    bias = np.ascontiguousarray(desc["bias"], dtype=np.float64).reshape(-1)
    keep += [P, M, T, bias]
    return d, mats, len(desc["materials"]), bias, keep


def run_noalloc(N, desc, n, seed):
    d, mats, nm, bias, keep = marshal(N, desc)
    tb = sum(t["bins"][0] * t["bins"][1] for t in desc["tallies"])
    out_sum = torch.zeros(tb, dtype=torch.float64, device="cuda")
    out_sq = torch.zeros(tb, dtype=torch.float64, device="cuda")
    counts = np.array([n], dtype=np.uint64)
    run = N.tp_run(seed, counts.ctypes.data_as(C.POINTER(C.c_uint64)), None, 0,
                   torch.cuda.current_stream().cuda_stream, 0, 0, None, 0, 0, 0)
    cnt = (C.c_int64 * 8)()
    st = N.lib.tp_run_histories_noalloc(C.byref(d), mats, nm, bias.ctypes.data_as(N.DP) if bias.size else None,
                                        C.byref(run), out_sum.data_ptr(), out_sq.data_ptr(), cnt)
    assert st == N.TP_OK, N.tp_last_error()
    return out_sum.cpu().numpy(), out_sq.cpu().numpy(), list(cnt)


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
        s, s2, c = run_noalloc(N, desc, n, seed=4096)
        assert c[0] == n and c[1] == ref_c["events"], (call, c, ref_c)
        assert np.allclose(s, ref_sum, rtol=1e-9, atol=1e-12), call
        assert np.allclose(s2, ref_sq, rtol=1e-9, atol=1e-12), call


def test_noalloc_rejects_sizes_beyond_its_limits(env):
    engine, N = env
    desc = W.slab(n_histories=10, precision="f64")
    d, mats, nm, bias, keep = marshal(N, desc)
    d.n_instances = 65   # TP_NOALLOC_MAX_INSTANCES + 1
    counts = np.ones(d.n_instances, dtype=np.uint64)
    run = N.tp_run(1, counts.ctypes.data_as(C.POINTER(C.c_uint64)), None, 0, None, 0, 0, None, 0, 0, 0)
    buf = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = N.lib.tp_run_histories_noalloc(C.byref(d), mats, nm, None, C.byref(run), buf.data_ptr(), buf.data_ptr(), None)
    assert st == N.TP_ERR_INVALID_ARG
    assert "64" in N.tp_last_error()
