"""High-level use of the C ABI from Python with PyTorch device memory and streams.

`Scene` marshals a workload description (module `workloads`) into the tp_*
structures and owns the library handle; `TransportFn` is the
torch.autograd.Function whose forward runs the histories and whose backward
calls tp_backward.  Nothing here computes transport: it moves arguments."""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import native as N

_SHAPES = {"box": N.TP_BOX, "tube": N.TP_TUBE, "sphere": N.TP_SPHERE}
_ROLES = {"bulk": N.TP_ROLE_BULK, "detector": N.TP_ROLE_DETECTOR, "black": N.TP_ROLE_BLACK}
_TALLY = {"count": N.TP_TALLY_COUNT, "angular": N.TP_TALLY_ANGULAR, "psd": N.TP_TALLY_PSD,
          "wlx": N.TP_TALLY_WLX, "multiscat": N.TP_TALLY_MULTISCAT, "dq": N.TP_TALLY_DQ,
          "tof": N.TP_TALLY_TOF}
_PTS = {"entry": N.TP_PTS_ENTRY, "exit": N.TP_PTS_EXIT}
_PAR = {"radius": N.TP_PAR_RADIUS, "scale": N.TP_PAR_SCALE, "density": N.TP_PAR_DENSITY}


_SRC = {"pencil": N.TP_SRC_PENCIL, "rect": N.TP_SRC_RECT, "moderator": N.TP_SRC_MODERATOR}


def source_struct(src: dict) -> N.tp_source:
    ap = src.get("aperture")
    return N.tp_source(_SRC[src["kind"]], N.D3(*src["centre"]), N.D2(*src["half"]), src["lambda"][0],
                       src["lambda"][1], N.D2(*src["div"]), 1 if ap else 0,
                       N.D2(*(ap if ap else (0.0, 0.0))), float(src.get("slit_z", 0.0)),
                       N.D2(*src.get("slit_half", (0.0, 0.0))), float(src.get("temperature", 0.0)))


def scene_struct(desc: dict, precision: str | None = None):
    """The workload description as a tp_scene_desc; returns (desc struct,
    objects to keep alive while it is used)."""
    prims = desc["prims"]
    mirrors, choppers = [], []
    P = (N.tp_prim * max(1, len(prims)))()
    for i, p in enumerate(prims):
        mi = ci = -1
        if p.get("mirror"):
            mi = len(mirrors)
            mirrors.append(p["mirror"])
        if p.get("chopper"):
            ci = len(choppers)
            choppers.append(p["chopper"])
        P[i] = N.tp_prim(shape=_SHAPES[p["shape"]], axis=p["axis"], material=p["material"],
                         role=_ROLES[p["role"]], mirror=mi, bind_rmin=int(p["bind_rmin"]),
                         bind_rmax=int(p["bind_rmax"]), chopper=ci, centre=N.D3(*p["centre"]),
                         params=N.D3(*p["params"]))
    M = (N.tp_mirror * max(1, len(mirrors)))()
    for i, m in enumerate(mirrors):
        M[i] = N.tp_mirror(m["m"], m["R0"], m["Qc"], m["alpha"], m["W"])
    CH = (N.tp_chopper * max(1, len(choppers)))()
    for i, c in enumerate(choppers):
        CH[i] = N.tp_chopper(c["r_black"], c["n"], c["freq"], c["theta0"], c["phase"])
    tallies = desc["tallies"]
    T = (N.tp_tally_desc * max(1, len(tallies)))()
    for i, t in enumerate(tallies):
        T[i] = N.tp_tally_desc(_TALLY[t["kind"]], _PTS[t["trigger"]], t["volume"], t["face"],
                               t["scat"], N.I2(*t["bins"]), N.D2(*t["lo"]), N.D2(*t["hi"]),
                               N.D3(*t["origin"]), N.D3(*t["axis"]))
    inst = desc["instances"]
    params = np.ascontiguousarray(inst["params"], dtype=np.float64)
    n_par = len(desc["params"])
    pk = np.array([_PAR[p["kind"]] for p in desc["params"]] or [0], dtype=np.int32)
    pflat = np.ascontiguousarray(params.reshape(-1)) if n_par else np.zeros(1)
    prec = precision or desc.get("precision", "f32")
    w = desc["world"]
    d = N.tp_scene_desc(world_shape=_SHAPES[w["shape"]], world_centre=N.D3(*w["centre"]),
                        world_params=N.D3(*w["params"]), n_prims=len(prims), prims=P,
                        n_mirrors=len(mirrors), mirrors=M, source=source_struct(desc["source"]),
                        n_tallies=len(tallies), tallies=T, n_instances=int(params.shape[0]),
                        inst_params=pflat.ctypes.data_as(N.DP), n_params=n_par,
                        param_kind=pk.ctypes.data_as(C.POINTER(C.c_int)),
                        radius_nominal=float(inst.get("radius_nominal", 0.0)),
                        precision=N.TP_FP64 if prec == "f64" else N.TP_FP32,
                        event_cap=int(desc.get("event_cap", 0)), n_choppers=len(choppers), choppers=CH)
    return d, [P, M, CH, T, pk, pflat]


def material_structs(mats):
    """tp_material array for a list of material descriptions; returns (array,
    objects to keep alive)."""
    arr, keep = (N.tp_material * max(1, len(mats)))(), []
    for i, m in enumerate(mats):
        br = m.get("bragg")
        if br:
            a = [np.ascontiguousarray(br[k], dtype=np.float64) for k in ("d", "mult", "F2")]
            keep += a
            arr[i] = N.tp_material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"], len(a[0]),
                                   br["V0"], *[x.ctypes.data_as(N.DP) for x in a], m["density_param"],
                                   m["scale_param"])
        else:
            arr[i] = N.tp_material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"], 0, 1.0,
                                   None, None, None, m["density_param"], m["scale_param"])
    return arr, keep


def _stream_handle(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Scene:
    """A scene on the current CUDA device built from a workload description."""

    def __init__(self, desc: dict, precision: str | None = None):
        self.desc = desc
        self._keep = []
        prec = precision or desc.get("precision", "f32")
        d, keep = scene_struct(desc, prec)
        self._keep += keep
        inst = desc["instances"]
        params = np.ascontiguousarray(inst["params"], dtype=np.float64)
        self.n_inst = int(params.shape[0])
        self.n_par = len(desc["params"])
        tallies = desc["tallies"]
        self.handle = N.tp_create_scene(d)
        self.precision = prec
        self.params = params.copy()
        self.tally_bins = [t["bins"][0] * t["bins"][1] for t in tallies]
        self.tally_off = np.concatenate([[0], np.cumsum(self.tally_bins)]).astype(int).tolist()
        self.total_bins = N.tp_total_bins(self.handle)
        self.counts = np.asarray(inst["counts"], dtype=np.int64)
        self.seed = int(desc.get("seed", 4096))
        self.set_materials(desc["materials"])
        bias = np.asarray(desc["bias"], dtype=np.float64).reshape(-1, 3)
        for m in range(bias.shape[0]):
            N.tp_set_bias(self.handle, m, bias[m])

    # ------------------------------------------------------------------
    def set_materials(self, mats) -> None:
        arr, keep = material_structs(mats)
        self._keep += keep
        N.tp_set_materials(self.handle, list(arr)[: len(mats)])

    def set_bias(self, material: int, g) -> None:
        N.tp_set_bias(self.handle, material, g)

    def set_params(self, params) -> None:
        p = np.ascontiguousarray(params, dtype=np.float64).reshape(self.n_inst, self.n_par)
        N.tp_set_params(self.handle, p)
        self.params = p.copy()

    def reset(self) -> None:
        N.tp_reset_tallies(self.handle)

    def run(self, n=None, seed: int | None = None, first=None, want_grad: bool = False, stream=None,
            block_size: int = 0, ctas_per_sm: int = 0, records: torch.Tensor | None = None,
            kernel: int = 0, graph: bool = False, secondaries: int = 0, regroup: int = 0,
            stage: int = 0) -> None:
        """Queue histories on `stream` (default: torch's current stream).  n: per
        instance counts (int for one instance, array for many; default: the
        workload's counts).  secondaries: 0 autotuned, 1 in place, 2 queued for a
        second pass (gradient runs).  regroup: events between regroupings of
        the event kernel (0 = autotuned or 1).  stage (explicit kernel): scene
        tables 0 = in shared memory when they fit, 1 = in shared memory, 2 =
        read from device memory."""
        counts = self.counts if n is None else np.broadcast_to(np.asarray(n, dtype=np.uint64),
                                                               (self.n_inst,))
        cnt = np.ascontiguousarray(counts, dtype=np.uint64)
        fst = None if first is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(first, dtype=np.uint64), (self.n_inst,)))
        self._run_keep = (cnt, fst)
        r = N.tp_run(seed if seed is not None else self.seed,
                     cnt.ctypes.data_as(C.POINTER(C.c_uint64)),
                     None if fst is None else fst.ctypes.data_as(C.POINTER(C.c_uint64)),
                     int(want_grad), _stream_handle(stream), block_size, ctas_per_sm,
                     None if records is None else records.data_ptr(),
                     0 if records is None else records.numel() * records.element_size() // C.sizeof(N.tp_record),
                     kernel, int(graph), int(secondaries), int(regroup), int(stage))
        N.tp_run_histories(self.handle, r)

    def tally(self, t: int, instance: int = 0, device: bool = True):
        nb = self.tally_bins[t]
        if device:
            mean = torch.empty(nb, dtype=torch.float64, device="cuda")
            err = torch.empty(nb, dtype=torch.float64, device="cuda")
            N.tp_read_tallies(self.handle, t, instance, mean.data_ptr(), err.data_ptr(), True)
            torch.cuda.synchronize()
            return mean, err
        mean = np.empty(nb)
        err = np.empty(nb)
        N.tp_read_tallies(self.handle, t, instance, mean.ctypes.data, err.ctypes.data, False)
        return mean, err

    def raw(self, instance: int = 0) -> dict:
        tb = self.total_bins
        out = {k: np.zeros(tb) for k in ("sum", "sumsq")}
        npar = max(1, self.n_par)
        out["J"] = np.zeros((npar, tb))
        out["J2"] = np.zeros((npar, tb))
        N.tp_read_raw(self.handle, instance, out["sum"].ctypes.data, out["sumsq"].ctypes.data,
                      out["J"].ctypes.data if self.n_par else None,
                      out["J2"].ctypes.data if self.n_par else None, False)
        out["J"] = out["J"][: self.n_par]
        out["J2"] = out["J2"][: self.n_par]
        return out

    def allreduce(self, histories_per_instance, group=None) -> None:
        """Sum the accumulators of this scene over the ranks of `group` (each
        rank ran disjoint history ids; histories_per_instance: what this rank
        ran per instance) and load the sums back, so that tallies and the
        backward pass give the statistics of all ranks' histories.  One FP64
        all-reduce (shard.reduce_sums)."""
        from . import shard
        tb, ni, npar = self.total_bins, self.n_inst, self.n_par
        parts = {"sum": torch.empty(ni, tb, dtype=torch.float64, device="cuda"),
                 "sumsq": torch.empty(ni, tb, dtype=torch.float64, device="cuda"),
                 "n": torch.as_tensor(np.broadcast_to(np.asarray(histories_per_instance, dtype=np.float64),
                                                      (ni,)).copy(), device="cuda")}
        if npar:
            parts["J"] = torch.empty(ni, npar, tb, dtype=torch.float64, device="cuda")
            parts["J2"] = torch.empty(ni, npar, tb, dtype=torch.float64, device="cuda")
        for q in range(ni):
            N.tp_read_raw(self.handle, q, parts["sum"][q].data_ptr(), parts["sumsq"][q].data_ptr(),
                          parts["J"][q].data_ptr() if npar else None, parts["J2"][q].data_ptr() if npar else None,
                          True)
        shard.reduce_sums(parts, group)
        n = parts["n"].cpu().numpy()
        for q in range(ni):
            N.tp_write_raw(self.handle, q, parts["sum"][q].data_ptr(), parts["sumsq"][q].data_ptr(),
                           parts["J"][q].data_ptr() if npar else None, parts["J2"][q].data_ptr() if npar else None,
                           float(n[q]), True)

    def counters(self) -> dict:
        return N.tp_get_counters(self.handle)

    def status(self) -> tuple[dict, int]:
        """(counters, device status) since the last reset; synchronises."""
        return N.tp_get_counters_status(self.handle)

    def abort(self) -> None:
        """Stop the runs of this scene that are queued or running (tp_abort)."""
        N.tp_abort(self.handle)

    def set_test_flags(self, flags: int) -> None:
        N.tp_set_test_flags(self.handle, flags)

    def launch(self) -> tuple[int, int, int]:
        """(kernel, block size, CTAs per SM) of the last run."""
        return N.tp_get_launch(self.handle)

    def launch_info(self) -> dict:
        """The last run's complete launch configuration (tp_get_launch_info)."""
        return N.tp_get_launch_info(self.handle)

    def launch_count(self) -> int:
        """Transport kernels the last run launched (two per chunk with queued secondaries)."""
        return N.tp_get_launch_count(self.handle)

    def means(self) -> torch.Tensor:
        """Per-instance means of every bin, [n_inst, total_bins] float64 on the GPU."""
        out = torch.empty(self.n_inst, self.total_bins, dtype=torch.float64, device="cuda")
        for q in range(self.n_inst):
            for t in range(len(self.tally_bins)):
                o = self.tally_off[t]
                N.tp_read_tallies(self.handle, t, q, out[q, o:].data_ptr(), None, True)
        return out

    def backward(self, grad: torch.Tensor, stream=None) -> torch.Tensor:
        g = grad.to(device="cuda", dtype=torch.float64).contiguous()
        out = torch.empty(self.n_inst, self.n_par, dtype=torch.float64, device="cuda")
        N.tp_backward(self.handle, g.data_ptr(), out.data_ptr(), True, _stream_handle(stream))
        return out

    def close(self) -> None:
        if getattr(self, "handle", None):
            N.tp_destroy_scene(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def new_records(n: int) -> torch.Tensor:
    """Device buffer for n tp_record, first-collision fields set to NaN."""
    rs = C.sizeof(N.tp_record)
    assert rs % 8 == 0
    buf = torch.zeros(n * rs // 8, dtype=torch.float64, device="cuda")
    v = buf.view(n, rs // 8)
    v[:, 0:6] = math.nan
    return buf


def records_to_numpy(buf: torch.Tensor) -> dict:
    rs = C.sizeof(N.tp_record)
    raw = buf.cpu().numpy().view(np.uint8)
    n = raw.size // rs
    dt = np.dtype([("first_collision", "f8", 3), ("dir_after_first", "f8", 3), ("final_pos", "f8", 3),
                   ("w_final", "f8"), ("A_final", "f8", N.TP_MAX_PARAMS), ("nscat", "i4"),
                   ("nevents", "i4"), ("end", "i4"), ("pad", "i4")])
    assert dt.itemsize == rs
    arr = raw[: n * rs].view(dt)
    return {k: arr[k].copy() for k in dt.names if k != "pad"}


class TransportFn(torch.autograd.Function):
    """Tally means as a differentiable function of the instance parameters.

    forward(params [n_inst, n_par]) sets the parameters, runs the histories with
    the score-function accumulators on, and returns the per-instance means of
    every bin [n_inst, total_bins]; backward contracts the incoming gradient
    with the accumulated derivative tallies (tp_backward)."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, scene: Scene, n=None, seed: int | None = None):
        scene.set_params(params.detach().cpu().numpy())
        scene.reset()
        scene.run(n=n, seed=seed, want_grad=True)
        ctx.scene = scene
        ctx.param_device = params.device
        ctx.param_dtype = params.dtype
        return scene.means()

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        g = ctx.scene.backward(grad_out)
        return g.to(device=ctx.param_device, dtype=ctx.param_dtype), None, None, None
