"""ctypes binding of the plain FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It reads the shared
workload descriptions (module `workloads`) and marshals them into the oracle's
own structures; nothing here comes from the CUDA package.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

MAX_PAR = 4
_SHAPES = {"box": 0, "tube": 1, "sphere": 2}
_ROLES = {"bulk": 0, "detector": 1, "black": 2}
_TALLY = {"count": 0, "angular": 1, "psd": 2, "wlx": 3, "multiscat": 4, "dq": 5, "tof": 6}
_PTS = {"entry": 0, "exit": 1}
_PAR = {"radius": 0, "scale": 1, "density": 2}
END_NAMES = ["escaped", "absorbed", "detected", "black", "mirror", "truncated", "aperture", "lost"]
COUNTERS = ["histories", "events", "collisions", "crossings", "truncated", "lost", "mirror_hits",
            "secondaries"]

_build_lock = threading.Lock()


def build(force: bool = False) -> Path:
    """Compile liboracle.so with gcc (plain C11, IEEE arithmetic, no fast-math)."""
    with _build_lock:
        if force or not LIB.exists() or LIB.stat().st_mtime < max(SRC.stat().st_mtime,
                                                                  (HERE / "oracle.h").stat().st_mtime):
            tmp = LIB.with_suffix(f".{os.getpid()}.tmp.so")
            subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                            "-fno-fast-math", "-ffp-contract=off", str(SRC), "-o", str(tmp), "-lm"],
                           check=True)
            os.replace(tmp, LIB)
    return LIB


class Prim(C.Structure):
    _fields_ = [("shape", C.c_int), ("axis", C.c_int), ("material", C.c_int), ("role", C.c_int),
                ("mirror", C.c_int), ("bind_rmin", C.c_int), ("bind_rmax", C.c_int),
                ("chopper", C.c_int), ("c", C.c_double * 3), ("p", C.c_double * 3)]


class Mirror(C.Structure):
    _fields_ = [("m", C.c_double), ("R0", C.c_double), ("Qc", C.c_double),
                ("alpha", C.c_double), ("W", C.c_double)]


class Material(C.Structure):
    _fields_ = [("sig_abs_ref", C.c_double), ("abs_1v", C.c_int), ("sig_inc", C.c_double),
                ("nlines", C.c_int), ("V0", C.c_double), ("d", C.POINTER(C.c_double)),
                ("mult", C.POINTER(C.c_double)), ("F2", C.POINTER(C.c_double)),
                ("density_par", C.c_int), ("scale_par", C.c_int), ("rod", C.c_int)]


class Chopper(C.Structure):
    _fields_ = [("r_black", C.c_double), ("n", C.c_int), ("freq", C.c_double), ("theta0", C.c_double),
                ("phase", C.c_double)]


class Tally(C.Structure):
    _fields_ = [("kind", C.c_int), ("trigger", C.c_int), ("volume", C.c_int), ("face", C.c_int),
                ("scat", C.c_int), ("nb", C.c_int * 2), ("lo", C.c_double * 2),
                ("hi", C.c_double * 2), ("origin", C.c_double * 3), ("axis", C.c_double * 3)]


class Source(C.Structure):
    _fields_ = [("kind", C.c_int), ("c", C.c_double * 3), ("half", C.c_double * 2),
                ("lam_lo", C.c_double), ("lam_hi", C.c_double), ("div", C.c_double * 2),
                ("has_aperture", C.c_int), ("aperture", C.c_double * 2), ("slit_z", C.c_double),
                ("slit_half", C.c_double * 2), ("temperature", C.c_double)]


class Scene(C.Structure):
    _fields_ = [("world_shape", C.c_int), ("world_c", C.c_double * 3), ("world_p", C.c_double * 3),
                ("nprim", C.c_int), ("prims", C.POINTER(Prim)),
                ("nmirror", C.c_int), ("mirrors", C.POINTER(Mirror)),
                ("nchopper", C.c_int), ("choppers", C.POINTER(Chopper)),
                ("nmat", C.c_int), ("mats", C.POINTER(Material)),
                ("bias", C.POINTER(C.c_double)), ("src", Source),
                ("ntally", C.c_int), ("tallies", C.POINTER(Tally)),
                ("npar", C.c_int), ("par_kind", C.POINTER(C.c_int)),
                ("radius_nominal", C.c_double), ("seed", C.c_uint64), ("event_cap", C.c_int)]


class Record(C.Structure):
    _fields_ = [("first_collision", C.c_double * 3), ("dir_after_first", C.c_double * 3),
                ("final_pos", C.c_double * 3),
                ("w_final", C.c_double), ("A_final", C.c_double * MAX_PAR),
                ("nscat", C.c_int), ("nevents", C.c_int), ("end", C.c_int), ("pad", C.c_int)]


class Accum(C.Structure):
    _fields_ = [("sum", C.POINTER(C.c_double)), ("sumsq", C.POINTER(C.c_double)),
                ("J", C.POINTER(C.c_double)), ("J2", C.POINTER(C.c_double)),
                ("counters", C.c_int64 * 8)]


_lib = None


def _load(path) -> C.CDLL:
    L = C.CDLL(str(path))
    dp = C.POINTER(C.c_double)
    L.or_run.argtypes = [C.POINTER(Scene), C.c_int, dp, C.c_uint64, C.c_uint64, C.c_int,
                         C.c_int, C.POINTER(Accum), C.POINTER(Record)]
    L.or_run.restype = C.c_int
    L.or_philox4x32_10.argtypes = [C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                   C.POINTER(C.c_uint32)]
    L.or_u01.argtypes = [C.c_uint32]
    L.or_u01.restype = C.c_double
    L.or_sigma.argtypes = [C.POINTER(Scene), C.c_int, dp, C.c_double, dp]
    L.or_mirror_R.argtypes = [C.POINTER(Mirror), C.c_double]
    L.or_mirror_R.restype = C.c_double
    for fn in ("or_prim_exit", "or_prim_entry"):
        f = getattr(L, fn)
        f.argtypes = [C.POINTER(Scene), C.POINTER(Prim), dp, dp, dp, C.POINTER(C.c_int)]
        f.restype = C.c_double
    L.or_prim_inside.argtypes = [C.POINTER(Scene), C.POINTER(Prim), dp, dp]
    L.or_prim_inside.restype = C.c_int
    L.or_rotate.argtypes = [dp, C.c_double, C.c_double, dp]
    L.or_total_bins.argtypes = [C.POINTER(Scene)]
    L.or_total_bins.restype = C.c_int
    return L


@contextlib.contextmanager
def use_library(path):
    """Run the oracle calls inside the block with another build of oracle.c
    (the tests' planted-mistake copies), then restore the regular one."""
    global _lib
    old = _lib
    _lib = _load(path)
    try:
        yield _lib
    finally:
        _lib = old


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def philox(ctr, key) -> tuple[int, int, int, int]:
    c = (C.c_uint32 * 4)(*[int(x) & 0xffffffff for x in ctr])
    k = (C.c_uint32 * 2)(*[int(x) & 0xffffffff for x in key])
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


def mirror_R(Q, m, R0=0.99, Qc=0.0219, alpha=6.07, W=0.003) -> float:
    mm = Mirror(m, R0, Qc, alpha, W)
    return lib().or_mirror_R(C.byref(mm), float(Q))


def rotate(u, mu, phi):
    uu = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(3)
    lib().or_rotate(_dptr(uu), float(mu), float(phi), _dptr(out))
    return out


class OracleScene:
    """A workload description marshalled into the oracle's structures."""

    def __init__(self, desc: dict):
        self.desc = desc
        self._keep = []
        prims = desc["prims"]
        mirrors, choppers = [], []
        P = (Prim * max(1, len(prims)))()
        for i, p in enumerate(prims):
            mi = ci = -1
            if p.get("mirror"):
                mi = len(mirrors)
                mirrors.append(p["mirror"])
            if p.get("chopper"):
                ci = len(choppers)
                choppers.append(p["chopper"])
            P[i] = Prim(_SHAPES[p["shape"]], p["axis"], p["material"], _ROLES[p["role"]], mi,
                        int(p["bind_rmin"]), int(p["bind_rmax"]), ci,
                        (C.c_double * 3)(*p["centre"]), (C.c_double * 3)(*p["params"]))
        M = (Mirror * max(1, len(mirrors)))()
        for i, m in enumerate(mirrors):
            M[i] = Mirror(m["m"], m["R0"], m["Qc"], m["alpha"], m["W"])
        CH = (Chopper * max(1, len(choppers)))()
        for i, ch in enumerate(choppers):
            CH[i] = Chopper(ch["r_black"], ch["n"], ch["freq"], ch["theta0"], ch["phase"])
        mats = desc["materials"]
        MA = (Material * max(1, len(mats)))()
        for i, m in enumerate(mats):
            br = m.get("bragg")
            if br:
                d = np.ascontiguousarray(br["d"], dtype=np.float64)
                mu = np.ascontiguousarray(br["mult"], dtype=np.float64)
                f2 = np.ascontiguousarray(br["F2"], dtype=np.float64)
                self._keep += [d, mu, f2]
                MA[i] = Material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"],
                                 len(d), br["V0"], _dptr(d), _dptr(mu), _dptr(f2),
                                 m["density_param"], m["scale_param"], int(m.get("rod", False)))
            else:
                MA[i] = Material(m["sigma_abs_ref"], int(m["abs_mode"] == "1/v"), m["sigma_inc"],
                                 0, 1.0, None, None, None, m["density_param"], m["scale_param"],
                                 int(m.get("rod", False)))
        bias = np.ascontiguousarray(desc["bias"], dtype=np.float64).reshape(-1)
        if bias.size == 0:
            bias = np.ones(3)
        self._keep.append(bias)
        src = desc["source"]
        ap = src.get("aperture")
        if src.get("temperature", 0.0) > 0 and src["kind"] != "moderator" and max(src["div"]) > 0:
            raise ValueError("a Maxwellian source with divergence must be a moderator gun")
        S = Source({"pencil": 0, "rect": 1, "moderator": 2}[src["kind"]], (C.c_double * 3)(*src["centre"]),
                   (C.c_double * 2)(*src["half"]), src["lambda"][0], src["lambda"][1],
                   (C.c_double * 2)(*src["div"]), 1 if ap else 0,
                   (C.c_double * 2)(*(ap if ap else (0.0, 0.0))), float(src.get("slit_z", 0.0)),
                   (C.c_double * 2)(*src.get("slit_half", (0.0, 0.0))), float(src.get("temperature", 0.0)))
        tallies = desc["tallies"]
        T = (Tally * max(1, len(tallies)))()
        for i, t in enumerate(tallies):
            T[i] = Tally(_TALLY[t["kind"]], _PTS[t["trigger"]], t["volume"], t["face"], t["scat"],
                         (C.c_int * 2)(*t["bins"]), (C.c_double * 2)(*t["lo"]),
                         (C.c_double * 2)(*t["hi"]), (C.c_double * 3)(*t["origin"]),
                         (C.c_double * 3)(*t["axis"]))
        pk = np.array([_PAR[p["kind"]] for p in desc["params"]] or [0], dtype=np.int32)
        self._keep.append(pk)
        w = desc["world"]
        inst = desc["instances"]
        self.scene = Scene(_SHAPES[w["shape"]], (C.c_double * 3)(*w["centre"]),
                           (C.c_double * 3)(*w["params"]), len(prims), P, len(mirrors), M,
                           len(choppers), CH, len(mats), MA, _dptr(bias), S, len(tallies), T, len(desc["params"]),
                           pk.ctypes.data_as(C.POINTER(C.c_int)),
                           float(inst.get("radius_nominal", 0.0)), desc["seed"] & (2**64 - 1),
                           int(desc["event_cap"]))
        self._keep += [P, M, CH, MA, T]
        self.npar = len(desc["params"])
        self.total_bins = lib().or_total_bins(C.byref(self.scene))
        self.tally_bins = [t["bins"][0] * t["bins"][1] for t in tallies]
        self.tally_off = np.concatenate([[0], np.cumsum(self.tally_bins)]).astype(int)

    # ------------------------------------------------------------------
    def inst_params(self, inst: int) -> np.ndarray:
        p = np.asarray(self.desc["instances"]["params"], dtype=np.float64)
        row = p[inst] if p.shape[1] else np.zeros(0)
        out = np.zeros(MAX_PAR)
        out[:row.size] = row
        return out

    def run(self, n: int | None = None, inst: int = 0, first: int = 0, threads: int | None = None,
            want_grad: bool = False, records: bool = False, params=None) -> dict:
        if n is None:
            n = int(self.desc["instances"]["counts"][inst])
        threads = threads or os.cpu_count() or 1
        tb = self.total_bins
        npar = max(1, self.npar)
        s = np.zeros(tb); s2 = np.zeros(tb)
        J = np.zeros((npar, tb)); J2 = np.zeros((npar, tb))
        acc = Accum(_dptr(s), _dptr(s2), _dptr(J) if want_grad else None,
                    _dptr(J2) if want_grad else None)
        ip = self.inst_params(inst) if params is None else np.pad(
            np.asarray(params, dtype=np.float64), (0, MAX_PAR - len(params)))
        recs = (Record * n)() if records else None
        rc = lib().or_run(C.byref(self.scene), inst, _dptr(ip), first, n, threads, int(want_grad),
                          C.byref(acc), recs)
        if rc != 0:
            raise RuntimeError(f"or_run failed: {rc}")
        out = {"n": n, "sum": s, "sumsq": s2, "counters": dict(zip(COUNTERS, list(acc.counters)))}
        if want_grad:
            out["J"] = J[: self.npar]
            out["J2"] = J2[: self.npar]
        if records:
            out["records"] = records_to_numpy(recs)
        return out

    def sigma(self, mat: int, lam: float, params=None) -> np.ndarray:
        ip = np.zeros(MAX_PAR) if params is None else np.pad(
            np.asarray(params, dtype=np.float64), (0, MAX_PAR - len(params)))
        out = np.zeros(3)
        lib().or_sigma(C.byref(self.scene), mat, _dptr(ip), float(lam), _dptr(out))
        return out

    def _prim_call(self, fn, i, r, u, params=None):
        ip = np.zeros(MAX_PAR) if params is None else np.pad(
            np.asarray(params, dtype=np.float64), (0, MAX_PAR - len(params)))
        rr = np.ascontiguousarray(r, dtype=np.float64)
        uu = np.ascontiguousarray(u, dtype=np.float64)
        face = C.c_int(-1)
        t = getattr(lib(), fn)(C.byref(self.scene), C.byref(self.scene.prims[i]), _dptr(ip),
                               _dptr(rr), _dptr(uu), C.byref(face))
        return t, face.value

    def prim_exit(self, i, r, u, params=None):
        return self._prim_call("or_prim_exit", i, r, u, params)

    def prim_entry(self, i, r, u, params=None):
        return self._prim_call("or_prim_entry", i, r, u, params)

    def prim_inside(self, i, r, params=None) -> bool:
        ip = np.zeros(MAX_PAR) if params is None else np.pad(
            np.asarray(params, dtype=np.float64), (0, MAX_PAR - len(params)))
        rr = np.ascontiguousarray(r, dtype=np.float64)
        return bool(lib().or_prim_inside(C.byref(self.scene), C.byref(self.scene.prims[i]),
                                         _dptr(ip), _dptr(rr)))


def records_to_numpy(recs) -> dict:
    n = len(recs)
    raw = np.ctypeslib.as_array(
        (C.c_byte * (n * C.sizeof(Record))).from_address(C.addressof(recs))).copy()
    dt = np.dtype([("first_collision", "f8", 3), ("dir_after_first", "f8", 3),
                   ("final_pos", "f8", 3), ("w_final", "f8"),
                   ("A_final", "f8", MAX_PAR), ("nscat", "i4"), ("nevents", "i4"), ("end", "i4"),
                   ("pad", "i4")])
    arr = raw.view(dt)
    return {k: arr[k].copy() for k in dt.names if k != "pad"}


def tally_stats(sum_, sumsq, n):
    """Per-bin mean and standard error of the mean per source history."""
    sum_ = np.asarray(sum_, dtype=np.float64)
    sumsq = np.asarray(sumsq, dtype=np.float64)
    mean = sum_ / n
    var = np.maximum(sumsq / n - mean * mean, 0.0)
    return mean, np.sqrt(var / max(n - 1, 1))
