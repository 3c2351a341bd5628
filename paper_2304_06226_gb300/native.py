"""ctypes binding of libtp.so: the C ABI of include/tp.h under the same names.

Argument marshalling only -- every step of the transport runs in the CUDA
kernels of the library.  Importing this module loads the library and fails
loudly (ImportError) if it has not been built; there is no CPU fallback."""
from __future__ import annotations

import ctypes as C
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "libtp.so"

(TP_OK, TP_ERR_INVALID_ARG, TP_ERR_GEOMETRY, TP_ERR_CUDA, TP_ERR_OOM, TP_ERR_TIMEOUT, TP_ERR_STATE,
 TP_ERR_ABORTED) = range(8)
STATUS_NAMES = ["TP_OK", "TP_ERR_INVALID_ARG", "TP_ERR_GEOMETRY", "TP_ERR_CUDA", "TP_ERR_OOM",
                "TP_ERR_TIMEOUT", "TP_ERR_STATE", "TP_ERR_ABORTED"]
TP_TEST_SKIP_TABLE_COPY = 1
TP_TEST_FULL_BUILD = 2
TP_TEST_SMALL_SEC_QUEUE = 4
TP_BOX, TP_TUBE, TP_SPHERE = 0, 1, 2
TP_ROLE_BULK, TP_ROLE_DETECTOR, TP_ROLE_BLACK = 0, 1, 2
TP_PROC_ABS, TP_PROC_INC, TP_PROC_BRAGG, TP_NPROC = 0, 1, 2, 3
TP_TALLY_COUNT, TP_TALLY_ANGULAR, TP_TALLY_PSD, TP_TALLY_WLX, TP_TALLY_MULTISCAT, TP_TALLY_DQ, TP_TALLY_TOF = range(7)
TP_PTS_ENTRY, TP_PTS_EXIT = 0, 1
TP_PAR_RADIUS, TP_PAR_SCALE, TP_PAR_DENSITY = 0, 1, 2
TP_SRC_PENCIL, TP_SRC_RECT, TP_SRC_MODERATOR = 0, 1, 2
TP_FP32, TP_FP64 = 0, 1
TP_KERNEL_AUTO, TP_KERNEL_HISTORY, TP_KERNEL_EVENT, TP_KERNEL_WARPQ = 0, 1, 2, 3
TP_MAX_PARAMS = 4
TP_MAX_TALLIES = 16
TP_MAX_PRIMS = 16777214
COUNTER_NAMES = ["histories", "events", "collisions", "crossings", "truncated", "lost", "mirror_hits",
                 "secondaries"]
END_NAMES = ["escaped", "absorbed", "detected", "black", "mirror", "truncated", "aperture", "lost"]

D3 = C.c_double * 3
D2 = C.c_double * 2
I2 = C.c_int * 2


class tp_prim(C.Structure):
    _fields_ = [("shape", C.c_int), ("axis", C.c_int), ("material", C.c_int), ("role", C.c_int),
                ("mirror", C.c_int), ("bind_rmin", C.c_int), ("bind_rmax", C.c_int), ("chopper", C.c_int),
                ("centre", D3), ("params", D3)]


class tp_mirror(C.Structure):
    _fields_ = [("m", C.c_double), ("R0", C.c_double), ("Qc", C.c_double), ("alpha", C.c_double),
                ("W", C.c_double)]


class tp_chopper(C.Structure):
    _fields_ = [("r_black", C.c_double), ("n_windows", C.c_int), ("freq", C.c_double),
                ("theta0", C.c_double), ("phase", C.c_double)]


class tp_tally_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("trigger", C.c_int), ("volume", C.c_int), ("face", C.c_int),
                ("scat", C.c_int), ("nbins", I2), ("lo", D2), ("hi", D2), ("origin", D3),
                ("axis", D3)]


class tp_source(C.Structure):
    _fields_ = [("kind", C.c_int), ("centre", D3), ("half", D2), ("lambda_lo", C.c_double),
                ("lambda_hi", C.c_double), ("div", D2), ("has_aperture", C.c_int),
                ("aperture", D2), ("slit_z", C.c_double), ("slit_half", D2),
                ("temperature", C.c_double)]


class tp_scene_desc(C.Structure):
    _fields_ = [("world_shape", C.c_int), ("world_centre", D3), ("world_params", D3),
                ("n_prims", C.c_int), ("prims", C.POINTER(tp_prim)),
                ("n_mirrors", C.c_int), ("mirrors", C.POINTER(tp_mirror)),
                ("source", tp_source),
                ("n_tallies", C.c_int), ("tallies", C.POINTER(tp_tally_desc)),
                ("n_instances", C.c_int), ("inst_params", C.POINTER(C.c_double)),
                ("n_params", C.c_int), ("param_kind", C.POINTER(C.c_int)),
                ("radius_nominal", C.c_double), ("precision", C.c_int), ("event_cap", C.c_int),
                ("n_choppers", C.c_int), ("choppers", C.POINTER(tp_chopper))]


class tp_material(C.Structure):
    _fields_ = [("sigma_abs_ref", C.c_double), ("abs_1v", C.c_int), ("sigma_inc", C.c_double),
                ("n_lines", C.c_int), ("V0", C.c_double), ("d", C.POINTER(C.c_double)),
                ("mult", C.POINTER(C.c_double)), ("F2", C.POINTER(C.c_double)),
                ("density_param", C.c_int), ("scale_param", C.c_int)]


class tp_record(C.Structure):
    _fields_ = [("first_collision", D3), ("dir_after_first", D3), ("final_pos", D3),
                ("w_final", C.c_double), ("A_final", C.c_double * TP_MAX_PARAMS),
                ("nscat", C.c_int), ("nevents", C.c_int), ("end", C.c_int), ("pad", C.c_int)]


class tp_run(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("n_histories", C.POINTER(C.c_uint64)),
                ("first_history", C.POINTER(C.c_uint64)), ("want_grad", C.c_int),
                ("stream", C.c_void_p), ("block_size", C.c_int), ("ctas_per_sm", C.c_int),
                ("records", C.c_void_p), ("n_records", C.c_uint64), ("kernel", C.c_int),
                ("use_graph", C.c_int), ("secondaries", C.c_int), ("regroup", C.c_int),
                ("stage", C.c_int)]


class tp_launch_info(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("kernel", "block_size", "ctas_per_sm", "staged", "registers", "full_build",
                                      "regroup", "queued_secondaries", "launches")]


class tp_peaks(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("fp32_fma", "int32_imad", "int32_logic", "mufu_lg2", "mufu_ex2",
                                         "mufu_sin", "fp64_fma", "atomic_f64_spread", "atomic_f64_hot",
                                         "l2_read_bytes", "sm_clock_mhz")] + [("sm_count", C.c_int)]


SCENE_P = C.c_void_p
DP = C.POINTER(C.c_double)

# name -> (restype, argtypes); every entry point declared in include/tp.h
SIGNATURES = {
    "tp_create_scene": (C.c_int, [C.POINTER(tp_scene_desc), C.POINTER(SCENE_P)]),
    "tp_set_materials": (C.c_int, [SCENE_P, C.POINTER(tp_material), C.c_int]),
    "tp_set_bias": (C.c_int, [SCENE_P, C.c_int, DP]),
    "tp_run_histories": (C.c_int, [SCENE_P, C.POINTER(tp_run)]),
    "tp_read_tallies": (C.c_int, [SCENE_P, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int]),
    "tp_read_raw": (C.c_int, [SCENE_P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_int]),
    "tp_backward": (C.c_int, [SCENE_P, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "tp_write_raw": (C.c_int, [SCENE_P, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                               C.c_int]),
    "tp_set_params": (C.c_int, [SCENE_P, DP]),
    "tp_reset_tallies": (C.c_int, [SCENE_P]),
    "tp_get_counters": (C.c_int, [SCENE_P, C.POINTER(C.c_int64)]),
    "tp_get_launch": (C.c_int, [SCENE_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tp_total_bins": (C.c_int, [SCENE_P]),
    "tp_get_launch_count": (C.c_int, [SCENE_P]),
    "tp_get_launch_info": (C.c_int, [SCENE_P, C.POINTER(tp_launch_info)]),
    "tp_abort": (C.c_int, [SCENE_P]),
    "tp_measure_peaks": (C.c_int, [C.POINTER(tp_peaks), C.c_void_p]),
    "tp_set_test_flags": (C.c_int, [SCENE_P, C.c_int]),
    "tp_destroy_scene": (None, [SCENE_P]),
    "tp_last_error": (C.c_char_p, []),
    "tp_run_histories_noalloc": (C.c_int, [C.POINTER(tp_scene_desc), C.POINTER(tp_material), C.c_int,
                                           DP, C.POINTER(tp_run), C.c_void_p, C.c_void_p,
                                           C.POINTER(C.c_int64)]),
}


def load(path: Path | str = LIB_PATH) -> C.CDLL:
    p = Path(path)
    if not p.exists():
        raise ImportError(f"{p} is missing: build the CUDA library first "
                          "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(str(p))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()


class TPError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib.tp_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != TP_OK:
        raise TPError(status, where)


# thin wrappers with the C names (argument marshalling only)
def tp_create_scene(desc: tp_scene_desc) -> int:
    out = SCENE_P()
    check(lib.tp_create_scene(C.byref(desc), C.byref(out)), "tp_create_scene")
    return out.value


def tp_set_materials(scene: int, mats) -> None:
    arr = (tp_material * max(1, len(mats)))(*mats)
    check(lib.tp_set_materials(scene, arr, len(mats)), "tp_set_materials")


def tp_set_bias(scene: int, material: int, g) -> None:
    arr = (C.c_double * 3)(*[float(x) for x in g])
    check(lib.tp_set_bias(scene, material, arr), "tp_set_bias")


def tp_run_histories(scene: int, run: tp_run) -> None:
    check(lib.tp_run_histories(scene, C.byref(run)), "tp_run_histories")


def tp_read_tallies(scene: int, tally: int, instance: int, mean_ptr: int, err_ptr: int | None,
                    on_device: bool) -> None:
    check(lib.tp_read_tallies(scene, tally, instance, mean_ptr, err_ptr, int(on_device)),
          "tp_read_tallies")


def tp_read_raw(scene: int, instance: int, sum_ptr, sumsq_ptr, J_ptr, J2_ptr, on_device: bool) -> None:
    check(lib.tp_read_raw(scene, instance, sum_ptr, sumsq_ptr, J_ptr, J2_ptr, int(on_device)),
          "tp_read_raw")


def tp_write_raw(scene: int, instance: int, sum_ptr, sumsq_ptr, J_ptr, J2_ptr, n_histories: float,
                 on_device: bool) -> None:
    check(lib.tp_write_raw(scene, instance, sum_ptr, sumsq_ptr, J_ptr, J2_ptr, float(n_histories), int(on_device)),
          "tp_write_raw")


def tp_backward(scene: int, grad_ptr: int, out_ptr: int, on_device: bool, stream: int | None) -> None:
    check(lib.tp_backward(scene, grad_ptr, out_ptr, int(on_device), stream), "tp_backward")


def tp_set_params(scene: int, params) -> None:
    import numpy as np
    a = np.ascontiguousarray(params, dtype=np.float64).reshape(-1)
    check(lib.tp_set_params(scene, a.ctypes.data_as(DP)), "tp_set_params")


def tp_reset_tallies(scene: int) -> None:
    check(lib.tp_reset_tallies(scene), "tp_reset_tallies")


def tp_get_counters(scene: int) -> dict:
    out = (C.c_int64 * 8)()
    check(lib.tp_get_counters(scene, out), "tp_get_counters")
    return dict(zip(COUNTER_NAMES, list(out)))


def tp_abort(scene: int) -> None:
    check(lib.tp_abort(scene), "tp_abort")


def tp_set_test_flags(scene: int | None, flags: int) -> None:
    check(lib.tp_set_test_flags(scene, flags), "tp_set_test_flags")


def tp_get_counters_status(scene: int) -> tuple[dict, int]:
    """Counters and the device status of the runs since the last reset
    (tp_get_counters without raising)."""
    out = (C.c_int64 * 8)()
    st = lib.tp_get_counters(scene, out)
    return dict(zip(COUNTER_NAMES, list(out))), st


def tp_measure_peaks(stream: int | None = None) -> dict:
    out = tp_peaks()
    check(lib.tp_measure_peaks(C.byref(out), stream), "tp_measure_peaks")
    return {n: getattr(out, n) for n, _ in tp_peaks._fields_}


def tp_get_launch(scene: int) -> tuple[int, int, int]:
    k, b, c = C.c_int(), C.c_int(), C.c_int()
    check(lib.tp_get_launch(scene, C.byref(k), C.byref(b), C.byref(c)), "tp_get_launch")
    return k.value, b.value, c.value


def tp_get_launch_info(scene: int) -> dict:
    out = tp_launch_info()
    check(lib.tp_get_launch_info(scene, C.byref(out)), "tp_get_launch_info")
    return {n: getattr(out, n) for n, _ in tp_launch_info._fields_}


def tp_get_launch_count(scene: int) -> int:
    return lib.tp_get_launch_count(scene)


def tp_total_bins(scene: int) -> int:
    return lib.tp_total_bins(scene)


def tp_destroy_scene(scene: int) -> None:
    lib.tp_destroy_scene(scene)


def tp_last_error() -> str:
    return lib.tp_last_error().decode(errors="replace")
