"""The C ABI without a GPU: the library loads, exports every entry point that
include/tp.h declares, its structures have the header's layout, and
descriptions are rejected with the documented status before any device work."""
import ctypes as C
import re
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
HEADER = ROOT / "include" / "tp.h"


@pytest.fixture(scope="module")
def native():
    from paper_2304_06226_gb300 import build
    build.build()
    from paper_2304_06226_gb300 import native as N
    return N


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tp_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(native):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(native.lib, n), n
    assert set(names) == set(native.SIGNATURES), set(names) ^ set(native.SIGNATURES)


def test_struct_layout_matches_header(native, tmp_path):
    structs = ["tp_prim", "tp_mirror", "tp_chopper", "tp_tally_desc", "tp_source", "tp_scene_desc",
               "tp_material", "tp_record", "tp_run", "tp_launch_info", "tp_peaks"]
    src = tmp_path / "sz.c"
    body = "".join(f'printf("%zu\\n", sizeof({s}));' for s in structs)
    src.write_text(f'#include <stdio.h>\n#include "tp.h"\nint main(void){{{body}return 0;}}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    sizes = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    for s, n in zip(structs, sizes):
        assert C.sizeof(getattr(native, s)) == n, s


def _desc(native, **kw):
    N = native
    prims = (N.tp_prim * 1)(N.tp_prim(N.TP_BOX, 2, 0, 0, -1, 0, 0, -1, N.D3(0, 0, 0.5), N.D3(5, 5, 0.5)))
    src = N.tp_source(N.TP_SRC_PENCIL, N.D3(0, 0, -1), N.D2(0, 0), 1.8, 1.8, N.D2(0, 0), 0, N.D2(0, 0),
                      0.0, N.D2(0, 0), 0.0)
    tallies = (N.tp_tally_desc * 1)(N.tp_tally_desc(N.TP_TALLY_COUNT, N.TP_PTS_EXIT, 0, 5, -1, N.I2(1, 1),
                                                    N.D2(0, 0), N.D2(1, 1), N.D3(0, 0, 0), N.D3(0, 0, 1)))
    d = N.tp_scene_desc(N.TP_SPHERE, N.D3(0, 0, 0.5), N.D3(0, 100, 0), 1, prims, 0, None, src, 1, tallies,
                        1, None, 0, None, 0.0, N.TP_FP64, 0)
    for k, v in kw.items():
        setattr(d, k, v)
    d._keep = (prims, tallies)
    return d


@pytest.mark.parametrize("field,value,status", [
    ("precision", 7, 1), ("world_shape", 9, 1), ("n_instances", 0, 1), ("n_tallies", 99, 1),
    ("n_params", 9, 1), ("event_cap", -1, 1),
    ("n_prims", 16777215, 1),   # TP_MAX_PRIMS + 1: primitive indices must stay below the "none" marker
])
def test_invalid_descriptions_rejected_before_device_work(native, field, value, status):
    d = _desc(native, **{field: value})
    out = C.c_void_p()
    st = native.lib.tp_create_scene(C.byref(d), C.byref(out))
    assert st == status
    assert out.value is None
    assert native.tp_last_error()


def test_invalid_primitives_rejected(native):
    N = native
    d = _desc(native)
    bad = (N.tp_prim * 1)(N.tp_prim(N.TP_BOX, 2, 0, 0, -1, 0, 0, -1, N.D3(0, 0, 0.5), N.D3(-1, 5, 0.5)))
    d.prims = bad
    assert native.lib.tp_create_scene(C.byref(d), C.byref(C.c_void_p())) == N.TP_ERR_INVALID_ARG
    outside = (N.tp_prim * 1)(N.tp_prim(N.TP_BOX, 2, 0, 0, -1, 0, 0, -1, N.D3(0, 0, 99.0), N.D3(5, 5, 5)))
    d.prims = outside
    assert native.lib.tp_create_scene(C.byref(d), C.byref(C.c_void_p())) == N.TP_ERR_GEOMETRY
    two = (N.tp_prim * 2)(N.tp_prim(N.TP_BOX, 2, 0, 0, -1, 0, 0, -1, N.D3(0, 0, 0.5), N.D3(5, 5, 0.5)),
                          N.tp_prim(N.TP_SPHERE, 2, 0, 0, -1, 0, 0, -1, N.D3(1, 1, 0.8), N.D3(0, 1.0, 0)))
    d.prims = two
    d.n_prims = 2
    assert native.lib.tp_create_scene(C.byref(d), C.byref(C.c_void_p())) == N.TP_ERR_GEOMETRY
    assert "overlap" in native.tp_last_error()


def test_null_arguments(native):
    N = native
    assert N.lib.tp_create_scene(None, None) == N.TP_ERR_INVALID_ARG
    assert N.lib.tp_run_histories(None, None) == N.TP_ERR_INVALID_ARG
    assert N.lib.tp_set_materials(None, None, 0) == N.TP_ERR_INVALID_ARG
    assert N.lib.tp_read_tallies(None, 0, 0, None, None, 0) == N.TP_ERR_INVALID_ARG
    assert N.lib.tp_get_launch_info(None, None) == N.TP_ERR_INVALID_ARG
    assert N.lib.tp_total_bins(None) == 0
    assert N.lib.tp_get_launch_count(None) == 0


def test_invalid_choppers_rejected_before_device_work(native):
    N = native
    d = _desc(native)
    tube = lambda **kw: N.tp_prim(**{"shape": N.TP_TUBE, "axis": 2, "material": -1, "role": 0, "mirror": -1,
                                    "bind_rmin": 0, "bind_rmax": 0, "chopper": 0, "centre": N.D3(0, 0, 0.5),
                                    "params": N.D3(0, 5, 0.05), **kw})
    good = N.tp_chopper(1.0, 4, 100.0, 0.35, 0.0)
    cases = [
        (tube(shape=N.TP_BOX, params=N.D3(5, 5, 0.05)), good),   # not a tube
        (tube(material=0), good),                                # not vacuum
        (tube(chopper=1), good),                                 # index out of range
        (tube(), N.tp_chopper(1.0, 0, 100.0, 0.35, 0.0)),        # no window
        (tube(), N.tp_chopper(1.0, 4, 100.0, 0.0, 0.0)),         # closed window
        (tube(), N.tp_chopper(-1.0, 4, 100.0, 0.35, 0.0)),       # negative radius
        (tube(), N.tp_chopper(1.0, 4, float("nan"), 0.35, 0.0)),  # no frequency
    ]
    for prim, ch in cases:
        prims = (N.tp_prim * 1)(prim)
        chs = (N.tp_chopper * 1)(ch)
        d.prims, d.n_choppers, d.choppers = prims, 1, chs
        out = C.c_void_p()
        assert N.lib.tp_create_scene(C.byref(d), C.byref(out)) == N.TP_ERR_INVALID_ARG, (prim.shape, ch.n_windows)
        assert out.value is None
        assert "chopper" in N.tp_last_error()


def test_tof_scorer_is_one_dimensional(native):
    N = native
    d = _desc(native)
    t = (N.tp_tally_desc * 1)(N.tp_tally_desc(N.TP_TALLY_TOF, N.TP_PTS_EXIT, 0, -1, -1, N.I2(10, 2),
                                              N.D2(0, 0), N.D2(0.01, 1), N.D3(0, 0, 0), N.D3(0, 0, 1)))
    d.tallies = t
    assert N.lib.tp_create_scene(C.byref(d), C.byref(C.c_void_p())) == N.TP_ERR_INVALID_ARG
    assert "1-D" in N.tp_last_error()
