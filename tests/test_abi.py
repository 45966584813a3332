"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; argument checks that fire before any device work.
CPU only: no call here touches a GPU."""
import ctypes
import glob
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_1906_04722_gb300 as lbm
    return lbm


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("lbm_create_domain", "lbm_set_pressure_bc", "lbm_step", "lbm_measure", "lbm_destroy",
              "lbm_last_error", "lbm_get_density"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    path = lib.library_path()
    lib.load()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = declared_symbols() - exported
    assert not missing, missing
    # the binding knows every declared symbol too
    assert declared_symbols() <= set(lib.SIGNATURES)


def test_library_is_built_for_sm_103a_only():
    """The build compiles every source for sm_103a and nothing else (checked on the
    build configuration; no tool reads the compiled code)."""
    from paper_1906_04722_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_new_entry_points_reject_bad_arguments_before_device_work(lib):
    """Lattice features, the GEMM wait self-test and the batch form are checked
    on the host before any device work (documented in lbm.h)."""
    L = lib.load()
    out = np.zeros(14)
    assert L.lbm_throat_lattice_features(None, 1, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))) == lib.LBM_ERR_ARG
    collinear = np.array([[0, 0, 0, 5], [10, 0, 0, 5], [20, 0, 0, 5]], dtype=np.float64)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_throat_lattice_features(collinear)
    assert e.value.code == lib.LBM_ERR_ARG
    flag = ctypes.c_int(7)
    assert L.lbm_surrogate_selftest_wait(0, ctypes.byref(flag)) == lib.LBM_ERR_ARG
    assert L.lbm_surrogate_selftest_wait(20000000, ctypes.byref(flag)) == lib.LBM_ERR_ARG
    with pytest.raises(ValueError):
        lib.lbm_run_throat_batch(collinear, lib.make_params(), [2.0], 1, 2.0, form=7)
    # the C check itself, past the binding
    ladder = np.array([2.0])
    sch = lib.lbm_schedule()
    sch.n_incr, sch.n_steps, sch.rho_out_w, sch.batch_form = 1, 1, 2.0, 7
    sch.rho_in_nw = ladder.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    res = (lib.lbm_throat_result * 1)()
    rows = (lib.lbm_increment * 1)()
    tri = np.array([[0, 0, 0, 5], [10, 0, 0, 5], [5, 9, 0, 5]], dtype=np.float64)
    rc = L.lbm_run_throat_batch(tri.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 1, ctypes.byref(lib.make_params()),
                                ctypes.byref(sch), res, rows, None)
    assert rc == lib.LBM_ERR_ARG
    # the marching form's launch shape: 128, 256, 384 or 512 threads, 1 .. 64 planes
    for march in ((100, 16), (256, 65), (256, -1), (-128, 8)):
        with pytest.raises(lib.LbmError) as e:
            lib.lbm_run_throat_batch(tri, lib.make_params(), [2.0], 1, 2.0, form=lib.BATCH_MARCH, march=march)
        assert e.value.code == lib.LBM_ERR_ARG
        assert "march" in lib.lbm_last_error()


@pytest.mark.parametrize("field,value", [("tau", (0.5, 1.0)), ("precision", 3), ("membrane_layers", -1),
                                         ("G", float("nan"))])
def test_bad_params_rejected_before_device_work(lib, field, value):
    p = lib.make_params()
    if field == "tau":
        p.tau[0], p.tau[1] = value
    else:
        setattr(p, field, value)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create_domain(p, None, (4, 4, 4), stream=ctypes.c_void_p(0))
    assert e.value.code == lib.LBM_ERR_ARG


@pytest.mark.parametrize("box", [(0, 4, 4), (4, -1, 4), (5000, 4, 4), (4096, 4096, 4)])
def test_bad_boxes_rejected(lib, box):
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create_domain(lib.make_params(), None, box, stream=ctypes.c_void_p(0))
    assert e.value.code == lib.LBM_ERR_ARG


def test_bad_spheres_rejected(lib):
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create_domain(lib.make_params(), np.array([[1.0, 2.0, np.inf, 3.0]]), (8, 8, 8),
                              stream=ctypes.c_void_p(0))
    assert e.value.code == lib.LBM_ERR_ARG
    with pytest.raises(lib.LbmError):
        lib.lbm_create_domain(lib.make_params(prism_clip=True), np.array([[1.0, 2.0, 3.0, 1.0]]), (8, 8, 8),
                              stream=ctypes.c_void_p(0))


def test_null_domain_calls_rejected(lib):
    L = lib.load()
    assert L.lbm_step(None, 1) == lib.LBM_ERR_ARG
    assert L.lbm_set_pressure_bc(None, 2.0, 2.0) == lib.LBM_ERR_ARG
    assert "NULL" in lib.lbm_last_error()
    L.lbm_destroy(None)  # ignored


def test_throat_rows_sequence(lib):
    """The batch's rows as the binding returns them: throat t's list of rows,
    built from the library's array on first access, with len, negative indices,
    slices and iteration of a list of lists."""
    n, n_incr = 3, 4
    arr = (lib.lbm_increment * (n * n_incr))()
    for t in range(n):
        for i in range(n_incr):
            arr[t * n_incr + i].S_w = t + 0.1 * i
            arr[t * n_incr + i].n_interface = 10 * t + i
    rows = lib.ThroatRows(arr, n, n_incr)
    assert len(rows) == n
    assert rows[1][2]["S_w"] == 1.2 and rows[1][2]["n_interface"] == 12
    assert rows[-1][0] == arr[2 * n_incr].as_dict()
    assert rows[0:2] == [rows[0], rows[1]]
    assert rows[1] is rows[1]  # built once
    flat = []
    flat += rows
    assert flat == [[arr[t * n_incr + i].as_dict() for i in range(n_incr)] for t in range(n)]
    with pytest.raises(IndexError):
        rows[3]
