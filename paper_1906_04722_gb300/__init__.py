"""Python binding of liblbm.so, the GB300 two-component Shan-Chen D3Q19 library.

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  The functions carry the C-ABI names of include/lbm.h; ``Domain`` is a
small convenience wrapper over them.  Arrays are numpy (host) arrays in the
ABI layouts: masks uint8[nz, ny, nx], densities float64[2, nz, ny, nx],
stored populations float32[2, 19, nz, ny, nx].  If the compiled library is
missing and cannot be built, loading raises: there is no CPU fallback.
"""
from __future__ import annotations

import collections.abc
import ctypes
import os
import threading

import numpy as np

from . import build as _build

LBM_OK = 0
LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_TIMEOUT, LBM_ERR_NONFINITE, LBM_ERR_STATE = -1, -2, -3, -4, -5, -6
MASK_SOLID, MASK_ADHESIVE, MASK_MEMBRANE, MASK_INLET, MASK_OUTLET = 1, 2, 4, 8, 16
Q = 19

_lock = threading.Lock()
_lib = None


class LbmError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


class lbm_params(ctypes.Structure):
    _fields_ = [("tau", ctypes.c_double * 2), ("G", ctypes.c_double), ("G_ads", ctypes.c_double * 2),
                ("body_force", ctypes.c_double * 3), ("rho_major", ctypes.c_double),
                ("rho_minor", ctypes.c_double), ("precision", ctypes.c_int), ("periodic", ctypes.c_int * 3),
                ("reservoirs", ctypes.c_int), ("membrane_layers", ctypes.c_int), ("prism_clip", ctypes.c_int)]


class lbm_measurement(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2),
                ("p_w", ctypes.c_double), ("p_nw", ctypes.c_double), ("p_c", ctypes.c_double),
                ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("p_c_res", ctypes.c_double),
                ("S_w", ctypes.c_double),
                ("n_fluid", ctypes.c_longlong), ("n_w", ctypes.c_longlong), ("n_interface", ctypes.c_longlong),
                ("n_bulk_w", ctypes.c_longlong), ("n_bulk_nw", ctypes.c_longlong), ("n_in", ctypes.c_longlong),
                ("n_out", ctypes.c_longlong), ("n_nonfinite", ctypes.c_longlong),
                ("n_negative", ctypes.c_longlong), ("status_flags", ctypes.c_int)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if name == "mass" else v
        return out


class lbm_increment(ctypes.Structure):
    _fields_ = [("rho_in_nw", ctypes.c_double), ("p_c", ctypes.c_double), ("p_c_res", ctypes.c_double),
                ("S_w", ctypes.c_double), ("p_w", ctypes.c_double), ("p_nw", ctypes.c_double),
                ("phi_probe", ctypes.c_double), ("n_interface", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


class lbm_schedule(ctypes.Structure):
    _fields_ = [("n_incr", ctypes.c_int), ("n_steps", ctypes.c_int),
                ("rho_in_nw", ctypes.POINTER(ctypes.c_double)), ("rho_out_w", ctypes.c_double),
                ("per_throat", ctypes.c_int), ("batch_form", ctypes.c_int), ("march_threads", ctypes.c_int),
                ("march_planes", ctypes.c_int)]


class lbm_throat_result(ctypes.Structure):
    _fields_ = [("p_ce", ctypes.c_double), ("invaded_at", ctypes.c_int), ("dims", ctypes.c_int * 3),
                ("probe", ctypes.c_int * 3), ("n_fluid", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        return {"p_ce": self.p_ce, "invaded_at": self.invaded_at, "dims": tuple(self.dims),
                "probe": tuple(self.probe), "n_fluid": self.n_fluid}


class lbm_throat_surrogate_config(ctypes.Structure):
    _fields_ = [("n_incr", ctypes.c_int), ("n_members", ctypes.c_int), ("n_hidden", ctypes.c_int),
                ("n_layers", ctypes.c_int), ("half", ctypes.c_int), ("seed", ctypes.c_ulonglong),
                ("theta", ctypes.c_double)]


class lbm_tune_result(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("by", ctypes.c_int), ("lz", ctypes.c_int), ("lead", ctypes.c_int),
                ("ms_per_step", ctypes.c_double), ("n_candidates", ctypes.c_int), ("prefetch", ctypes.c_int),
                ("shape", ctypes.c_int), ("order", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {"kind": {0: "staged", 1: "tma", 2: "split", 3: "staged2", 4: "push"}.get(self.kind, "?"),
                "by": self.by, "lz": self.lz, "lead": self.lead,
                "ms_per_step": self.ms_per_step, "n_candidates": self.n_candidates, "prefetch": self.prefetch,
                "shape": self.shape, "order": self.order}


class lbm_surrogate_config(ctypes.Structure):
    _fields_ = [("n_in", ctypes.c_int), ("n_hidden", ctypes.c_int), ("n_layers", ctypes.c_int),
                ("n_out", ctypes.c_int), ("n_members", ctypes.c_int), ("half", ctypes.c_int),
                ("seed", ctypes.c_ulonglong)]


# exported symbol -> (restype, argtypes)
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_FP = ctypes.POINTER(ctypes.c_float)
_U8P = ctypes.POINTER(ctypes.c_uint8)
_IP = ctypes.POINTER(ctypes.c_int)
_LLP = ctypes.POINTER(ctypes.c_longlong)
SIGNATURES = {
    "lbm_create_domain": (ctypes.c_int, [ctypes.POINTER(lbm_params), _DP, ctypes.c_int, _IP, _VP, ctypes.POINTER(_VP)]),
    "lbm_create_domain_mask": (ctypes.c_int, [ctypes.POINTER(lbm_params), _U8P, _IP, _VP, ctypes.POINTER(_VP)]),
    "lbm_set_densities": (ctypes.c_int, [_VP, _DP]),
    "lbm_set_pressure_bc": (ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_double]),
    "lbm_step": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_measure": (ctypes.c_int, [_VP, ctypes.POINTER(lbm_measurement)]),
    "lbm_get_density": (ctypes.c_int, [_VP, _DP]),
    "lbm_get_density_at": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP]),
    "lbm_run_drainage": (ctypes.c_int, [_VP, _DP, ctypes.c_int, ctypes.c_int, ctypes.c_double, _IP,
                                        ctypes.POINTER(lbm_increment), _DP, _IP]),
    "lbm_get_mask": (ctypes.c_int, [_VP, _U8P]),
    "lbm_get_dims": (ctypes.c_int, [_VP, _IP, _LLP]),
    "lbm_get_state": (ctypes.c_int, [_VP, _FP, _LLP]),
    "lbm_set_state": (ctypes.c_int, [_VP, _FP, ctypes.c_longlong]),
    "lbm_measure_state_noalloc": (ctypes.c_int, [ctypes.POINTER(lbm_params), _IP, _VP, _VP, _VP,
                                                 ctypes.POINTER(lbm_measurement)]),
    "lbm_set_tile": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "lbm_set_push_shape": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "lbm_set_push_prefetch": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_set_push_order": (ctypes.c_int, [_VP, ctypes.c_int]),
    "lbm_get_tile": (ctypes.c_int, [_VP, _IP, _IP, _IP]),
    "lbm_set_step_kernel": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int]),
    "lbm_get_step_kernel": (ctypes.c_int, [_VP, _IP, _IP]),
    "lbm_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(lbm_tune_result)]),
    "lbm_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int, _IP]),
    "lbm_surrogate_selftest_wait": (ctypes.c_int, [ctypes.c_int, _IP]),
    "lbm_throat_geometry": (ctypes.c_int, [_DP, _IP, _U8P, _IP]),
    "lbm_throat_lattice_features": (ctypes.c_int, [_DP, ctypes.c_int, _DP]),
    "lbm_regular_triangulation": (ctypes.c_int, [_DP, ctypes.c_int, _IP, ctypes.c_int, _IP]),
    "lbm_pn_build": (ctypes.c_int, [_DP, ctypes.c_int, _IP, ctypes.c_int, _U8P, _IP, _DP, _IP, _IP, _IP,
                                    ctypes.c_int]),
    "lbm_pn_drainage": (ctypes.c_int, [ctypes.c_int, _DP, ctypes.c_int, _IP, _DP, ctypes.c_int, _DP, _DP, _IP,
                                       _IP]),
    "lbm_throat_incircle": (ctypes.c_int, [_DP, ctypes.c_int, _DP]),
    "lbm_throat_pce_incircle": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP]),
    "lbm_throat_pce_msp": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP]),
    "lbm_throat_msp_terms": (ctypes.c_int, [_DP, ctypes.c_double, ctypes.c_double, _DP]),
    "lbm_contact_angle_estimate": (ctypes.c_int, [ctypes.c_double] * 5 + [_DP]),
    "lbm_partition_lpt": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_int, _IP, _DP]),
    "lbm_packing_throats": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, _IP, ctypes.c_int, _IP]),
    "lbm_pressure_ladder": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_int] + [ctypes.c_double] * 5 + [_DP]),
    "lbm_throat_surrogate_inputs": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.c_double, _FP, _DP]),
    "lbm_throat_surrogate_create": (ctypes.c_int, [ctypes.POINTER(lbm_throat_surrogate_config), _VP,
                                                   ctypes.POINTER(_VP)]),
    "lbm_throat_surrogate_fit": (ctypes.c_int, [_VP, _DP, ctypes.c_int, ctypes.POINTER(lbm_throat_result),
                                                ctypes.POINTER(lbm_increment), ctypes.c_int, ctypes.c_int,
                                                ctypes.c_float, ctypes.c_ulonglong, _DP, _IP]),
    "lbm_throat_surrogate_predict": (ctypes.c_int, [_VP, _DP, ctypes.c_int, _DP, _DP, _FP]),
    "lbm_throat_surrogate_predict_with_fallback": (ctypes.c_int, [_VP, _DP, ctypes.c_int, ctypes.c_double,
                                                                  ctypes.POINTER(lbm_params),
                                                                  ctypes.POINTER(lbm_schedule), _DP, _IP, _DP]),
    "lbm_throat_surrogate_scaling": (ctypes.c_int, [_VP, _DP, _DP, _DP, _DP]),
    "lbm_throat_surrogate_network": (_VP, [_VP]),
    "lbm_throat_surrogate_destroy": (None, [_VP]),
    "lbm_run_throat_batch": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.POINTER(lbm_params),
                                            ctypes.POINTER(lbm_schedule), ctypes.POINTER(lbm_throat_result),
                                            ctypes.POINTER(lbm_increment), _VP]),
    "lbm_run_throat_batch_refined": (ctypes.c_int, [_DP, ctypes.c_int, ctypes.POINTER(lbm_params),
                                                    ctypes.POINTER(lbm_schedule), ctypes.c_int,
                                                    ctypes.POINTER(lbm_throat_result), ctypes.POINTER(lbm_increment),
                                                    _DP, _VP]),
    "lbm_surrogate_create": (ctypes.c_int, [ctypes.POINTER(lbm_surrogate_config), _VP, ctypes.POINTER(_VP)]),
    "lbm_surrogate_num_params": (ctypes.c_int, [_VP]),
    "lbm_surrogate_get_params": (ctypes.c_int, [_VP, ctypes.c_int, _FP]),
    "lbm_surrogate_set_params": (ctypes.c_int, [_VP, ctypes.c_int, _FP]),
    "lbm_surrogate_forward": (ctypes.c_int, [_VP, ctypes.c_int, _FP, ctypes.c_int, _FP]),
    "lbm_surrogate_gradients": (ctypes.c_int, [_VP, ctypes.c_int, _FP, _FP, ctypes.c_int, _FP, _DP]),
    "lbm_surrogate_train": (ctypes.c_int, [_VP, _FP, _FP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_float,
                                           ctypes.c_ulonglong, _DP]),
    "lbm_surrogate_predict": (ctypes.c_int, [_VP, _FP, ctypes.c_int, _FP, _FP]),
    "lbm_surrogate_destroy": (None, [_VP]),
    "lbm_destroy": (None, [_VP]),
    "lbm_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def load():
    """Load liblbm.so (building it first when its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise ImportError(f"liblbm.so is missing at {_build.LIB}; run paper_1906_04722_gb300/build.py")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(rc: int, where: str):
    if rc != LBM_OK:
        raise LbmError(rc, where, load().lbm_last_error().decode())


def _torch_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return ctypes.c_void_p(0)


def make_params(tau=(1.0, 1.0), G=0.9, G_ads=(-0.3, 0.3), body_force=(0.0, 0.0, 0.0), rho_major=2.0,
                rho_minor=0.06, periodic=(0, 0, 0), reservoirs=False, membrane_layers=0, prism_clip=False,
                precision=0) -> lbm_params:
    p = lbm_params()
    for s in range(2):
        p.tau[s] = float(tau[s])
        p.G_ads[s] = float(G_ads[s])
    p.G = float(G)
    for d in range(3):
        p.body_force[d] = float(body_force[d])
        p.periodic[d] = int(bool(periodic[d]))
    p.rho_major = float(rho_major)
    p.rho_minor = float(rho_minor)
    p.precision = int(precision)
    p.reservoirs = int(bool(reservoirs))
    p.membrane_layers = int(membrane_layers)
    p.prism_clip = int(bool(prism_clip))
    return p


# --------------------------------------------------------- C-ABI functions
def lbm_create_domain(params: lbm_params, spheres, box, stream=None):
    L = load()
    sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4)) if spheres is not None else None
    n = 0 if sp is None else sp.shape[0]
    bx = (ctypes.c_int * 3)(*[int(v) for v in box])
    h = ctypes.c_void_p()
    rc = L.lbm_create_domain(ctypes.byref(params), sp.ctypes.data_as(_DP) if n else None, n, bx,
                             stream if stream is not None else _torch_stream(), ctypes.byref(h))
    _check(rc, "lbm_create_domain")
    return h


def lbm_create_domain_mask(params: lbm_params, mask: np.ndarray, stream=None):
    L = load()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = m.shape
    bx = (ctypes.c_int * 3)(nx, ny, nz)
    h = ctypes.c_void_p()
    rc = L.lbm_create_domain_mask(ctypes.byref(params), m.ctypes.data_as(_U8P), bx,
                                  stream if stream is not None else _torch_stream(), ctypes.byref(h))
    _check(rc, "lbm_create_domain_mask")
    return h


def lbm_get_dims(h):
    d = (ctypes.c_int * 3)()
    nf = ctypes.c_longlong()
    _check(load().lbm_get_dims(h, d, ctypes.byref(nf)), "lbm_get_dims")
    return (d[0], d[1], d[2]), nf.value


def lbm_set_densities(h, rho: np.ndarray):
    r = np.ascontiguousarray(rho, dtype=np.float64)
    _check(load().lbm_set_densities(h, r.ctypes.data_as(_DP)), "lbm_set_densities")


def lbm_set_pressure_bc(h, rho_in_nw: float, rho_out_w: float):
    _check(load().lbm_set_pressure_bc(h, float(rho_in_nw), float(rho_out_w)), "lbm_set_pressure_bc")


def lbm_step(h, n_steps: int):
    _check(load().lbm_step(h, int(n_steps)), "lbm_step")


def lbm_measure(h, allow_nonfinite: bool = False) -> dict:
    m = lbm_measurement()
    rc = load().lbm_measure(h, ctypes.byref(m))
    if not (allow_nonfinite and rc == LBM_ERR_NONFINITE):
        _check(rc, "lbm_measure")
    return m.as_dict()


def lbm_get_density(h) -> np.ndarray:
    (nx, ny, nz), _ = lbm_get_dims(h)
    out = np.empty((2, nz, ny, nx), dtype=np.float64)
    _check(load().lbm_get_density(h, out.ctypes.data_as(_DP)), "lbm_get_density")
    return out


def lbm_get_density_at(h, x: int, y: int, z: int):
    out = (ctypes.c_double * 2)()
    _check(load().lbm_get_density_at(h, int(x), int(y), int(z), out), "lbm_get_density_at")
    return out[0], out[1]


def lbm_run_drainage(h, rho_in_nw, n_steps: int, rho_out_w: float, probe):
    """Pressure ladder; returns {'rows': [...], 'p_ce': float, 'invaded_at': int}."""
    lad = np.ascontiguousarray(np.asarray(rho_in_nw, dtype=np.float64))
    n = lad.shape[0]
    rows = (lbm_increment * n)()
    pr = (ctypes.c_int * 3)(*[int(v) for v in probe])
    pce = ctypes.c_double()
    inv = ctypes.c_int()
    _check(load().lbm_run_drainage(h, lad.ctypes.data_as(_DP), n, int(n_steps), float(rho_out_w), pr, rows,
                                   ctypes.byref(pce), ctypes.byref(inv)), "lbm_run_drainage")
    return {"rows": [r.as_dict() for r in rows], "p_ce": pce.value, "invaded_at": inv.value}


def lbm_get_mask(h) -> np.ndarray:
    (nx, ny, nz), _ = lbm_get_dims(h)
    out = np.empty((nz, ny, nx), dtype=np.uint8)
    _check(load().lbm_get_mask(h, out.ctypes.data_as(_U8P)), "lbm_get_mask")
    return out


def lbm_get_state(h):
    (nx, ny, nz), _ = lbm_get_dims(h)
    out = np.empty((2, Q, nz, ny, nx), dtype=np.float32)
    st = ctypes.c_longlong()
    _check(load().lbm_get_state(h, out.ctypes.data_as(_FP), ctypes.byref(st)), "lbm_get_state")
    return out, st.value


def lbm_set_state(h, f: np.ndarray, step: int):
    a = np.ascontiguousarray(f, dtype=np.float32)
    _check(load().lbm_set_state(h, a.ctypes.data_as(_FP), int(step)), "lbm_set_state")


def lbm_measure_state_noalloc(params: lbm_params, box, f_dev_ptr: int, mask_dev_ptr: int, stream=None,
                              allow_nonfinite: bool = False) -> dict:
    """Measurements of a state in caller-owned device memory (raw device
    pointers, lbm_get_state / mask layouts) without any device allocation."""
    m = lbm_measurement()
    bx = (ctypes.c_int * 3)(*[int(v) for v in box])
    rc = load().lbm_measure_state_noalloc(ctypes.byref(params), bx, ctypes.c_void_p(f_dev_ptr),
                                          ctypes.c_void_p(mask_dev_ptr),
                                          stream if stream is not None else _torch_stream(), ctypes.byref(m))
    if not (allow_nonfinite and rc == LBM_ERR_NONFINITE):
        _check(rc, "lbm_measure_state_noalloc")
    return m.as_dict()


def lbm_set_tile(h, by: int, lz: int, lead: int):
    _check(load().lbm_set_tile(h, int(by), int(lz), int(lead)), "lbm_set_tile")


def lbm_get_tile(h):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().lbm_get_tile(h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "lbm_get_tile")
    return a.value, b.value, c.value


KERNEL_STAGED = 0
KERNEL_TMA = 1
KERNEL_SPLIT = 2
KERNEL_STAGED2 = 3
KERNEL_PUSH = 4
# lbm_set_push_shape index -> (box rows, plane stages, CTAs per SM, pairs held in registers)
PUSH_SHAPE_TABLE = [(8, 4, 1, False), (6, 3, 2, False), (10, 3, 1, False), (7, 3, 2, False), (10, 4, 1, False),
                    (12, 3, 1, False), (6, 3, 2, True), (10, 4, 1, True), (12, 3, 1, True), (5, 4, 2, True),
                    (8, 4, 1, True), (7, 3, 2, True)]
PUSH_SHAPES = len(PUSH_SHAPE_TABLE)
# lbm_set_push_shape index on a 16-bit domain -> (box rows, plane stages, CTAs per SM, words held in registers)
PUSH16_SHAPE_TABLE = [(8, 4, 2, False), (6, 4, 2, False), (7, 4, 2, False), (10, 3, 2, False), (6, 4, 2, True),
                      (8, 4, 2, True), (9, 3, 2, False), (7, 3, 3, False), (6, 3, 3, False), (11, 3, 2, False),
                      (12, 3, 1, True), (8, 3, 2, True)]
BATCH_AUTO = 0
BATCH_PERSISTENT = 1
BATCH_PER_STEP = 2
BATCH_CELLS = 3
BATCH_MARCH = 4


def lbm_set_step_kernel(h, kind: int, lz: int = 0):
    _check(load().lbm_set_step_kernel(h, int(kind), int(lz)), "lbm_set_step_kernel")


def lbm_set_push_shape(h, shape: int, lz: int = 0):
    _check(load().lbm_set_push_shape(h, int(shape), int(lz)), "lbm_set_push_shape")


def lbm_set_push_prefetch(h, planes: int):
    _check(load().lbm_set_push_prefetch(h, int(planes)), "lbm_set_push_prefetch")


def lbm_set_push_order(h, order: int):
    _check(load().lbm_set_push_order(h, int(order)), "lbm_set_push_order")


def lbm_get_step_kernel(h):
    a, b = ctypes.c_int(), ctypes.c_int()
    _check(load().lbm_get_step_kernel(h, ctypes.byref(a), ctypes.byref(b)), "lbm_get_step_kernel")
    return a.value, b.value


def lbm_autotune(h, trial_steps: int = 20):
    """Times the step kernels / shapes on the domain, keeps the fastest, restores the state."""
    r = lbm_tune_result()
    _check(load().lbm_autotune(h, int(trial_steps), ctypes.byref(r)), "lbm_autotune")
    return r.as_dict()


def lbm_selftest_bounded_wait(limit_us: int) -> bool:
    """True when a bounded mbarrier wait that nothing completes gave up and said so."""
    flag = ctypes.c_int(0)
    _check(load().lbm_selftest_bounded_wait(int(limit_us), ctypes.byref(flag)), "lbm_selftest_bounded_wait")
    return flag.value == 1

def lbm_surrogate_selftest_wait(limit_us: int) -> bool:
    """True when the surrogate GEMM's bounded wait for its MMAs, run with no MMA
    issued, gave up after limit_us and reported it (lbm_surrogate_selftest_wait)."""
    flag = ctypes.c_int(0)
    _check(load().lbm_surrogate_selftest_wait(int(limit_us), ctypes.byref(flag)), "lbm_surrogate_selftest_wait")
    return bool(flag.value)


def lbm_throat_geometry(spheres3):
    """(mask uint8[nz, ny, nx], probe (x, y, z)) of the throat box of three spheres."""
    sp = np.ascontiguousarray(np.asarray(spheres3, dtype=np.float64).reshape(3, 4))
    dims = (ctypes.c_int * 3)()
    _check(load().lbm_throat_geometry(sp.ctypes.data_as(_DP), dims, None, None), "lbm_throat_geometry")
    nx, ny, nz = dims
    mask = np.empty((nz, ny, nx), dtype=np.uint8)
    probe = (ctypes.c_int * 3)()
    _check(load().lbm_throat_geometry(sp.ctypes.data_as(_DP), dims, mask.ctypes.data_as(_U8P), probe),
           "lbm_throat_geometry")
    return mask, tuple(probe)


THROAT_LATTICE_FEATURES = 14


PN_INLET, PN_OUTLET = -1, -2


def lbm_regular_triangulation(spheres) -> np.ndarray:
    """Tetrahedra (m x 4 sphere indices) of the regular triangulation of the
    sphere centres weighted by r^2 (Sec. 2.2.1)."""
    sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    n = ctypes.c_int()
    L = load()
    _check(L.lbm_regular_triangulation(sp.ctypes.data_as(_DP), sp.shape[0], None, 0, ctypes.byref(n)),
           "lbm_regular_triangulation")
    out = np.zeros((max(n.value, 1), 4), dtype=np.int32)
    _check(L.lbm_regular_triangulation(sp.ctypes.data_as(_DP), sp.shape[0], out.ctypes.data_as(_IP), out.shape[0],
                                       ctypes.byref(n)), "lbm_regular_triangulation")
    return out[:n.value]


def lbm_packing_throats(spheres, max_edge: float = 64.0) -> np.ndarray:
    """Interior facets of the packing's regular triangulation with longest centre
    distance below max_edge: m x 3 sphere indices (lbm_packing_throats)."""
    sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    n = ctypes.c_int()
    L = load()
    _check(L.lbm_packing_throats(sp.ctypes.data_as(_DP), sp.shape[0], float(max_edge), None, 0, ctypes.byref(n)),
           "lbm_packing_throats")
    out = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check(L.lbm_packing_throats(sp.ctypes.data_as(_DP), sp.shape[0], float(max_edge), out.ctypes.data_as(_IP),
                                 out.shape[0], ctypes.byref(n)), "lbm_packing_throats")
    return out[:n.value]


def packing_throat_sample(spheres, n, seed: int, max_edge: float = 64.0) -> np.ndarray:
    """n throats (n x 3 x 4 sphere records) of the packing's regular
    triangulation, drawn without replacement (seeded); n = None: all of them."""
    sp = np.asarray(spheres, dtype=np.float64).reshape(-1, 4)
    f = lbm_packing_throats(sp, max_edge)
    if n is not None:
        if n > len(f):
            raise ValueError(f"only {len(f)} throats, asked for {n}")
        f = f[np.sort(np.random.default_rng(seed).choice(len(f), size=n, replace=False))]
    return sp[f]


def lbm_pn_build(spheres, tets, mask: np.ndarray):
    """Pore network of a lattice sample: (pore_volume[m], throat_pores[t, 2],
    throat_spheres[t, 3]) with reservoir links as PN_INLET / PN_OUTLET."""
    sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    tt = np.ascontiguousarray(np.asarray(tets, dtype=np.int32).reshape(-1, 4))
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    nz, ny, nx = m.shape
    bx = (ctypes.c_int * 3)(nx, ny, nz)
    vol = np.zeros(tt.shape[0])
    n = ctypes.c_int()
    L = load()
    args = (sp.ctypes.data_as(_DP), sp.shape[0], tt.ctypes.data_as(_IP), tt.shape[0], m.ctypes.data_as(_U8P), bx,
            vol.ctypes.data_as(_DP), ctypes.byref(n))
    _check(L.lbm_pn_build(*args, None, None, 0), "lbm_pn_build")
    tp = np.zeros((max(n.value, 1), 2), dtype=np.int32)
    ts = np.zeros((max(n.value, 1), 3), dtype=np.int32)
    _check(L.lbm_pn_build(*args, tp.ctypes.data_as(_IP), ts.ctypes.data_as(_IP), tp.shape[0]), "lbm_pn_build")
    return vol, tp[:n.value], ts[:n.value]


def lbm_pn_drainage(pore_volume, throat_pores, throat_pce, p_c_levels):
    """Quasi-static drainage of a pore network: (S_w per level, invaded_at per
    pore, trapped_at per pore)."""
    vol = np.ascontiguousarray(pore_volume, dtype=np.float64)
    tp = np.ascontiguousarray(np.asarray(throat_pores, dtype=np.int32).reshape(-1, 2))
    pce = np.ascontiguousarray(throat_pce, dtype=np.float64)
    lev = np.ascontiguousarray(p_c_levels, dtype=np.float64)
    sw = np.zeros(lev.shape[0])
    inv = np.zeros(vol.shape[0], dtype=np.int32)
    trap = np.zeros(vol.shape[0], dtype=np.int32)
    _check(load().lbm_pn_drainage(vol.shape[0], vol.ctypes.data_as(_DP), tp.shape[0], tp.ctypes.data_as(_IP),
                                  pce.ctypes.data_as(_DP), lev.shape[0], lev.ctypes.data_as(_DP),
                                  sw.ctypes.data_as(_DP), inv.ctypes.data_as(_IP), trap.ctypes.data_as(_IP)),
           "lbm_pn_drainage")
    return sw, inv, trap


def lbm_partition_lpt(cost, parts: int):
    """(part of each item, load of each part): longest-processing-time-first split."""
    c = np.ascontiguousarray(np.asarray(cost, dtype=np.float64).reshape(-1))
    part = np.empty(c.shape[0], dtype=np.int32)
    lp = np.empty(int(parts))
    _check(load().lbm_partition_lpt(c.ctypes.data_as(_DP), c.shape[0], int(parts), part.ctypes.data_as(_IP),
                                    lp.ctypes.data_as(_DP)), "lbm_partition_lpt")
    return part, lp


def run_throat_batch_sharded(throats, params: lbm_params, rho_in_nw, n_steps: int, rho_out_w: float, rank: int,
                             world: int, gather, run=None):
    """The throats of one list split over `world` ranks (lbm_partition_lpt on
    the non-solid cells of each box), this rank's share run with
    lbm_run_throat_batch (or `run`, same signature), and every rank's results
    gathered back into the list's order.  gather(obj) -> list of every rank's obj
    (torch.distributed.all_gather_object, for one).  Returns (results, rows)."""
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 3, 4))
    F = lbm_throat_lattice_features(th)
    cost = F[:, 0] * F[:, 1] * F[:, 2] * F[:, 3]
    part, _ = lbm_partition_lpt(cost, world)
    mine = np.flatnonzero(part == rank)
    lad = np.asarray(rho_in_nw, dtype=np.float64)
    my_lad = lad[mine] if lad.ndim == 2 else lad
    res, rows = ([], []) if len(mine) == 0 else (run or lbm_run_throat_batch)(th[mine], params, my_lad, n_steps,
                                                                                rho_out_w)
    pieces = gather((mine.tolist(), res, rows))
    out_res, out_rows = [None] * len(th), [None] * len(th)
    for idx, r, w in pieces:
        for j, t in enumerate(idx):
            out_res[t], out_rows[t] = r[j], w[j]
    return out_res, out_rows


def lbm_throat_incircle(throats) -> np.ndarray:
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 12))
    out = np.zeros(th.shape[0])
    _check(load().lbm_throat_incircle(th.ctypes.data_as(_DP), th.shape[0], out.ctypes.data_as(_DP)),
           "lbm_throat_incircle")
    return out


def lbm_throat_pce_msp(throats, sigma: float, cos_theta: float) -> np.ndarray:
    """Mayer-Stowe-Princen p_c^e of each throat (+inf closed, NaN no regular meniscus)."""
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 12))
    out = np.zeros(th.shape[0])
    _check(load().lbm_throat_pce_msp(th.ctypes.data_as(_DP), th.shape[0], float(sigma), float(cos_theta),
                                     out.ctypes.data_as(_DP)), "lbm_throat_pce_msp")
    return out


def lbm_throat_msp_terms(throat, r: float, cos_theta: float):
    """(A_nw, L_nw, L_ns) of one throat at meniscus radius r."""
    th = np.ascontiguousarray(np.asarray(throat, dtype=np.float64).reshape(12))
    out = np.zeros(3)
    _check(load().lbm_throat_msp_terms(th.ctypes.data_as(_DP), float(r), float(cos_theta), out.ctypes.data_as(_DP)),
           "lbm_throat_msp_terms")
    return tuple(out)


def lbm_throat_pce_incircle(throats, sigma: float, cos_theta: float) -> np.ndarray:
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 12))
    out = np.zeros(th.shape[0])
    _check(load().lbm_throat_pce_incircle(th.ctypes.data_as(_DP), th.shape[0], float(sigma), float(cos_theta),
                                          out.ctypes.data_as(_DP)), "lbm_throat_pce_incircle")
    return out


def lbm_throat_lattice_features(throats) -> np.ndarray:
    """n x 14 lattice description of each throat box (lbm_throat_lattice_features)."""
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 3, 4))
    out = np.empty((th.shape[0], THROAT_LATTICE_FEATURES), dtype=np.float64)
    _check(load().lbm_throat_lattice_features(th.ctypes.data_as(_DP), th.shape[0], out.ctypes.data_as(_DP)),
           "lbm_throat_lattice_features")
    return out


class ThroatRows(collections.abc.Sequence):
    """The rows of a throat batch, throat by throat: item t is the list of that
    throat's n_incr rows (dicts of lbm_increment's fields).  The rows stay in the
    library's array until read; each throat's list is built on first access."""

    def __init__(self, arr, n: int, n_incr: int):
        self._arr, self._n, self._incr = arr, n, n_incr
        self._built = {}

    def __len__(self):
        return self._n

    def __getitem__(self, t):
        if isinstance(t, slice):
            return [self[i] for i in range(*t.indices(self._n))]
        t = int(t)
        if t < 0:
            t += self._n
        if not 0 <= t < self._n:
            raise IndexError("throat index out of range")
        out = self._built.get(t)
        if out is None:
            out = [self._arr[t * self._incr + i].as_dict() for i in range(self._incr)]
            self._built[t] = out
        return out


def _batch_schedule(n, rho_in_nw, n_steps, rho_out_w, form, march=(0, 0)):
    lad = np.ascontiguousarray(np.asarray(rho_in_nw, dtype=np.float64))
    sch = lbm_schedule()
    if lad.ndim == 2:
        if lad.shape[0] != n:
            raise ValueError("per-throat ladders need one row per throat")
        sch.per_throat = 1
    sch.n_incr = lad.shape[-1]
    sch.n_steps = int(n_steps)
    sch.rho_in_nw = lad.ctypes.data_as(_DP)
    sch.rho_out_w = float(rho_out_w)
    if form not in (BATCH_AUTO, BATCH_PERSISTENT, BATCH_PER_STEP, BATCH_CELLS, BATCH_MARCH):
        raise ValueError("form must be BATCH_AUTO, BATCH_PERSISTENT, BATCH_PER_STEP, BATCH_CELLS or BATCH_MARCH")
    sch.batch_form = int(form)
    sch.march_threads, sch.march_planes = int(march[0]), int(march[1])
    return sch, lad


def lbm_run_throat_batch(throats, params: lbm_params, rho_in_nw, n_steps: int, rho_out_w: float, stream=None,
                         form: int = 0, march=(0, 0)):
    """Batched per-throat drainage; returns (results: list of dict, rows: ThroatRows, a sequence whose
    item t is the list of throat t's rows as dicts).
    rho_in_nw: one ladder (n_incr,) for all throats, or one per throat (n, n_incr).
    form: BATCH_AUTO, BATCH_PERSISTENT, BATCH_PER_STEP, BATCH_CELLS or BATCH_MARCH.
    march: (threads per CTA, planes per chunk) of BATCH_MARCH, 0 for the defaults."""
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 3, 4))
    n = th.shape[0]
    sch, _lad = _batch_schedule(n, rho_in_nw, n_steps, rho_out_w, form, march)
    res = (lbm_throat_result * n)()
    rows = (lbm_increment * (n * sch.n_incr))()
    _check(load().lbm_run_throat_batch(th.ctypes.data_as(_DP), n, ctypes.byref(params), ctypes.byref(sch), res, rows,
                                       stream if stream is not None else _torch_stream()), "lbm_run_throat_batch")
    return [r.as_dict() for r in res], ThroatRows(rows, n, sch.n_incr)


def lbm_run_throat_batch_refined(throats, params: lbm_params, rho_in_nw, n_steps: int, rho_out_w: float,
                                 n_fine: int, stream=None, form: int = 0):
    """lbm_run_throat_batch plus the entry pressures refined to 1 / n_fine of a
    ladder step; returns (results, rows, p_ce_fine array)."""
    th = np.ascontiguousarray(np.asarray(throats, dtype=np.float64).reshape(-1, 3, 4))
    n = th.shape[0]
    sch, _lad = _batch_schedule(n, rho_in_nw, n_steps, rho_out_w, form)
    res = (lbm_throat_result * n)()
    rows = (lbm_increment * (n * sch.n_incr))()
    fine = np.empty(n)
    _check(load().lbm_run_throat_batch_refined(th.ctypes.data_as(_DP), n, ctypes.byref(params), ctypes.byref(sch),
                                               int(n_fine), res, rows, fine.ctypes.data_as(_DP),
                                               stream if stream is not None else _torch_stream()),
           "lbm_run_throat_batch_refined")
    return [r.as_dict() for r in res], ThroatRows(rows, n, sch.n_incr), fine


def lbm_destroy(h):
    if h:
        load().lbm_destroy(h)


def lbm_last_error() -> str:
    return load().lbm_last_error().decode()


class Domain:
    """Owning wrapper of one lbm_domain handle."""

    def __init__(self, params: lbm_params, spheres=None, box=None, mask=None, stream=None):
        if mask is not None:
            self.h = lbm_create_domain_mask(params, mask, stream)
        else:
            self.h = lbm_create_domain(params, spheres, box, stream)
        self.dims, self.n_fluid = lbm_get_dims(self.h)

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (nz, ny, nx)

    def set_densities(self, rho):
        lbm_set_densities(self.h, rho)

    def set_pressure_bc(self, rho_in_nw, rho_out_w):
        lbm_set_pressure_bc(self.h, rho_in_nw, rho_out_w)

    def step(self, n=1):
        lbm_step(self.h, n)

    def measure(self, allow_nonfinite=False):
        return lbm_measure(self.h, allow_nonfinite)

    def density(self):
        return lbm_get_density(self.h)

    def mask(self):
        return lbm_get_mask(self.h)

    def density_at(self, x, y, z):
        return lbm_get_density_at(self.h, x, y, z)

    def drainage(self, rho_in_nw, n_steps, rho_out_w, probe):
        return lbm_run_drainage(self.h, rho_in_nw, n_steps, rho_out_w, probe)

    def state(self):
        return lbm_get_state(self.h)

    def set_state(self, f, step):
        lbm_set_state(self.h, f, step)

    def set_tile(self, by, lz, lead):
        lbm_set_tile(self.h, by, lz, lead)

    def tile(self):
        return lbm_get_tile(self.h)

    def set_step_kernel(self, kind, lz=0):
        lbm_set_step_kernel(self.h, kind, lz)

    def step_kernel(self):
        return lbm_get_step_kernel(self.h)

    def set_push_shape(self, shape, lz=0):
        lbm_set_push_shape(self.h, shape, lz)

    def set_push_prefetch(self, planes):
        lbm_set_push_prefetch(self.h, planes)

    def set_push_order(self, order):
        lbm_set_push_order(self.h, order)

    def autotune(self, trial_steps=20):
        return lbm_autotune(self.h, trial_steps)

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


class Surrogate:
    """Ensemble MLP on the GPU (lbm_surrogate_* of the C ABI)."""

    def __init__(self, n_in, n_out, n_hidden=256, n_layers=4, n_members=5, half=False, seed=0, stream=None):
        cfg = lbm_surrogate_config(n_in, n_hidden, n_layers, n_out, n_members, int(bool(half)), int(seed))
        self.h = ctypes.c_void_p()
        _check(load().lbm_surrogate_create(ctypes.byref(cfg), stream if stream is not None else _torch_stream(),
                                           ctypes.byref(self.h)), "lbm_surrogate_create")
        self.n_in, self.n_out, self.n_members = n_in, n_out, n_members
        self.sizes = [n_in] + [n_hidden] * n_layers + [n_out]
        self.n_params = load().lbm_surrogate_num_params(self.h)

    def get_params(self, member):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(load().lbm_surrogate_get_params(self.h, member, out.ctypes.data_as(_FP)), "lbm_surrogate_get_params")
        return out

    def set_params(self, member, flat):
        a = _f32(flat)
        assert a.size == self.n_params
        _check(load().lbm_surrogate_set_params(self.h, member, a.ctypes.data_as(_FP)), "lbm_surrogate_set_params")

    def layers(self, flat):
        """Split a flat parameter vector into [(W, b), ...]."""
        out, off = [], 0
        for i in range(len(self.sizes) - 1):
            nin, nout = self.sizes[i], self.sizes[i + 1]
            W = flat[off:off + nin * nout].reshape(nout, nin)
            off += nin * nout
            b = flat[off:off + nout]
            off += nout
            out.append((W, b))
        return out

    def flatten(self, layers):
        return np.concatenate([np.concatenate([np.asarray(W).reshape(-1), np.asarray(b).reshape(-1)])
                               for W, b in layers]).astype(np.float32)

    def forward(self, member, X):
        X = _f32(X)
        Y = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        _check(load().lbm_surrogate_forward(self.h, member, X.ctypes.data_as(_FP), X.shape[0], Y.ctypes.data_as(_FP)),
               "lbm_surrogate_forward")
        return Y

    def gradients(self, member, X, T):
        X, T = _f32(X), _f32(T)
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        _check(load().lbm_surrogate_gradients(self.h, member, X.ctypes.data_as(_FP), T.ctypes.data_as(_FP),
                                              X.shape[0], g.ctypes.data_as(_FP), ctypes.byref(loss)),
               "lbm_surrogate_gradients")
        return g, loss.value

    def train(self, X, T, epochs, batch, lr, seed=0):
        X, T = _f32(X), _f32(T)
        losses = np.zeros(self.n_members * max(1, epochs))
        _check(load().lbm_surrogate_train(self.h, X.ctypes.data_as(_FP), T.ctypes.data_as(_FP), X.shape[0],
                                          int(epochs), int(batch), float(lr), int(seed),
                                          losses.ctypes.data_as(_DP)), "lbm_surrogate_train")
        return losses.reshape(self.n_members, max(1, epochs))

    def predict(self, X):
        X = _f32(X)
        mean = np.empty((X.shape[0], self.n_out), dtype=np.float32)
        spread = np.empty_like(mean)
        _check(load().lbm_surrogate_predict(self.h, X.ctypes.data_as(_FP), X.shape[0], mean.ctypes.data_as(_FP),
                                            spread.ctypes.data_as(_FP)), "lbm_surrogate_predict")
        return mean, spread

    def close(self):
        if getattr(self, "h", None):
            load().lbm_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
