"""FP64 CPU oracle of the two-component Shan-Chen D3Q19 step (test infrastructure).

This package is the independent checker of the CUDA library.  Only the tests,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import it;
the product path never does.  The arithmetic lives in ``sc_oracle.c`` (plain
loops, double precision, one cell at a time); this module only marshals numpy
arrays and runs the drainage ladder of Sec. 2.2.2 in plain Python.

Layouts: masks ``uint8[nz, ny, nx]``; densities ``float64[2, nz, ny, nx]``
(0 = wetting, 1 = non-wetting); populations ``float64[2, 19, nz, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

M_SOLID, M_ADHESIVE, M_MEMBRANE, M_INLET, M_OUTLET = 1, 2, 4, 8, 16
Q = 19


def build(force: bool = False) -> str:
    """Compile sc_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP over cells).

    -ffp-contract=off keeps every multiply and add separately rounded, so the
    voxeliser's sphere tests round the same way on x86-64 and aarch64.
    """
    os.makedirs(_LIB_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("periodic", ctypes.c_int * 3),
                ("tau", ctypes.c_double * 2),
                ("G", ctypes.c_double),
                ("G_ads", ctypes.c_double * 2),
                ("g", ctypes.c_double * 3),
                ("rho_in", ctypes.c_double * 2),
                ("rho_out", ctypes.c_double * 2)]


class Measurement(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double * 2),
                ("p_w", ctypes.c_double), ("p_nw", ctypes.c_double), ("p_c", ctypes.c_double),
                ("p_in", ctypes.c_double), ("p_out", ctypes.c_double), ("p_c_res", ctypes.c_double),
                ("S_w", ctypes.c_double),
                ("n_fluid", ctypes.c_longlong), ("n_w", ctypes.c_longlong),
                ("n_interface", ctypes.c_longlong), ("n_bulk_w", ctypes.c_longlong),
                ("n_bulk_nw", ctypes.c_longlong), ("n_in", ctypes.c_longlong),
                ("n_out", ctypes.c_longlong), ("n_nonfinite", ctypes.c_longlong),
                ("n_negative", ctypes.c_longlong)]

    def as_dict(self) -> dict:
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if name == "mass" else v
        return d


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            ip = ctypes.POINTER(ctypes.c_int)
            pp = ctypes.POINTER(Params)
            L.orc_lattice.argtypes = [ip, dp, ip]
            L.orc_equilibrium.argtypes = [ctypes.c_double, dp, dp]
            L.orc_init.argtypes = [pp, u8p, dp, dp]
            L.orc_density.argtypes = [pp, u8p, dp, dp]
            L.orc_force.argtypes = [pp, u8p, dp, dp]
            L.orc_step.argtypes = [pp, u8p, dp, ctypes.c_int]
            L.orc_step.restype = ctypes.c_int
            L.orc_measure.argtypes = [pp, u8p, dp, ctypes.POINTER(Measurement)]
            L.orc_velocity.argtypes = [pp, u8p, dp, dp]
            L.orc_voxelise.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, u8p]
            L.orc_throat_frame.argtypes = [dp, ip, dp, dp]
            L.orc_voxelise_throat.argtypes = [dp, u8p]
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


@dataclasses.dataclass
class Config:
    """Model parameters (lattice units).  Component 0 wets the grains, 1 does not."""
    shape: tuple  # (nz, ny, nx)
    tau: tuple = (1.0, 1.0)
    G: float = 0.9
    G_ads: tuple = (-0.3, 0.3)
    g: tuple = (0.0, 0.0, 0.0)
    periodic: tuple = (0, 0, 0)  # (x, y, z)
    rho_in: tuple = (0.06, 2.0)   # (w, nw) imposed on inlet cells
    rho_out: tuple = (2.0, 0.06)  # (w, nw) imposed on outlet cells

    def c(self) -> Params:
        nz, ny, nx = self.shape
        p = Params()
        p.nx, p.ny, p.nz = nx, ny, nz
        for i in range(3):
            p.periodic[i] = int(self.periodic[i])
            p.g[i] = float(self.g[i])
        for s in range(2):
            p.tau[s] = float(self.tau[s])
            p.G_ads[s] = float(self.G_ads[s])
            p.rho_in[s] = float(self.rho_in[s])
            p.rho_out[s] = float(self.rho_out[s])
        p.G = float(self.G)
        return p


# ------------------------------------------------------------------ lattice
def lattice():
    """(e[19,3] int, w[19], opposite[19]) as the oracle defines them."""
    e = np.zeros(57, dtype=np.int32)
    w = np.zeros(19)
    o = np.zeros(19, dtype=np.int32)
    lib().orc_lattice(e.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(w),
                      o.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return e.reshape(19, 3), w, o


def equilibrium(rho: float, u) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(19)
    lib().orc_equilibrium(float(rho), _dp(u), _dp(out))
    return out


# ----------------------------------------------------------------- geometry
def voxelise(shape, spheres, prism: bool = False, reservoirs: bool = False,
             membrane_layers: int = 0) -> np.ndarray:
    """Box-frame mask: cell (x,y,z) centred at (x,y,z); spheres n x (cx,cy,cz,r)."""
    nz, ny, nx = shape
    sp = np.ascontiguousarray(np.asarray(spheres, dtype=np.float64).reshape(-1, 4))
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    flags = (1 if prism else 0) | (2 if reservoirs else 0)
    lib().orc_voxelise(nx, ny, nz, _dp(sp), sp.shape[0], flags, int(membrane_layers), _u8(mask))
    return mask


def throat_frame(spheres3):
    sp = np.ascontiguousarray(np.asarray(spheres3, dtype=np.float64).reshape(3, 4))
    dims = np.zeros(3, dtype=np.int32)
    org = np.zeros(3)
    loc = np.zeros(12)
    lib().orc_throat_frame(_dp(sp), dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(org), _dp(loc))
    return tuple(int(v) for v in dims), org, loc.reshape(3, 4)


def voxelise_throat(spheres3) -> np.ndarray:
    dims, _, _ = throat_frame(spheres3)
    nx, ny, nz = dims
    sp = np.ascontiguousarray(np.asarray(spheres3, dtype=np.float64).reshape(3, 4))
    mask = np.zeros((nz, ny, nx), dtype=np.uint8)
    lib().orc_voxelise_throat(_dp(sp), _u8(mask))
    return mask


def throat_probe(spheres3, mask):
    """Probe cell of a throat box: the fluid cell of plane nz - 3 farthest from
    every sphere surface (max over cells of min_s |p - c_s| - r_s, the first in
    cell order on ties); (-1, -1, -1) when that plane holds no fluid."""
    dims, org, loc = throat_frame(spheres3)
    nx, ny, nz = dims
    k = nz - 3
    best, probe = -1e300, (-1, -1, -1)
    if k < 0:
        return probe
    for j in range(ny):
        for i in range(nx):
            if mask[k, j, i] & M_SOLID:
                continue
            p = (org[0] + float(i), org[1] + float(j), org[2] + float(k))
            dmin = 1e300
            for s in range(3):
                dx = p[0] - loc[s, 0]
                dy = p[1] - loc[s, 1]
                dz = p[2] - loc[s, 2]
                d = math.sqrt(dx * dx + dy * dy + dz * dz) - loc[s, 3]
                if d < dmin:
                    dmin = d
            if dmin > best:
                best, probe = dmin, (i, j, k)
    return probe


# -------------------------------------------------------------------- state
def init(cfg: Config, mask: np.ndarray, rho0: np.ndarray) -> np.ndarray:
    """Rest equilibrium of the initial densities rho0[2, nz, ny, nx]."""
    assert mask.shape == tuple(cfg.shape)
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    f = np.zeros((2, Q) + tuple(cfg.shape))
    p = cfg.c()
    lib().orc_init(ctypes.byref(p), _u8(np.ascontiguousarray(mask)), _dp(rho0), _dp(f))
    return f


def step(cfg: Config, mask: np.ndarray, f: np.ndarray, nsteps: int = 1) -> np.ndarray:
    """Advance f in place by nsteps time steps; returns f."""
    assert f.flags.c_contiguous and f.dtype == np.float64
    p = cfg.c()
    rc = lib().orc_step(ctypes.byref(p), _u8(np.ascontiguousarray(mask)), _dp(f), int(nsteps))
    if rc != 0:
        raise MemoryError("oracle step: allocation failed")
    return f


def density(cfg: Config, mask: np.ndarray, f: np.ndarray) -> np.ndarray:
    rho = np.zeros((2,) + tuple(cfg.shape))
    p = cfg.c()
    lib().orc_density(ctypes.byref(p), _u8(np.ascontiguousarray(mask)), _dp(np.ascontiguousarray(f)), _dp(rho))
    return rho


def force(cfg: Config, mask: np.ndarray, rho: np.ndarray) -> np.ndarray:
    """Total force per component, F[2, 3, nz, ny, nx] (cohesion + adhesion + body)."""
    F = np.zeros((2, 3) + tuple(cfg.shape))
    p = cfg.c()
    lib().orc_force(ctypes.byref(p), _u8(np.ascontiguousarray(mask)),
                    _dp(np.ascontiguousarray(rho, dtype=np.float64)), _dp(F))
    return F


def velocity(cfg: Config, mask: np.ndarray, f: np.ndarray) -> np.ndarray:
    u = np.zeros((3,) + tuple(cfg.shape))
    p = cfg.c()
    lib().orc_velocity(ctypes.byref(p), _u8(np.ascontiguousarray(mask)), _dp(np.ascontiguousarray(f)), _dp(u))
    return u


def measure(cfg: Config, mask: np.ndarray, f: np.ndarray) -> dict:
    m = Measurement()
    p = cfg.c()
    lib().orc_measure(ctypes.byref(p), _u8(np.ascontiguousarray(mask)), _dp(np.ascontiguousarray(f)),
                      ctypes.byref(m))
    return m.as_dict()


def pressure(cfg: Config, rho: np.ndarray) -> np.ndarray:
    """Eq. 5: p = (rho_w + rho_nw)/3 + G rho_w rho_nw / 3."""
    return (rho[0] + rho[1]) / 3.0 + cfg.G * rho[0] * rho[1] / 3.0


# ----------------------------------------------------------------- drainage
def entry_pressure(p_c_series, invaded_at):
    """p_c^e = largest p_c reached up to and including the invasion increment
    (Sec. 2.2.2: the maximum p_c during invasion); the first maximiser wins ties.
    Returns (p_c^e, index) or (inf, -1) when the throat was never invaded."""
    if invaded_at is None or invaded_at < 0:
        return math.inf, -1
    best, arg = -math.inf, -1
    for i in range(invaded_at + 1):
        v = p_c_series[i]
        if v == v and v > best:  # NaN never wins
            best, arg = v, i
    return best, arg


def drainage(cfg: Config, mask: np.ndarray, f: np.ndarray, ladder_nw, n_steps: int, probe):
    """Pressure ladder of Sec. 2.2.2: for each inlet non-wetting density in
    ``ladder_nw`` set the reservoir, run n_steps, measure.  Invasion is the first
    increment after which phi < 0 at the probe cell (x, y, z).  Returns a dict
    with the per-increment measurements, the invasion index and p_c^e."""
    rows = []
    invaded = -1
    px, py, pz = probe
    for i, rin in enumerate(ladder_nw):
        c = dataclasses.replace(cfg, rho_in=(cfg.rho_in[0], float(rin)))
        step(c, mask, f, n_steps)
        m = measure(c, mask, f)
        rho = density(c, mask, f)
        rw, rn = rho[0, pz, py, px], rho[1, pz, py, px]
        phi = (rw - rn) / (rw + rn) if (rw + rn) != 0 else 0.0
        m["phi_probe"] = phi
        rows.append(m)
        if invaded < 0 and phi < 0.0:
            invaded = i
    pce, arg = entry_pressure([r["p_c"] for r in rows], invaded)
    return {"rows": rows, "invaded_at": invaded, "p_ce": pce, "p_ce_index": arg}
