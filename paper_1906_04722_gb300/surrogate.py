"""Throat surrogate: binding of lbm_throat_surrogate_* and its helpers.

The hybrid method needs, for every pore throat, the entry capillary pressure
p_c^e and the drainage curve of that throat (Sec. 2.2.2), each from one LBM run.
The library learns the map from a throat's geometry to those outputs on throats
the batched LBM has simulated, predicts new throats with an ensemble, and sends
every throat whose ensemble members disagree on p_c^e by more than a relative
spread threshold back to the batched LBM.  Inputs, standardisation, targets,
the spread rule and the fallback run in the library (include/lbm.h); this
module only marshals arrays.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import (_DP, _FP, _IP, LbmError, _check, _torch_stream, lbm_increment, lbm_params, lbm_schedule,
               lbm_throat_incircle, lbm_throat_result, lbm_throat_surrogate_config, load)

N_INPUTS = 24  # LBM_SURROGATE_INPUTS


def contact_angle_estimate(g_ads_w: float, g_ads_nw: float, G: float, rho_major: float, rho_minor: float) -> float:
    """Contact angle of the wall adhesion in radians (lbm_contact_angle_estimate)."""
    out = ctypes.c_double()
    _check(load().lbm_contact_angle_estimate(float(g_ads_w), float(g_ads_nw), float(G), float(rho_major),
                                             float(rho_minor), ctypes.byref(out)), "lbm_contact_angle_estimate")
    return out.value


def surrogate_inputs(triples, theta: float):
    """n x N_INPUTS network inputs (float32) and the mean radii (lbm_throat_surrogate_inputs)."""
    t = np.ascontiguousarray(np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4))
    X = np.empty((t.shape[0], N_INPUTS), dtype=np.float32)
    R = np.empty(t.shape[0])
    _check(load().lbm_throat_surrogate_inputs(t.ctypes.data_as(_DP), t.shape[0], float(theta), X.ctypes.data_as(_FP),
                                              R.ctypes.data_as(_DP)), "lbm_throat_surrogate_inputs")
    return X, R


def throat_incircle(triples) -> np.ndarray:
    """Inscribed-circle radius of each throat (lbm_throat_incircle): the largest
    clearance over the triangle of the three centres, 0 where the spheres close
    the throat."""
    return lbm_throat_incircle(triples)


def pressure_ladder(r_in, n_incr, lo, hi, rho_major, rho_minor, G) -> np.ndarray:
    """Per-throat reservoir ladders, n x n_incr inlet densities (lbm_pressure_ladder)."""
    r = np.ascontiguousarray(np.asarray(r_in, dtype=np.float64).reshape(-1))
    out = np.empty((r.shape[0], int(n_incr)))
    _check(load().lbm_pressure_ladder(r.ctypes.data_as(_DP), r.shape[0], int(n_incr), float(lo), float(hi),
                                      float(rho_major), float(rho_minor), float(G), out.ctypes.data_as(_DP)),
           "lbm_pressure_ladder")
    return out


def _schedule(rho_in_nw, n, n_steps, rho_out_w):
    lad = np.ascontiguousarray(np.asarray(rho_in_nw, dtype=np.float64))
    sch = lbm_schedule()
    sch.per_throat = 1 if lad.ndim == 2 else 0
    if lad.ndim == 2 and lad.shape[0] != n:
        raise ValueError("per-throat ladders need one row per throat")
    sch.n_incr = lad.shape[-1]
    sch.n_steps = int(n_steps)
    sch.rho_in_nw = lad.ctypes.data_as(_DP)
    sch.rho_out_w = float(rho_out_w)
    return sch, lad


class ThroatSurrogate:
    """Ensemble surrogate of the per-throat LBM drainage (lbm_throat_surrogate_*)."""

    def __init__(self, n_incr: int, theta: float, n_members: int = 5, n_hidden: int = 256, n_layers: int = 4,
                 half: bool = False, seed: int = 0, spread_tol: float = 0.02, stream=None):
        cfg = lbm_throat_surrogate_config(int(n_incr), int(n_members), int(n_hidden), int(n_layers), int(bool(half)),
                                          int(seed), float(theta))
        self.h = ctypes.c_void_p()
        _check(load().lbm_throat_surrogate_create(ctypes.byref(cfg), stream if stream is not None else _torch_stream(),
                                                  ctypes.byref(self.h)), "lbm_throat_surrogate_create")
        self.n_incr, self.n_members, self.theta = int(n_incr), int(n_members), float(theta)
        self.spread_tol = spread_tol

    def fit(self, triples, results, rows, epochs=200, batch=256, lr=1e-3, seed=0):
        """Train on throats and their lbm_run_throat_batch outcome (results: list
        of dicts, rows: list of lists of dicts); returns the epoch losses
        (members x epochs) and the number of throats used."""
        t = np.ascontiguousarray(np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4))
        n = t.shape[0]
        res = (lbm_throat_result * n)()
        rw = (lbm_increment * (n * self.n_incr))()
        for i in range(n):
            r = results[i]
            res[i].p_ce, res[i].invaded_at, res[i].n_fluid = r["p_ce"], r["invaded_at"], r["n_fluid"]
            for k in range(self.n_incr):
                for name, _ in lbm_increment._fields_:
                    setattr(rw[i * self.n_incr + k], name, rows[i][k][name])
        losses = np.zeros(self.n_members * max(1, epochs))
        used = ctypes.c_int()
        _check(load().lbm_throat_surrogate_fit(self.h, t.ctypes.data_as(_DP), n, res, rw, int(epochs), int(batch),
                                               float(lr), int(seed), losses.ctypes.data_as(_DP), ctypes.byref(used)),
               "lbm_throat_surrogate_fit")
        return losses.reshape(self.n_members, max(1, epochs)), used.value

    def predict(self, triples):
        """p_c^e, its relative ensemble spread and the S_w curves of each throat."""
        t = np.ascontiguousarray(np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4))
        n = t.shape[0]
        pce, rel = np.empty(n), np.empty(n)
        curves = np.empty((n, self.n_incr), dtype=np.float32)
        _check(load().lbm_throat_surrogate_predict(self.h, t.ctypes.data_as(_DP), n, pce.ctypes.data_as(_DP),
                                                   rel.ctypes.data_as(_DP), curves.ctypes.data_as(_FP)),
               "lbm_throat_surrogate_predict")
        return pce, rel, curves

    def predict_with_fallback(self, triples, params: lbm_params, rho_in_nw, n_steps, rho_out_w):
        """Surrogate for confident throats, batched LBM for the rest.  Returns
        (p_ce, used_lbm mask, seconds in the network, seconds in the LBM)."""
        t = np.ascontiguousarray(np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4))
        n = t.shape[0]
        sch, _lad = _schedule(rho_in_nw, n, n_steps, rho_out_w)
        pce = np.empty(n)
        used = np.empty(n, dtype=np.int32)
        sec = np.zeros(2)
        _check(load().lbm_throat_surrogate_predict_with_fallback(self.h, t.ctypes.data_as(_DP), n,
                                                                 float(self.spread_tol), ctypes.byref(params),
                                                                 ctypes.byref(sch), pce.ctypes.data_as(_DP),
                                                                 used.ctypes.data_as(_IP), sec.ctypes.data_as(_DP)),
               "lbm_throat_surrogate_predict_with_fallback")
        return pce, used.astype(bool), float(sec[0]), float(sec[1])

    def scaling(self):
        x_mu, x_sd = np.empty(N_INPUTS), np.empty(N_INPUTS)
        y_mu, y_sd = np.empty(1 + self.n_incr), np.empty(1 + self.n_incr)
        _check(load().lbm_throat_surrogate_scaling(self.h, x_mu.ctypes.data_as(_DP), x_sd.ctypes.data_as(_DP),
                                                   y_mu.ctypes.data_as(_DP), y_sd.ctypes.data_as(_DP)),
               "lbm_throat_surrogate_scaling")
        return x_mu, x_sd, y_mu, y_sd

    def close(self):
        if getattr(self, "h", None):
            load().lbm_throat_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["N_INPUTS", "ThroatSurrogate", "contact_angle_estimate", "surrogate_inputs", "throat_incircle",
           "pressure_ladder", "LbmError"]
