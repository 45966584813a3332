"""Throat surrogate: an ensemble MLP standing in for the per-throat LBM runs.

The hybrid method needs, for every pore throat, the entry capillary pressure
p_c^e and the drainage curve of that throat (Sec. 2.2.2), each from one LBM run.
This module learns the map from a throat's geometry to those outputs on throats
the batched LBM has simulated, predicts new throats with an ensemble, and sends
every throat whose ensemble members disagree on p_c^e by more than a relative
spread threshold back to the batched LBM (the fallback against which the
network's error is also measured).  Host-side glue only: the LBM runs in lbm_run_throat_batch and
the network in the lbm_surrogate_* kernels.

Inputs per throat (24): the three radii and the three centre distances divided
by the mean radius R, spheres ordered by decreasing radius, and the contact
angle in radians (7); what the lattice makes of the throat box
(lbm_throat_lattice_features: its size, fluid fraction, the narrowest sections'
areas, lattice incircles and perimeter, 14); and three of those lengths over R.
The lattice part matters: the entry pressure follows the narrowest section as
the voxelised box resolves it, which the continuous geometry alone does not fix.
Outputs (1 + n_incr): p_c^e R (the capillary pressure made dimensionless by the
throat size, standardised) and the throat's S_w after each pressure increment.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import Surrogate, lbm_run_throat_batch, lbm_throat_lattice_features


def contact_angle_estimate(g_ads_w: float, g_ads_nw: float, G: float, rho_major: float, rho_minor: float) -> float:
    """Contact angle of the wall adhesion (Huang et al. 2007 estimate, radians):
    cos(theta) = (G_ads,nw - G_ads,w) / (G (rho_major - rho_minor) / 2)."""
    c = (g_ads_nw - g_ads_w) / (G * (rho_major - rho_minor) / 2.0)
    return math.acos(max(-1.0, min(1.0, c)))


def throat_features(triples: np.ndarray, theta: float) -> np.ndarray:
    """n x 7 feature matrix (see the module docstring) and the mean radii."""
    t = np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4)
    order = np.argsort(-t[:, :, 3], axis=1, kind="stable")
    t = np.take_along_axis(t, order[:, :, None], axis=1)
    r = t[:, :, 3]
    R = r.mean(axis=1)
    c = t[:, :, :3]
    d01 = np.linalg.norm(c[:, 0] - c[:, 1], axis=1)
    d12 = np.linalg.norm(c[:, 1] - c[:, 2], axis=1)
    d02 = np.linalg.norm(c[:, 0] - c[:, 2], axis=1)
    X = np.c_[r / R[:, None], d01 / R, d12 / R, d02 / R, np.full(len(t), theta)]
    return X.astype(np.float32), R


N_INPUTS = 24


def surrogate_inputs(triples, theta: float):
    """n x N_INPUTS network inputs (see the module docstring) and the mean radii."""
    X, R = throat_features(triples, theta)
    L = lbm_throat_lattice_features(triples)
    return np.c_[X, L, L[:, [5, 8, 9]] / R[:, None]].astype(np.float32), R


def throat_incircle(triples) -> np.ndarray:
    """Radius (lattice units) of the widest circle in the plane of a throat's
    three centres, inside their triangle, that stays clear of the three spheres:
    the constriction the non-wetting fluid has to pass (Sec. 2.2.2), whose entry
    pressure scales as its inverse (Young-Laplace).  Maximises
    min_k(|p - c_k| - r_k) over the triangle: a barycentric grid, then two local
    refinements; 0 where the spheres close the throat."""
    t = np.asarray(triples, dtype=np.float64).reshape(-1, 3, 4)
    n = len(t)
    c, r = t[:, :, :3], t[:, :, 3]
    e1 = c[:, 1] - c[:, 0]
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    w = c[:, 2] - c[:, 0]
    e2 = w - (w * e1).sum(axis=1, keepdims=True) * e1
    e2 /= np.linalg.norm(e2, axis=1, keepdims=True)
    # centres in the plane's 2-D frame
    q = np.stack([((c - c[:, :1]) * e1[:, None]).sum(-1), ((c - c[:, :1]) * e2[:, None]).sum(-1)], axis=-1)

    def clearance(pts):  # n x m x 2
        d = np.linalg.norm(pts[:, :, None, :] - q[:, None, :, :], axis=-1) - r[:, None, :]
        return d.min(axis=2)

    def search(lam):  # lam: n x m x 3 barycentric weights (>= 0, summing to 1)
        pts = np.einsum("nmk,nkd->nmd", lam, q)
        val = clearance(pts)
        k = val.argmax(axis=1)
        return lam[np.arange(n), k], val[np.arange(n), k]

    N = 48
    ij = np.array([(a, b) for a in range(N + 1) for b in range(N + 1 - a)], dtype=np.float64) / N
    lam0 = np.stack([ij[:, 0], ij[:, 1], 1.0 - ij[:, 0] - ij[:, 1]], axis=-1)
    best, val = search(np.broadcast_to(lam0, (n,) + lam0.shape))
    h = 1.0 / N
    g = np.linspace(-1.0, 1.0, 21)
    da, db = np.meshgrid(g, g, indexing="ij")
    for _ in range(2):
        la = best[:, None, 0] + h * da.ravel()[None]
        lb = best[:, None, 1] + h * db.ravel()[None]
        lam = np.stack([la, lb, 1.0 - la - lb], axis=-1)
        lam = np.clip(lam, 0.0, None)
        lam /= lam.sum(axis=-1, keepdims=True)
        best, val = search(lam)
        h /= 10.0
    return np.maximum(val, 0.0)


def pressure_ladder(r_in, n_incr, lo, hi, rho_major, rho_minor, G):
    """Per-throat reservoir ladders: n_incr inlet densities per throat whose
    reservoir pressure differences p_c,res span [lo, hi] / r_in (Eq. 5 at the
    inlet and outlet layers: p_c,res = (rho_in - rho_major) (1 + G rho_minor) / 3)."""
    r_in = np.maximum(np.asarray(r_in, dtype=np.float64), 0.5)
    pc = np.linspace(lo, hi, n_incr)[None, :] / r_in[:, None]
    return rho_major + 3.0 * pc / (1.0 + G * rho_minor)


class ThroatSurrogate:
    """Ensemble surrogate of the per-throat LBM drainage."""

    def __init__(self, n_incr: int, n_members: int = 5, n_hidden: int = 256, n_layers: int = 4, half: bool = False,
                 seed: int = 0, spread_tol: float = 0.02):
        self.n_incr = n_incr
        self.net = Surrogate(N_INPUTS, 1 + n_incr, n_hidden=n_hidden, n_layers=n_layers, n_members=n_members, half=half,
                             seed=seed)
        self.spread_tol = spread_tol
        self.x_mu = self.x_sd = None
        self.y_mu = self.y_sd = None

    @staticmethod
    def targets(results, rows, R):
        """(n x (1 + n_incr)) targets from LBM results; rows of throats that never
        invaded are flagged in the returned mask."""
        pce = np.array([r["p_ce"] for r in results])
        ok = np.isfinite(pce)
        sw = np.array([[row["S_w"] for row in rr] for rr in rows])
        Y = np.c_[np.where(ok, pce, 0.0) * R, sw]
        return Y, ok

    def fit(self, X, Y, epochs=200, batch=256, lr=1e-3, seed=0):
        X = np.asarray(X, dtype=np.float64)
        Y = np.asarray(Y, dtype=np.float64)
        self.x_mu, self.x_sd = X.mean(axis=0), X.std(axis=0) + 1e-6
        self.y_mu, self.y_sd = Y.mean(axis=0), Y.std(axis=0) + 1e-6
        Xn = (X - self.x_mu) / self.x_sd
        Yn = (Y - self.y_mu) / self.y_sd
        return self.net.train(Xn, Yn, epochs=epochs, batch=batch, lr=lr, seed=seed)

    def predict(self, X, R):
        """p_c^e (absolute), its relative ensemble spread, and the S_w curves."""
        Xn = (np.asarray(X, dtype=np.float64) - self.x_mu) / self.x_sd
        mean, spread = self.net.predict(Xn)
        mean = mean * self.y_sd + self.y_mu
        spread = spread * self.y_sd
        pce = mean[:, 0] / R
        rel = np.abs(spread[:, 0]) / np.maximum(np.abs(mean[:, 0]), 1e-12)
        return pce, rel, mean[:, 1:]

    def predict_with_fallback(self, triples, theta, params, rho_in_nw, n_steps, rho_out_w):
        """Surrogate for confident throats, batched LBM for the rest.  Returns
        (p_ce, used_lbm mask, seconds in the network, seconds in the LBM)."""
        t0 = time.perf_counter()
        X, R = surrogate_inputs(triples, theta)
        pce, rel, _ = self.predict(X, R)
        t_net = time.perf_counter() - t0
        fall = rel > self.spread_tol
        t_lbm = 0.0
        if fall.any():
            t0 = time.perf_counter()
            lad = np.asarray(rho_in_nw)
            res, _ = lbm_run_throat_batch(np.asarray(triples)[fall], params, lad[fall] if lad.ndim == 2 else lad,
                                          n_steps, rho_out_w)
            t_lbm = time.perf_counter() - t0
            pce = pce.copy()
            pce[fall] = [r["p_ce"] for r in res]
        return pce, fall, t_net, t_lbm
