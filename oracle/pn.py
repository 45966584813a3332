"""Plain pore-network drainage and throat incircle (test infrastructure).

Only the tests import this module; the product path never does.  It restates
the drainage of Sec. 2.2.2 / Sec. 3.1.1 the slow way, in plain Python: at every
step it scans all throats for the lowest entry pressure the non-wetting fluid
can pass, and after every invasion it recomputes which wetting pores still
reach the wetting reservoir by a flood over the network.

Network convention: throats are (a, b) pairs, a a pore index, b a pore index or
INLET (-1, the non-wetting reservoir) or OUTLET (-2, the wetting reservoir
behind the membrane, which the non-wetting fluid never enters).
"""
from __future__ import annotations

import math

import numpy as np

INLET, OUTLET = -1, -2


def trapped_pores(state, throats):
    """Wetting pores with no path of wetting pores to the wetting reservoir."""
    n = len(state)
    reach = [False] * n
    stack = [a for (a, b) in throats if b == OUTLET and state[a] == "w"]
    for a in stack:
        reach[a] = True
    while stack:
        u = stack.pop()
        for (a, b) in throats:
            for (x, y) in ((a, b), (b, a)):
                if x == u and y >= 0 and not reach[y] and state[y] == "w":
                    reach[y] = True
                    stack.append(y)
    return [i for i in range(n) if state[i] == "w" and not reach[i]]


def drainage(volume, throats, pce, levels):
    """Quasi-static drainage: at level l the non-wetting fluid passes, one throat
    at a time and lowest entry pressure first (ties: lower throat index, then
    lower pore), every throat with p_c^e < levels[l] from a non-wetting pore or
    the inlet into a wetting pore; trapped wetting pores are never entered.
    Returns (S_w per level, invaded_at per pore, trapped_at per pore)."""
    n = len(volume)
    state = ["w"] * n
    invaded_at, trapped_at = [-1] * n, [-1] * n
    for i in trapped_pores(state, throats):
        state[i], trapped_at[i] = "t", 0
    vtot = sum(volume)
    S_w = []
    for l, pc in enumerate(levels):
        while True:
            best = None
            for i, (a, b) in enumerate(throats):
                for (u, v) in ((a, b), (b, a)):
                    if v < 0 or state[v] != "w":
                        continue
                    if not (u == INLET or (u >= 0 and state[u] == "n")):
                        continue
                    if pce[i] < pc:
                        key = (pce[i], i, v)
                        if best is None or key < best:
                            best = key
            if best is None:
                break
            v = best[2]
            state[v], invaded_at[v] = "n", l
            for i in trapped_pores(state, throats):
                state[i], trapped_at[i] = "t", l
        vw = sum(volume[i] for i in range(n) if state[i] != "n")
        S_w.append(vw / vtot)
    return S_w, invaded_at, trapped_at


def incircle_search(spheres3, grid: int = 400):
    """Inscribed circle of a throat by search: in the plane of the three centres,
    the largest min_i(|p - c_i| - r_i) over points p of their triangle (the
    circle touching the three sphere sections), maximised on a grid and refined
    by shrinking the search window around the best point."""
    s = np.asarray(spheres3, dtype=float).reshape(3, 4)
    c, r = s[:, :3], s[:, 3]
    e1 = (c[1] - c[0]) / np.linalg.norm(c[1] - c[0])
    n = np.cross(c[1] - c[0], c[2] - c[0])
    n /= np.linalg.norm(n)
    e2 = np.cross(n, e1)
    P = np.stack([[(ci - c[0]) @ e1, (ci - c[0]) @ e2] for ci in c])

    def f(x, y):
        d = np.stack([np.hypot(x - P[i, 0], y - P[i, 1]) - r[i] for i in range(3)])
        return d.min(axis=0)

    def inside(x, y):
        def side(i, j):
            return (P[j, 0] - P[i, 0]) * (y - P[i, 1]) - (P[j, 1] - P[i, 1]) * (x - P[i, 0])
        s0, s1, s2 = side(0, 1), side(1, 2), side(2, 0)
        return ((s0 >= 0) & (s1 >= 0) & (s2 >= 0)) | ((s0 <= 0) & (s1 <= 0) & (s2 <= 0))

    lo, hi = P.min(axis=0), P.max(axis=0)
    best_v, best_p = -math.inf, None
    for _ in range(12):
        xs = np.linspace(lo[0], hi[0], grid)
        ys = np.linspace(lo[1], hi[1], grid)
        X, Y = np.meshgrid(xs, ys)
        V = np.where(inside(X, Y), f(X, Y), -np.inf)
        k = np.unravel_index(np.argmax(V), V.shape)
        if V[k] > best_v:
            best_v, best_p = float(V[k]), (X[k], Y[k])
        span = (hi - lo) / 8.0
        lo = np.array(best_p) - span
        hi = np.array(best_p) + span
    return best_v


def _throat_plane(spheres3):
    """Centres of a throat in the plane through them (counter-clockwise) and radii."""
    s = np.asarray(spheres3, dtype=float).reshape(3, 4)
    c, r = s[:, :3], s[:, 3]
    e1 = (c[1] - c[0]) / np.linalg.norm(c[1] - c[0])
    n = np.cross(c[1] - c[0], c[2] - c[0])
    n /= np.linalg.norm(n)
    e2 = np.cross(n, e1)
    P = np.stack([[(ci - c[0]) @ e1, (ci - c[0]) @ e2] for ci in c])
    return P, r


def msp_terms_raster(spheres3, r, cos_theta, h):
    """A_nw, L_nw, L_ns of the Mayer-Stowe-Princen construction (Sec. 1 cites
    MS-P) by brute force on a pixel grid of spacing h, for a throat taken as a
    prism with neutral side walls: the section is the triangle T of the centres
    minus the sphere sections; meniscus discs of radius r may be centred at any
    point of T at a distance of at least sqrt(R_i^2 + r^2 + 2 R_i r cos(theta))
    from every centre (so that a disc cuts grain i at the contact angle); the
    non-wetting region is what those discs cover of the section.  A_nw counts
    its pixels; L_nw is the length of the level set {distance to the allowed
    centres = r} inside the section (coarea formula, a band of width 8 h);
    L_ns the measure of grain-circle points inside T within r of an allowed
    centre (circles sampled densely).  No arcs, no case analysis."""
    from scipy import ndimage
    from scipy.spatial import cKDTree

    P, R = _throat_plane(spheres3)
    lo, hi = P.min(axis=0) - 2 * h, P.max(axis=0) + 2 * h
    xs = np.arange(lo[0], hi[0], h)
    ys = np.arange(lo[1], hi[1], h)
    X, Y = np.meshgrid(xs, ys)

    def in_T(x, y):
        def side(i, j):
            return (P[j, 0] - P[i, 0]) * (y - P[i, 1]) - (P[j, 1] - P[i, 1]) * (x - P[i, 0])
        return (side(0, 1) >= 0) & (side(1, 2) >= 0) & (side(2, 0) >= 0)

    inT = in_T(X, Y)
    dist_c = [np.hypot(X - P[i, 0], Y - P[i, 1]) for i in range(3)]
    grain = (dist_c[0] < R[0]) | (dist_c[1] < R[1]) | (dist_c[2] < R[2])
    rho = np.sqrt(R * R + r * r + 2 * R * r * cos_theta)
    allowed = inT & (dist_c[0] >= rho[0]) & (dist_c[1] >= rho[1]) & (dist_c[2] >= rho[2])
    if not allowed.any():
        return 0.0, 0.0, 0.0
    d = ndimage.distance_transform_edt(~allowed, sampling=h)
    pore = inT & ~grain
    a_nw = float((pore & (d <= r)).sum()) * h * h
    eps = 8 * h
    l_nw = float((pore & (np.abs(d - r) < eps / 2)).sum()) * h * h / eps
    tree = cKDTree(np.column_stack([X[allowed], Y[allowed]]))
    l_ns = 0.0
    for i in range(3):
        t = np.linspace(0.0, 2 * np.pi, 40000, endpoint=False)
        px, py = P[i, 0] + R[i] * np.cos(t), P[i, 1] + R[i] * np.sin(t)
        keep = in_T(px, py)
        for j in range(3):
            if j != i:
                keep &= np.hypot(px - P[j, 0], py - P[j, 1]) >= R[j]
        if not keep.any():
            continue
        dd, _ = tree.query(np.column_stack([px[keep], py[keep]]))
        l_ns += R[i] * 2 * np.pi * float((dd <= r + 0.5 * h).sum()) / len(t)
    return a_nw, l_nw, l_ns


def msp_radius_raster(spheres3, cos_theta, h, r_hi):
    """Meniscus radius of the MS-P condition A_nw = r (L_nw + L_ns cos(theta)),
    by bisection on [0, r_hi] over msp_terms_raster."""
    lo, hi = 0.0, float(r_hi)
    for _ in range(22):
        mid = 0.5 * (lo + hi)
        a, lnw, lns = msp_terms_raster(spheres3, mid, cos_theta, h)
        if a - mid * (lnw + lns * cos_theta) > 0:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)
