"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws sphere packings,
initial density fields, pressure ladders and throat triples from fixed seeds.
Both the CUDA library and the FP64 oracle take these as inputs and build
everything else (masks, frames, populations) themselves.

Workloads (lattice units):
  * throat32   -- one pore throat: 32^3 box, three touching spheres of radius 10
                  on an equilateral triangle of side 20 around the z axis,
                  prism clip, inlet layer z = 0 (non-wetting reservoir), outlet
                  layer z = 31 (wetting reservoir), 500 steps with the inlet
                  density raised by 0.01 every 25 steps.
  * sample192  -- fully resolved drainage sample: 192^3 box, 300 non-overlapping
                  spheres with radii uniform in [10, 14] placed by seeded random
                  sequential addition, inlet z = 0, 3 membrane layers above the
                  outlet layer z = 191.
  * throats    -- pore throats (sphere triples) from a Delaunay tetrahedralisation
                  of a seeded packing's centres: the facets of the tetrahedra.
"""
from __future__ import annotations

import math

import numpy as np

RHO_MAJOR = 2.0
RHO_MINOR = 0.06
G_COHESION = 0.9
G_ADS = (-0.3, 0.3)   # (wetting, non-wetting)
TAU = (1.0, 1.0)


# ------------------------------------------------------------- throat32
def throat32_spheres() -> np.ndarray:
    """Three touching spheres, r = 10, centres on an equilateral triangle of
    side 20 whose circumcentre is (16, 16), all at z = 16."""
    R = 20.0 / math.sqrt(3.0)
    out = []
    for a in (90.0, 210.0, 330.0):
        t = math.radians(a)
        out.append((16.0 + R * math.cos(t), 16.0 + R * math.sin(t), 16.0, 10.0))
    return np.array(out)


def throat32_ladder(n_incr: int = 20, d_rho: float = 0.01):
    """Inlet non-wetting densities: rho_major + i * d_rho, i = 0..n_incr-1."""
    return [RHO_MAJOR + i * d_rho for i in range(n_incr)]


def initial_densities(shape, rho_in_nw: float = RHO_MAJOR, noise: float = 0.0, seed: int = 1,
                      inlet_layer: bool = True) -> np.ndarray:
    """Initial (rho_w, rho_nw)[2, nz, ny, nx]: wetting fluid fills the box; the
    z = 0 layer holds the non-wetting reservoir (rho_nw = rho_in_nw, rho_w =
    rho_minor).  Optional multiplicative noise (1 + noise * N(0,1)), seeded.
    Values at solid cells are ignored by both sides."""
    nz, ny, nx = shape
    rho = np.empty((2, nz, ny, nx))
    rho[0] = RHO_MAJOR
    rho[1] = RHO_MINOR
    if inlet_layer:
        rho[0, 0] = RHO_MINOR
        rho[1, 0] = rho_in_nw
    if noise:
        rng = np.random.default_rng(seed)
        rho *= 1.0 + noise * rng.standard_normal(rho.shape)
    return rho


def droplet_densities(shape, center, radius, seed: int = 0, noise: float = 1e-3) -> np.ndarray:
    """A non-wetting droplet in wetting fluid (closed or periodic boxes)."""
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    r = np.sqrt((x - center[0]) ** 2 + (y - center[1]) ** 2 + (z - center[2]) ** 2)
    inside = r < radius
    rho = np.stack([np.where(inside, RHO_MINOR, RHO_MAJOR), np.where(inside, RHO_MAJOR, RHO_MINOR)])
    if noise:
        rng = np.random.default_rng(seed)
        rho = rho * (1.0 + noise * rng.standard_normal(rho.shape))
    return rho


# --------------------------------------------------------------- packings
def rsa_packing(n: int, box, rmin: float, rmax: float, seed: int, z_margin=(0.0, 0.0),
                max_tries: int = 2_000_000) -> np.ndarray:
    """Random sequential addition: draw r ~ U[rmin, rmax] and a centre uniform in
    [r, L - r] per axis (z additionally kept z_margin away from the two ends),
    accept when it overlaps no earlier sphere.  Returns n x (cx, cy, cz, r)."""
    rng = np.random.default_rng(seed)
    L = np.asarray(box, dtype=float)
    cell = 2.0 * rmax
    grid = {}
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"RSA stalled after {len(out)} spheres")
        r = rng.uniform(rmin, rmax)
        lo = np.array([r, r, r + z_margin[0]])
        hi = L - np.array([r, r, r + z_margin[1]])
        c = lo + rng.uniform(size=3) * (hi - lo)
        key = tuple((c // cell).astype(int))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        o = out[j]
                        if (c[0] - o[0]) ** 2 + (c[1] - o[1]) ** 2 + (c[2] - o[2]) ** 2 < (r + o[3]) ** 2:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            grid.setdefault(key, []).append(len(out))
            out.append((c[0], c[1], c[2], r))
    return np.array(out)


def sample192_spheres(seed: int = 2) -> np.ndarray:
    """300 spheres, radii U[10, 14], in a 192^3 box; centres kept 2 layers clear
    of the inlet end and 5 of the outlet end (reservoir and membrane layers)."""
    return rsa_packing(300, (192, 192, 192), 10.0, 14.0, seed, z_margin=(2.0, 5.0))


def sample_spheres(edge: int, seed: int = 2) -> np.ndarray:
    """The drainage-sample recipe at another box edge: the sphere count scales
    with the box volume (300 at 192^3), same radii, same margins."""
    if edge == 192:
        return sample192_spheres(seed)
    n = max(1, int(round(300 * (edge / 192.0) ** 3)))
    return rsa_packing(n, (edge, edge, edge), 10.0, 14.0, seed, z_margin=(2.0, 5.0))


def delaunay_throats(spheres: np.ndarray, n: int, seed: int, max_edge: float = 64.0):
    """Throats as sphere triples: the triangular facets of a Delaunay
    tetrahedralisation of the centres that two tetrahedra share, whose longest
    centre-to-centre edge is below max_edge; n of them drawn without
    replacement (seeded).  Returns n x 3 x 4 (cx, cy, cz, r)."""
    from scipy.spatial import Delaunay

    tri = Delaunay(spheres[:, :3])
    count = {}
    for simplex in tri.simplices:
        s = sorted(int(v) for v in simplex)
        for drop in range(4):
            face = tuple(v for i, v in enumerate(s) if i != drop)
            count[face] = count.get(face, 0) + 1
    faces = sorted(f for f, c in count.items() if c == 2)
    keep = []
    for f in faces:
        c = spheres[list(f), :3]
        e = max(np.linalg.norm(c[0] - c[1]), np.linalg.norm(c[1] - c[2]), np.linalg.norm(c[0] - c[2]))
        if e < max_edge:
            keep.append(f)
    rng = np.random.default_rng(seed)
    if n > len(keep):
        raise ValueError(f"only {len(keep)} interior facets, asked for {n}")
    pick = rng.choice(len(keep), size=n, replace=False)
    return np.stack([spheres[list(keep[i])] for i in sorted(pick)])


def throat_features(triples: np.ndarray, contact_angle: np.ndarray) -> np.ndarray:
    """Descriptor per throat: three radii, three centre distances (0-1, 1-2,
    0-2), contact angle in radians.  n x 7."""
    c = triples[:, :, :3]
    r = triples[:, :, 3]
    d01 = np.linalg.norm(c[:, 0] - c[:, 1], axis=1)
    d12 = np.linalg.norm(c[:, 1] - c[:, 2], axis=1)
    d02 = np.linalg.norm(c[:, 0] - c[:, 2], axis=1)
    return np.c_[r, d01, d12, d02, contact_angle]
