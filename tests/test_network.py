"""The pore network of a sphere packing (Sec. 2.2.1) and drainage on it
(Sec. 2.2.2, Sec. 3.1.1): host code of the library, checked on the CPU.

* The regular triangulation equals the Delaunay tetrahedralisation of the
  centres for equal radii and the lower convex hull of the lifted weighted
  points (x, y, z, |x|^2 - r^2) for unequal ones (both by qhull through scipy),
  and every tetrahedron's orthogonal sphere is empty: no centre has negative
  power with respect to it.
* Drainage equals a plain re-statement (oracle/pn.py) on random networks, and a
  five-pore network whose invasion order and trapping are worked by hand.
* The throat incircle follows Descartes' theorem for touching circles, the
  closed form of three equal circles on an equilateral triangle, and a search
  for the largest circle between the sphere sections.
* The Mayer-Stowe-Princen terms (non-wetting area, meniscus and grain-contact
  lengths) follow the closed form of three touching equal circles at zero
  contact angle and, at other contact angles and arrangements (unequal radii,
  gaps, a meniscus disc reaching over a wall), a brute-force raster of the same
  construction (oracle/pn.py); the MS-P radius likewise, and it lies below the
  incircle at zero contact angle.
"""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lbm():
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def _tset(t):
    return {tuple(sorted(x)) for x in np.asarray(t).tolist()}


def _lifted_lower_hull(sp):
    from scipy.spatial import ConvexHull
    P = sp[:, :3]
    L = np.c_[P, (P ** 2).sum(1) - sp[:, 3] ** 2]
    h = ConvexHull(L)
    return _tset(h.simplices[h.equations[:, 3] < 0])


# ------------------------------------------------------------ triangulation
@pytest.mark.parametrize("seed", [2, 3, 7])
def test_equal_radii_is_delaunay(lbm, seed):
    from scipy.spatial import Delaunay
    sp = W.sample_spheres(192, seed=seed)
    sp[:, 3] = 12.0
    assert _tset(lbm.lbm_regular_triangulation(sp)) == _tset(Delaunay(sp[:, :3]).simplices)


@pytest.mark.parametrize("seed", [2, 3, 7])
def test_weighted_is_lifted_lower_hull(lbm, seed):
    sp = W.sample_spheres(192, seed=seed)
    t = lbm.lbm_regular_triangulation(sp)
    assert _tset(t) == _lifted_lower_hull(sp)


def test_orthogonal_spheres_are_empty_and_cover_the_hull(lbm):
    """The regular property by its definition: for every tetrahedron the centre
    c and squared radius R^2 with |p_i - c|^2 - r_i^2 = R^2 at its corners leave
    every other sphere at non-negative power |p - c|^2 - r^2 - R^2 >= 0; and the
    tetrahedra fill the convex hull of the centres (volumes add up)."""
    from scipy.spatial import ConvexHull
    rng = np.random.default_rng(4)
    sp = np.zeros((120, 4))
    sp[:, :3] = rng.uniform(0, 50, (120, 3))
    sp[:, 3] = rng.uniform(0.5, 3.0, 120)
    t = lbm.lbm_regular_triangulation(sp)
    P, w = sp[:, :3], sp[:, 3] ** 2
    vol = 0.0
    for tet in t:
        a = P[tet]
        A = 2 * (a[1:] - a[0])
        b = (a[1:] ** 2).sum(1) - (a[0] ** 2).sum() - (w[tet[1:]] - w[tet[0]])
        c = np.linalg.solve(A, b)
        R2 = ((a[0] - c) ** 2).sum() - w[tet[0]]
        pw = ((P - c) ** 2).sum(1) - w - R2
        pw[tet] = 0.0
        assert pw.min() >= -1e-7 * max(1.0, abs(R2))
        o = np.linalg.det(a[1:] - a[0])
        assert o > 0  # positively oriented
        vol += o / 6.0
    assert abs(vol - ConvexHull(P).volume) <= 1e-9 * vol


def test_triangulation_rejects_bad_input(lbm):
    with pytest.raises(lbm.LbmError):
        lbm.lbm_regular_triangulation(np.zeros((3, 4)))
    flat = np.zeros((6, 4))
    flat[:, 0] = np.arange(6.0)
    flat[:, 1] = np.arange(6.0) ** 2
    with pytest.raises(lbm.LbmError):
        lbm.lbm_regular_triangulation(flat)


# ------------------------------------------------------------------ network
def test_network_of_sample_volumes_and_links(lbm):
    """Every interior void cell of the sample belongs to exactly one pore;
    interior throats are the facets shared by two tetrahedra; the reservoir
    links sit on pores that reach the inlet and the membrane."""
    sp = W.sample_spheres(96, seed=2)
    import oracle
    mask = oracle.voxelise((96, 96, 96), sp, reservoirs=True, membrane_layers=3)
    t = lbm.lbm_regular_triangulation(sp)
    vol, tp, ts = lbm.lbm_pn_build(sp, t, mask)
    assert vol.sum() == int((mask == 0).sum())
    inner = tp[:, 1] >= 0
    # facets shared by two tetrahedra, counted independently
    from collections import Counter
    cnt = Counter()
    for tet in t.tolist():
        for f in range(4):
            cnt[tuple(sorted(tet[:f] + tet[f + 1:]))] += 1
    shared = {k for k, v in cnt.items() if v == 2}
    assert _tset(ts[inner]) == shared and inner.sum() == len(shared)
    for (a, b), tri in zip(tp[inner], ts[inner]):
        assert set(tri) <= set(t[a]) and set(tri) <= set(t[b])
    assert (tp[:, 1] == lbm.PN_INLET).sum() > 0 and (tp[:, 1] == lbm.PN_OUTLET).sum() > 0
    assert np.all(ts[~inner] == -1)


# ----------------------------------------------------------------- drainage
def _hand_network():
    """Five pores, volumes 1..5.  The inlet touches pore 0; pore 1 hangs off
    pore 0 (entry 0.7) and off pore 3 (0.8); pores 0-2 (0.3), 2-3 (0.4), 3-4
    (0.5); pore 4 drains into the wetting reservoir."""
    vol = [1.0, 2.0, 3.0, 4.0, 5.0]
    th = [(0, -1), (0, 1), (0, 2), (1, 3), (2, 3), (3, 4), (4, -2)]
    pce = [0.1, 0.7, 0.3, 0.8, 0.4, 0.5, 0.0]
    return vol, th, pce


def test_drainage_worked_by_hand(lbm):
    """Levels 0.2, 0.45, 0.6, 0.75, 1.0:
      0.20  the inlet throat (0.1) opens pore 0                      S_w 14/15
      0.45  0-2 (0.3) opens pore 2, then 2-3 (0.4) opens pore 3; pore 1 now has
            only non-wetting neighbours: trapped                      S_w 7/15
      0.60  3-4 (0.5) opens pore 4                                    S_w 2/15
      0.75  0-1 (0.7) leads into the trapped pore 1: nothing          S_w 2/15
      1.00  1-3 (0.8) likewise                                        S_w 2/15"""
    vol, th, pce = _hand_network()
    levels = [0.2, 0.45, 0.6, 0.75, 1.0]
    sw, inv, trap = lbm.lbm_pn_drainage(vol, th, pce, levels)
    assert np.allclose(sw, [14 / 15, 7 / 15, 2 / 15, 2 / 15, 2 / 15], rtol=0, atol=1e-15)
    assert list(inv) == [0, -1, 1, 1, 2]
    assert list(trap) == [-1, 1, -1, -1, -1]


def test_drainage_entry_is_strict_and_membrane_holds(lbm):
    """A level equal to an entry pressure does not pass it (the capillary
    pressure must exceed it); the wetting reservoir is never entered."""
    vol, th, pce = _hand_network()
    sw, inv, _ = lbm.lbm_pn_drainage(vol, th, pce, [0.1, 0.3000001])
    assert inv[0] == 1 and sw[0] == 1.0
    sw, inv, trap = lbm.lbm_pn_drainage(vol, th, pce, [1e9])
    assert sw[0] == pytest.approx(2 / 15) and inv[1] == -1


def test_drainage_matches_plain_restatement(lbm):
    """Random networks (pores on a grid, random entry pressures, inlet on one
    face, outlet on the other): identical invasion and trapping levels and
    S_w to rounding."""
    from oracle import pn
    rng = np.random.default_rng(8)
    for trial in range(6):
        nxg, nyg = 7, 6
        n = nxg * nyg
        idx = lambda i, j: j * nxg + i
        th = []
        for j in range(nyg):
            for i in range(nxg):
                if i + 1 < nxg and rng.random() < 0.85:
                    th.append((idx(i, j), idx(i + 1, j)))
                if j + 1 < nyg and rng.random() < 0.85:
                    th.append((idx(i, j), idx(i, j + 1)))
            th.append((idx(0, j), pn.INLET))
            th.append((idx(nxg - 1, j), pn.OUTLET))
        pce = rng.uniform(0.0, 1.0, len(th)).round(2)  # ties on purpose
        vol = rng.uniform(0.5, 2.0, n)
        levels = np.linspace(0.05, 1.05, 12)
        sw, inv, trap = lbm.lbm_pn_drainage(vol, th, pce, levels)
        sw_o, inv_o, trap_o = pn.drainage(list(vol), th, list(pce), list(levels))
        assert list(inv) == inv_o, trial
        assert list(trap) == trap_o, trial
        assert np.allclose(sw, sw_o, rtol=0, atol=1e-12), trial
        assert np.all(np.diff(sw) <= 1e-15)
        assert (np.array(trap) >= 0).sum() > 0 or trial > 2


# ----------------------------------------------------------------- incircle
def test_incircle_descartes_touching(lbm):
    """Three mutually touching spheres (touching circles in the plane of the
    centres): the inner circle's curvature k4 = k1 + k2 + k3 + 2 sqrt(k1 k2 +
    k2 k3 + k3 k1) (Descartes)."""
    rng = np.random.default_rng(1)
    for _ in range(10):
        r = rng.uniform(5.0, 14.0, 3)
        a, b, c = r[1] + r[2], r[0] + r[2], r[0] + r[1]  # side lengths
        x2 = (b * b - a * a + c * c) / (2 * c)
        y2 = math.sqrt(max(b * b - x2 * x2, 0.0))
        th = np.array([[0, 0, 0, r[0]], [c, 0, 0, r[1]], [x2, y2, 0, r[2]]], float)
        R = rng.standard_normal((3, 3))
        Qm, _ = np.linalg.qr(R)
        th[:, :3] = th[:, :3] @ Qm.T + rng.uniform(-50, 50, 3)  # any frame
        k = 1.0 / r
        k4 = k.sum() + 2 * math.sqrt(k[0] * k[1] + k[1] * k[2] + k[2] * k[0])
        assert lbm.lbm_throat_incircle(th)[0] == pytest.approx(1.0 / k4, rel=1e-10)


@pytest.mark.parametrize("d,r", [(20.0, 10.0), (24.0, 10.0), (30.0, 11.0)])
def test_incircle_equilateral(lbm, d, r):
    """Equal spheres on an equilateral triangle of side d: r_i = d / sqrt(3) - r."""
    th = np.array([[0, 0, 5, r], [d, 0, 5, r], [d / 2, d * math.sqrt(3) / 2, 5, r]], float)
    assert lbm.lbm_throat_incircle(th)[0] == pytest.approx(d / math.sqrt(3) - r, rel=1e-12)
    pce = lbm.lbm_throat_pce_incircle(th, 0.08, math.cos(math.radians(45)))[0]
    assert pce == pytest.approx(2 * 0.08 * math.cos(math.radians(45)) / (d / math.sqrt(3) - r), rel=1e-12)


def test_incircle_matches_search(lbm):
    """Separated unequal spheres, acute and obtuse triangles (where the circle
    touching the three sections has its centre outside the triangle and the
    widest clearance lies on an edge): the search's value."""
    from oracle import pn
    rng = np.random.default_rng(5)
    for trial in range(12):
        r = rng.uniform(9.0, 14.0, 3)
        if trial < 6:
            ang = np.array([0.0, 2.1, 4.2]) + rng.uniform(-0.2, 0.2, 3)
            rad = r.mean() * 1.35 + rng.uniform(0.5, 3.0, 3)
            xy = np.c_[np.cos(ang) * rad, np.sin(ang) * rad]
        else:  # long, flat triangles
            xy = np.array([[0.0, 0.0], [rng.uniform(40, 60), 0.0], [rng.uniform(5, 50), rng.uniform(4, 9)]])
        th = np.c_[xy, np.zeros(3), r]
        assert lbm.lbm_throat_incircle(th)[0] == pytest.approx(max(pn.incircle_search(th), 0.0), abs=1e-6), trial


def test_incircle_closed_throat(lbm):
    """Overlapping sections leave no clearance anywhere in the triangle: 0 and an
    infinite entry pressure."""
    th = np.array([[0, 0, 0, 10.0], [12, 0, 0, 10.0], [6, 10, 0, 10.0]])
    assert lbm.lbm_throat_incircle(th)[0] == 0
    assert math.isinf(lbm.lbm_throat_pce_incircle(th, 0.1, 1.0)[0])


def test_packing_throats_are_shared_facets(lbm):
    """lbm_packing_throats: for equal radii the interior facets of the Delaunay
    tetrahedralisation (qhull), for unequal ones those of the lifted lower hull,
    each with its longest centre distance below the limit."""
    from collections import Counter
    from scipy.spatial import Delaunay
    for equal in (True, False):
        sp = W.sample_spheres(192, seed=6)
        if equal:
            sp[:, 3] = 12.0
            simp = Delaunay(sp[:, :3]).simplices
        else:
            from scipy.spatial import ConvexHull
            P = sp[:, :3]
            h = ConvexHull(np.c_[P, (P ** 2).sum(1) - sp[:, 3] ** 2])
            simp = h.simplices[h.equations[:, 3] < 0]
        cnt = Counter()
        for tet in np.asarray(simp).tolist():
            for f in range(4):
                cnt[tuple(sorted(tet[:f] + tet[f + 1:]))] += 1
        want = set()
        for k, v in cnt.items():
            if v == 2:
                c = sp[list(k), :3]
                e = max(np.linalg.norm(c[a] - c[b]) for a in range(3) for b in range(a + 1, 3))
                if e < 64.0:
                    want.add(k)
        got = lbm.lbm_packing_throats(sp, 64.0)
        assert {tuple(x) for x in got.tolist()} == want
        assert [tuple(x) for x in got.tolist()] == sorted(want)


# --------------------------------------------------------------- MS-P estimate
def _touching_terms(R, r, cos_t=1.0):
    """Three equal circles of radius R touching on an equilateral triangle.  A
    corner meniscus cuts both circles at the contact angle: its centre V lies at
    rho = sqrt(R^2 + r^2 + 2 R r cos(theta)) from both centres, above the touching
    point T0; it meets circle i at polar angle alpha = phi - delta (phi the
    direction of V, cos(delta) = (R^2 + rho^2 - r^2) / (2 R rho)).  The wet
    corner is the triangle (T0, P_j, P_i) minus the two grain segments of angle
    alpha and the meniscus segment of angle gamma (chord |P_i P_j|)."""
    rho = math.sqrt(R * R + r * r + 2 * R * r * cos_t)
    phi = math.atan2(math.sqrt(rho * rho - R * R), R)
    alpha = phi - math.acos(min(1.0, (R * R + rho * rho - r * r) / (2 * R * rho)))
    gamma = 2 * math.asin(R * (1 - math.cos(alpha)) / r)
    wet = (R * R * (1 - math.cos(alpha)) * math.sin(alpha) - R * R * (alpha - math.sin(alpha))
           - 0.5 * r * r * (gamma - math.sin(gamma)))
    a_nw = (math.sqrt(3) - math.pi / 2) * R * R - 3 * wet
    return a_nw, 3 * r * gamma, 3 * R * (math.pi / 3 - 2 * alpha)


_TOUCH = np.array([[0, 0, 0, 1.0], [2, 0, 0, 1.0], [1, math.sqrt(3), 0, 1.0]])


@pytest.mark.parametrize("r", [0.01, 0.05, 0.1, 0.14])
@pytest.mark.parametrize("cos_t", [1.0, math.cos(math.radians(30)), math.cos(math.radians(50))])
def test_msp_terms_touching_closed_form(lbm, r, cos_t):
    got = lbm.lbm_throat_msp_terms(_TOUCH * 7.5, r * 7.5, cos_t)  # any scale
    want = _touching_terms(7.5, r * 7.5, cos_t)
    for g, w in zip(got, want):
        assert abs(g - w) <= 1e-9 * max(1.0, abs(w))


def test_msp_radius_touching_closed_form(lbm):
    """The root of A_nw = r (L_nw + L_ns cos(theta)) of the closed form
    (bisection here) against lbm_throat_pce_msp with sigma = 1."""
    for cos_t in (1.0, math.cos(math.radians(40))):
        lo, hi = 1e-6, 2 / math.sqrt(3) - 1
        for _ in range(100):
            mid = 0.5 * (lo + hi)
            a, lnw, lns = _touching_terms(1.0, mid, cos_t)
            lo, hi = (mid, hi) if a - mid * (lnw + lns * cos_t) > 0 else (lo, mid)
        r_star = 0.5 * (lo + hi)
        assert abs(1.0 / lbm.lbm_throat_pce_msp(_TOUCH, 1.0, cos_t)[0] - r_star) <= 1e-9


def test_msp_raster_oracle_touching_closed_form():
    """The brute-force raster of oracle/pn.py against the closed form of
    touching circles at 50 degrees (where its meniscus band is well posed)."""
    from oracle import pn
    ct = math.cos(math.radians(50))
    for r in (0.05, 0.12):
        want = _touching_terms(1.0, r, ct)
        got = pn.msp_terms_raster(_TOUCH, r, ct, 0.002)
        assert abs(got[0] - want[0]) <= 0.01 * want[0]
        assert abs(got[1] - want[1]) <= 0.04 * want[1]
        assert abs(got[2] - want[2]) <= 0.015 * want[2]


# (throat, cos theta, r): unequal radii; gaps on every edge; a wall corner where
# the meniscus disc reaches over the edge and leaves two slivers; the same edge
# with the disc covering both grains' edge points (a dry corner)
_RASTER_CASES = [
    (np.array([[0, 0, 0, 1.0], [2.3, 0.2, 0.1, 0.8], [0.9, 2.1, -0.2, 1.2]]), 0.7, 0.1),
    (np.array([[0, 0, 0, 1.0], [2.3, 0.2, 0.1, 0.8], [0.9, 2.1, -0.2, 1.2]]), 0.7, 0.2),
    (np.array([[0, 0, 0, 1.0], [2.2, 0, 0, 1.0], [1.1, 2.2 * math.sqrt(3) / 2, 0, 1.0]]), 0.8, 0.2),
    (np.array([[0, 0, 0, 1.0], [2.6, 0, 0, 1.0], [1.3, 2.8, 0, 1.0]]), 0.5, 0.65),
    (np.array([[0, 0, 0, 1.0], [2.6, 0, 0, 1.0], [1.3, 2.8, 0, 1.0]]), 0.5, 0.5),
]


@pytest.mark.parametrize("case", range(len(_RASTER_CASES)))
def test_msp_terms_match_raster(lbm, case):
    """Exact terms against the pixel count of the same construction (h = 0.002
    on unit radii): area within 1 %, grain contact within 1.5 %, menisci within
    4 % or 0.02 (the raster's level-set band)."""
    from oracle import pn
    th, ct, r = _RASTER_CASES[case]
    a, lnw, lns = lbm.lbm_throat_msp_terms(th, r, ct)
    ra, rlnw, rlns = pn.msp_terms_raster(th, r, ct, 0.002)
    assert abs(a - ra) <= 0.01 * ra
    assert abs(lns - rlns) <= 0.015 * rlns
    assert abs(lnw - rlnw) <= max(0.04 * rlnw, 0.02)


def test_msp_radius_matches_raster(lbm):
    from oracle import pn
    th, ct = _RASTER_CASES[0][0], 0.7
    r_exact = 1.0 / lbm.lbm_throat_pce_msp(th, 1.0, ct)[0]
    r_raster = pn.msp_radius_raster(th, ct, 0.003, 2 * lbm.lbm_throat_incircle(th)[0])
    assert abs(r_exact - r_raster) <= 0.02 * r_raster


def test_msp_packing_below_incircle_and_closed(lbm):
    """On every throat of a packing the zero-contact-angle MS-P meniscus is no
    wider than the incircle: beyond r_i no meniscus centre is allowed.  It
    reaches r_i only where the walls, not the grains, bound the section (the
    non-wetting region then spills over the neutral walls and F stays positive
    until the allowed centres run out): a few throats.  All finite; a closed
    throat gives +inf."""
    tri = lbm.packing_throat_sample(W.sample_spheres(192, seed=3), None, 3)
    p = lbm.lbm_throat_pce_msp(tri, 1.0, 1.0)
    rin = lbm.lbm_throat_incircle(tri)
    assert np.isfinite(p).all()
    assert (1.0 / p <= rin * (1 + 1e-9)).all()
    assert (1.0 / p < rin * (1 - 1e-6)).mean() > 0.99
    th = np.array([[0, 0, 0, 10.0], [12, 0, 0, 10.0], [6, 10, 0, 10.0]])
    assert math.isinf(lbm.lbm_throat_pce_msp(th, 0.1, 1.0)[0])
    with pytest.raises(lbm.LbmError):
        lbm.lbm_throat_pce_msp(_TOUCH, 1.0, 0.0)
