"""Throat domains (Sec. 2.2.2): the library's host voxeliser and probe agree with
the oracle's bit for bit.  CPU only (lbm_throat_geometry does no device work)."""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lbm():
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def test_throat_masks_and_probes_match_oracle(lbm, orc):
    spheres = W.sample_spheres(128)
    for t in W.delaunay_throats(spheres, 30, seed=7):
        m_lib, probe_lib = lbm.lbm_throat_geometry(t)
        m_orc = orc.voxelise_throat(t)
        assert np.array_equal(m_lib, m_orc)
        assert probe_lib == orc.throat_probe(t, m_orc)
        assert (m_lib == orc.M_INLET).any() and (m_lib == orc.M_OUTLET).any()


def test_collinear_throat_rejected(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_throat_geometry([[0, 0, 0, 5], [10, 0, 0, 5], [20, 0, 0, 5]])
    assert e.value.code == lbm.LBM_ERR_ARG


def test_throat_incircle_closed_forms():
    """Three equal spheres of radius r on an equilateral triangle of side a leave
    a gap of a / sqrt(3) - r at the centroid; an unequal case against a brute
    force search over the triangle."""
    import math
    from paper_1906_04722_gb300 import surrogate as S
    for a, r in ((20.0, 10.0), (20.0, 5.0), (27.0, 11.0)):
        t = np.array([[0, 0, 0, r], [a, 0, 0, r], [a / 2, a * math.sqrt(3) / 2, 0, r]], dtype=float)
        # any rigid motion of the triple gives the same radius
        rot = np.array([[0.36, 0.48, -0.8], [-0.8, 0.6, 0.0], [0.48, 0.64, 0.6]])
        t2 = t.copy()
        t2[:, :3] = t[:, :3] @ rot.T + np.array([3.3, -7.1, 12.9])
        got = S.throat_incircle(np.stack([t, t2]))
        assert np.allclose(got, a / math.sqrt(3) - r, atol=1e-9)
    t = np.array([[0, 0, 0, 9.0], [24, 0, 0, 12.0], [9, 19, 0, 10.5]])
    q = t[:, :2]
    best = 0.0
    for u in np.linspace(0, 1, 401):
        for v in np.linspace(0, 1 - u, max(2, int(401 * (1 - u)))):
            p = u * q[0] + v * q[1] + (1 - u - v) * q[2]
            best = max(best, float((np.linalg.norm(q - p, axis=1) - t[:, 3]).min()))
    # the brute force's grid (about 0.06 cells apart) can only fall short of the maximum
    got = S.throat_incircle(t[None])[0]
    assert best - 1e-9 <= got <= best + 0.06


def _lattice_features_reference(mask):
    """The 14 numbers of lbm_throat_lattice_features, from their definitions in
    lbm.h, with scipy's exact Euclidean distance transform."""
    from scipy import ndimage
    nz, ny, nx = mask.shape
    fl = (mask & 1) == 0
    area = fl.reshape(nz, -1).sum(axis=1)
    planes = np.arange(1, nz - 1) if nz >= 3 else np.arange(nz)
    planes = planes[np.argsort(area[planes], kind="stable")]
    first = planes[:3]
    inc = [float(ndimage.distance_transform_edt(fl[k]).max()) for k in first]
    p = np.pad(fl[planes[0]], 1, constant_values=False)
    edge = (~p[:-2, 1:-1]) | (~p[2:, 1:-1]) | (~p[1:-1, :-2]) | (~p[1:-1, 2:])
    perim = int((fl[planes[0]] & edge).sum())
    amin = float(area[planes[0]])
    return np.array([nx, ny, nz, fl.mean(), amin, np.sqrt(amin / np.pi), area[planes].mean(), planes[0] / nz,
                     inc[0], max(inc), np.mean(inc), amin / max(perim, 1), perim, area[first].mean()])


def test_throat_lattice_features_match_reference(lbm):
    """Host lattice description of throat boxes (surrogate inputs) against the
    definitions in lbm.h computed with numpy and scipy.ndimage."""
    pytest.importorskip("scipy")
    throats = W.delaunay_throats(W.sample_spheres(192, seed=3), 40, seed=5)
    F = lbm.lbm_throat_lattice_features(throats)
    assert F.shape == (len(throats), lbm.THROAT_LATTICE_FEATURES)
    for t, th in enumerate(throats):
        mask, _ = lbm.lbm_throat_geometry(th)
        np.testing.assert_allclose(F[t], _lattice_features_reference(mask), rtol=1e-12, atol=1e-9)


def test_lattice_reference_against_brute_force(lbm):
    """Pin the reference itself on hand-made planes: its incircle equals the brute
    force max over fluid cells of the min distance to a solid cell, and its
    perimeter the count of fluid cells with a solid 4-neighbour."""
    rng = np.random.default_rng(4)
    for r in (3, 6, 8.5):
        y, x = np.mgrid[-10:11, -12:13]
        plane = np.where(x * x + (1.3 * y) ** 2 <= r * r, 0, 1).astype(np.uint8)
        plane[rng.random(plane.shape) < 0.03] = 1  # a few grains inside
        mask = np.stack([np.ones_like(plane)] + [plane] * 3 + [np.ones_like(plane)])
        f = _lattice_features_reference(mask)
        fy, fx = np.nonzero(plane == 0)
        sy, sx = np.nonzero(plane == 1)
        d2 = (fy[:, None] - sy[None]) ** 2 + (fx[:, None] - sx[None]) ** 2
        assert f[8] == pytest.approx(np.sqrt(d2.min(axis=1).max()))
        solid = np.pad(plane == 1, 1, constant_values=True)
        edge = solid[:-2, 1:-1] | solid[2:, 1:-1] | solid[1:-1, :-2] | solid[1:-1, 2:]
        assert f[12] == ((plane == 0) & edge).sum()
        assert f[4] == (plane == 0).sum()


def test_surrogate_inputs_layout(lbm):
    """The surrogate's 24 inputs (lbm_throat_surrogate_inputs): the three radii
    and three centre distances over the mean radius, spheres ordered by
    decreasing radius, and the contact angle; the 14 lattice numbers of each
    box; then three of those lengths over the mean radius -- each recomputed
    here from that definition."""
    from paper_1906_04722_gb300 import surrogate as S
    throats = W.delaunay_throats(W.sample_spheres(128), 12, seed=3)
    throats[0, 1, 3] = throats[0, 2, 3]  # a tie keeps the input order
    X, R = S.surrogate_inputs(throats, 0.8)
    assert X.shape == (len(throats), S.N_INPUTS) and X.dtype == np.float32
    L = lbm.lbm_throat_lattice_features(throats)
    for i, t in enumerate(throats):
        order = sorted(range(3), key=lambda j: -t[j, 3])  # stable: ties in input order
        c, r = t[order, :3], t[order, 3]
        Ri = r.mean()
        d = [np.linalg.norm(c[0] - c[1]), np.linalg.norm(c[1] - c[2]), np.linalg.norm(c[0] - c[2])]
        want = np.r_[r / Ri, np.array(d) / Ri, 0.8, L[i], L[i, [5, 8, 9]] / Ri].astype(np.float32)
        assert R[i] == pytest.approx(Ri, rel=1e-15)
        np.testing.assert_array_equal(X[i], want)


def test_pressure_ladder_closed_form(lbm):
    """Per-throat ladders: the reservoir capillary pressure of Eq. 5 at rest,
    p_c,res = (rho_in - rho_major)(1 + G rho_minor)/3, runs from lo/r to hi/r in
    equal steps; radii below 0.5 count as 0.5."""
    from paper_1906_04722_gb300 import surrogate as S
    r = np.array([2.0, 4.0, 0.1])
    lad = S.pressure_ladder(r, 5, 0.4, 1.6, 2.0, 0.06, 0.9)
    pc = (lad - 2.0) * (1 + 0.9 * 0.06) / 3.0
    for i, ri in enumerate([2.0, 4.0, 0.5]):
        np.testing.assert_allclose(pc[i], np.linspace(0.4, 1.6, 5) / ri, rtol=1e-13)


def test_contact_angle_estimate(lbm):
    """cos(theta) = (G_ads,nw - G_ads,w) / (G (rho_major - rho_minor) / 2), clamped."""
    import math
    from paper_1906_04722_gb300 import surrogate as S
    th = S.contact_angle_estimate(-0.3, 0.3, 0.9, 2.0, 0.06)
    assert math.cos(th) == pytest.approx(0.6 / (0.9 * 0.97), rel=1e-14)
    assert S.contact_angle_estimate(0.0, 0.0, 0.9, 2.0, 0.06) == pytest.approx(math.pi / 2)
    assert S.contact_angle_estimate(-5.0, 5.0, 0.9, 2.0, 0.06) == 0.0
