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
        assert np.allclose(got, a / math.sqrt(3) - r, atol=1e-6)
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
