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
