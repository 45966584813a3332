"""The push kernel of 16-bit storage (FP16 / BF16 deviations, FP32 collision).

It stores each word of the pull kernel at the cell that reads it, encoded against
the same densities, so after any number of steps its densities and measurements
equal the staged 16-bit kernel's bit for bit: every shape, ragged x, y and z
tiles, short and long z segments, reservoirs with a membrane (the components
then stream apart and are stored as separate halves) or a wrapped z axis.  The
state changes layout when the kernel kind changes, without changing a bit.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

SHAPE = (45, 29, 68)  # (nz, ny, nx): nx a multiple of 4; ragged x, y and z tiles
SPHERES = np.array([[10.0, 8.0, 6.0, 5.3], [40.2, 20.5, 15.0, 6.1], [60.0, 3.0, 30.0, 4.0],
                    [33.0, 14.0, 40.0, 5.5]])


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def _domain(lbm, precision, periodic_z, tau=W.TAU):
    nz, ny, nx = SHAPE
    if periodic_z:
        kw = dict(periodic=(0, 0, 1))
        rho0 = W.droplet_densities(SHAPE, (20, 14, 40), 7.0, seed=21)
    else:
        kw = dict(reservoirs=True, membrane_layers=2)
        rho0 = W.initial_densities(SHAPE, noise=1e-3, seed=22)
    params = lbm.make_params(tau=tau, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, precision=precision, **kw)
    dom = lbm.Domain(params, SPHERES, (nx, ny, nz))
    dom.set_densities(rho0)
    if not periodic_z:
        dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    return dom


def _same(a, b):
    da, db = a.density(), b.density()
    assert np.array_equal(da, db)
    ma, mb = a.measure(), b.measure()
    for key in ("n_fluid", "n_w", "n_interface", "n_in", "n_out"):
        assert ma[key] == mb[key], key
    assert ma["mass"] == mb["mass"]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("shape,lz", [(0, 13), (1, 7), (2, 45), (3, 16), (0, 1), (1, 2), (4, 13), (5, 7), (6, 45),
                                      (7, 16), (8, 1), (9, 2), (10, 13), (11, 5)])
@pytest.mark.parametrize("periodic_z", [0, 1])
def test_push16_equals_staged16_bitwise(lbm, precision, shape, lz, periodic_z):
    a = _domain(lbm, precision, periodic_z)
    a.set_push_shape(shape, lz)
    assert a.step_kernel() == (lbm.KERNEL_PUSH, lz)
    a.step(60)
    b = _domain(lbm, precision, periodic_z)
    b.set_tile(8, 16, 2)
    b.step(60)
    _same(a, b)


@pytest.mark.parametrize("precision", [1, 2])
def test_push16_unequal_tau_bitwise(lbm, precision):
    a = _domain(lbm, precision, 0, tau=(0.8, 1.2))
    a.set_push_shape(0, 11)
    a.step(50)
    b = _domain(lbm, precision, 0, tau=(0.8, 1.2))
    b.step(50)
    _same(a, b)


@pytest.mark.parametrize("precision", [1, 2])
def test_push16_switches_layout_bitwise(lbm, precision):
    """Push 20 steps, read the densities (a converted copy), staged 20, push 20
    in another shape: the same as 60 staged steps."""
    a = _domain(lbm, precision, 0)
    a.set_push_shape(0, 8)
    a.step(20)
    a.density()
    a.measure()
    a.set_tile(6, 16, 2)
    a.step(20)
    a.set_push_shape(3, 0)
    a.step(20)
    b = _domain(lbm, precision, 0)
    b.step(60)
    _same(a, b)


def test_push16_applicability(lbm):
    nz, ny, nx = SHAPE
    p = lbm.make_params(precision=1, periodic=(1, 0, 0))
    d1 = lbm.Domain(p, SPHERES, (nx, ny, nz))
    with pytest.raises(lbm.LbmError):
        d1.set_step_kernel(lbm.KERNEL_PUSH)
    d2 = lbm.Domain(lbm.make_params(precision=1), SPHERES, (nx - 2, ny, nz))  # nx % 4 == 2
    with pytest.raises(lbm.LbmError):
        d2.set_push_shape(0)
    d3 = lbm.Domain(lbm.make_params(precision=2), SPHERES, (nx, ny, nz))
    with pytest.raises(lbm.LbmError):
        d3.set_push_shape(len(lbm.PUSH16_SHAPE_TABLE))
    d3.set_step_kernel(lbm.KERNEL_PUSH, 9)
    assert d3.step_kernel() == (lbm.KERNEL_PUSH, 9)


@pytest.mark.parametrize("precision", [1, 2])
def test_push16_autotune_keeps_state(lbm, precision):
    a = _domain(lbm, precision, 0)
    a.step(5)
    before = a.density()
    res = a.autotune(trial_steps=3)
    assert np.array_equal(before, a.density())
    assert res["n_candidates"] >= 16
    a.step(25)
    b = _domain(lbm, precision, 0)
    b.step(30)
    _same(a, b)
