"""The FP32 step kernels (staged cp.async, its double-pull variant, TMA plane
loads, the two-launch form, the paired push-form kernel) against the FP64
oracle and against each other.

Boxes are chosen so that the TMA kernel's 32 x 8 tiles have ragged tails in x
and y and its z segments ragged ends; grains carry adhesion, the closed-z case
has reservoirs and a membrane, the periodic-z case wraps the plane loads.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

RTOL_RHO = 1e-5


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def _params(lbm, **kw):
    base = dict(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR, rho_minor=W.RHO_MINOR)
    base.update(kw)
    return lbm.make_params(**base)


def _rel_err(rho_gpu, rho_orc, mask, orc):
    err = 0.0
    for s in range(2):
        fl = (mask & orc.M_SOLID) == 0
        if s == 1:
            fl &= (mask & orc.M_MEMBRANE) == 0
        d = np.abs(rho_gpu[s][fl] - rho_orc[s][fl]) / np.abs(rho_orc[s][fl])
        err = max(err, float(d.max()))
    return err


SHAPE = (45, 29, 68)  # (nz, ny, nx): x tiles 32 + 32 + 4, y tiles 8 x 3 + 5
SPHERES = np.array([[10.0, 8.0, 6.0, 5.3], [40.2, 20.5, 15.0, 6.1], [60.0, 3.0, 30.0, 4.0],
                    [33.0, 14.0, 40.0, 5.5]])


def _case(lbm, orc, periodic_z):
    nz, ny, nx = SHAPE
    if periodic_z:
        flags, oflags = dict(periodic=(0, 0, 1)), dict()
        rho0 = W.droplet_densities(SHAPE, (20, 14, 40), 7.0, seed=21)
        ckw = dict(periodic=(0, 0, 1))
    else:
        flags, oflags = dict(reservoirs=True, membrane_layers=2), dict(reservoirs=True, membrane_layers=2)
        rho0 = W.initial_densities(SHAPE, noise=1e-3, seed=22)
        ckw = dict(rho_in=(W.RHO_MINOR, 2.08), rho_out=(W.RHO_MAJOR, W.RHO_MINOR))
    mask = orc.voxelise(SHAPE, SPHERES, **oflags)
    cfg = orc.Config(shape=SHAPE, tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, **ckw)
    return flags, mask, cfg, rho0


def _gpu_run(lbm, flags, rho0, steps, kernel, lz=0):
    nz, ny, nx = SHAPE
    dom = lbm.Domain(_params(lbm, **flags), SPHERES, (nx, ny, nz))
    if kernel in (lbm.KERNEL_TMA, lbm.KERNEL_SPLIT):
        dom.set_step_kernel(kernel, lz)
    elif isinstance(lz, tuple):
        dom.set_tile(*lz)
    else:
        dom.set_tile(6, 16, 2)
    assert dom.step_kernel()[0] == kernel
    dom.set_densities(rho0)
    if not flags.get("periodic"):
        dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    dom.step(steps)
    return dom


@pytest.mark.parametrize("periodic_z", [0, 1])
def test_tma_kernel_matches_oracle(lbm, orc, periodic_z):
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    dom = _gpu_run(lbm, flags, rho0, 70, lbm.KERNEL_TMA, lz=13)
    assert np.array_equal(dom.mask(), mask)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 70)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


def test_tma_default_kernel_choice(lbm):
    nz, ny, nx = SHAPE
    d1 = lbm.Domain(_params(lbm), SPHERES, (nx, ny, nz))
    assert d1.step_kernel()[0] == lbm.KERNEL_STAGED  # the default
    d1.set_step_kernel(lbm.KERNEL_TMA)
    assert d1.step_kernel()[0] == lbm.KERNEL_TMA
    d2 = lbm.Domain(_params(lbm, periodic=(1, 0, 0)), SPHERES, (nx, ny, nz))
    assert d2.step_kernel()[0] == lbm.KERNEL_STAGED
    with pytest.raises(lbm.LbmError):
        d2.set_step_kernel(lbm.KERNEL_TMA)
    d3 = lbm.Domain(_params(lbm), SPHERES, (nx - 1, ny, nz))  # nx % 4 != 0
    with pytest.raises(lbm.LbmError):
        d3.set_step_kernel(lbm.KERNEL_TMA)


def test_tma_segments_bitwise(lbm, orc):
    """The z-segment length changes which CTA computes a plane, not how."""
    flags, mask, cfg, rho0 = _case(lbm, orc, 0)
    ref = _gpu_run(lbm, flags, rho0, 40, lbm.KERNEL_TMA, lz=45).state()[0]
    for lz in (4, 7, 11):
        got = _gpu_run(lbm, flags, rho0, 40, lbm.KERNEL_TMA, lz=lz).state()[0]
        assert np.array_equal(got, ref), lz


@pytest.mark.parametrize("periodic_z", [0, 1])
def test_staged_and_tma_agree(lbm, orc, periodic_z):
    """Same FP32 arithmetic per cell, different summation contexts (the compiler
    may contract differently): after 100 steps the densities differ by at most
    about one FP32 ulp (6e-8 relative) per step, 6e-6; the bar is 5e-6, each
    kernel being held to the FP64 oracle at 1e-5 separately."""
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    a = _gpu_run(lbm, flags, rho0, 100, lbm.KERNEL_TMA).density()
    b = _gpu_run(lbm, flags, rho0, 100, lbm.KERNEL_STAGED).density()
    assert _rel_err(a, b, mask, orc) <= 5e-6


def test_autotune_restores_state_and_keeps_parity(lbm, orc):
    """Tuning runs trial steps on the domain itself; afterwards the state and the
    step counter are the ones before, bit for bit, and the tuned kernel still
    matches the oracle."""
    flags, mask, cfg, rho0 = _case(lbm, orc, 0)
    nz, ny, nx = SHAPE
    dom = lbm.Domain(_params(lbm, **flags), SPHERES, (nx, ny, nz))
    dom.set_densities(rho0)
    dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    dom.step(5)
    before, st = dom.state()
    res = dom.autotune(trial_steps=4)
    after, st2 = dom.state()
    assert st2 == st == 5
    assert np.array_equal(before, after)
    assert res["n_candidates"] >= 10 and res["ms_per_step"] > 0
    kind, lz = dom.step_kernel()
    assert kind == {"staged": lbm.KERNEL_STAGED, "tma": lbm.KERNEL_TMA, "split": lbm.KERNEL_SPLIT,
                    "staged2": lbm.KERNEL_STAGED2, "push": lbm.KERNEL_PUSH}[res["kind"]]
    if res["kind"] != "split":
        assert lz == res["lz"]
    dom.step(65)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 70)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


@pytest.mark.parametrize("periodic_z", [0, 1])
def test_split_kernel_matches_oracle(lbm, orc, periodic_z):
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    dom = _gpu_run(lbm, flags, rho0, 70, lbm.KERNEL_SPLIT)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 70)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


def test_split_kernel_periodic_xy(lbm, orc):
    """The two-launch kernel serves any periodicity (the TMA kernel does not)."""
    shape = (20, 13, 41)
    spheres = np.array([[20.0, 6.0, 10.0, 4.5]])
    rho0 = W.droplet_densities(shape, (8, 6, 9), 4.0, seed=3)
    nz, ny, nx = shape
    dom = lbm.Domain(_params(lbm, periodic=(1, 1, 0)), spheres, (nx, ny, nz))
    dom.set_step_kernel(lbm.KERNEL_SPLIT)
    dom.set_densities(rho0)
    dom.step(60)
    mask = orc.voxelise(shape, spheres)
    cfg = orc.Config(shape=shape, tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, periodic=(1, 1, 0))
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 60)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


@pytest.mark.parametrize("shape", [(6, 8, 0), (8, 8, 1), (10, 16, 0), (8, 16, 3), (10, 8, 2)])
def test_staged_shapes_match_oracle(lbm, orc, shape):
    """Every staged shape the autotuner may pick (lead 0 and 1: the double-pull variant)."""
    flags, mask, cfg, rho0 = _case(lbm, orc, 0)
    dom = _gpu_run(lbm, flags, rho0, 40, lbm.KERNEL_STAGED, lz=shape)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 40)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


@pytest.mark.parametrize("by,lz", [(6, 8), (6, 16), (8, 13)])
@pytest.mark.parametrize("periodic_z", [0, 1])
def test_staged2_kernel_matches_oracle(lbm, orc, by, lz, periodic_z):
    """Two threads per cell (one per component), every shape the autotuner may pick."""
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    nz, ny, nx = SHAPE
    dom = lbm.Domain(_params(lbm, **flags), SPHERES, (nx, ny, nz))
    dom.set_tile(by, lz, 2)
    dom.set_step_kernel(lbm.KERNEL_STAGED2, lz)
    assert dom.step_kernel() == (lbm.KERNEL_STAGED2, lz)
    dom.set_densities(rho0)
    if not periodic_z:
        dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    dom.step(70)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 70)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


def test_staged2_periodic_xy(lbm, orc):
    shape = (20, 13, 41)
    spheres = np.array([[20.0, 6.0, 10.0, 4.5]])
    rho0 = W.droplet_densities(shape, (8, 6, 9), 4.0, seed=3)
    nz, ny, nx = shape
    dom = lbm.Domain(_params(lbm, periodic=(1, 1, 0)), spheres, (nx, ny, nz))
    dom.set_step_kernel(lbm.KERNEL_STAGED2, 8)
    dom.set_densities(rho0)
    dom.step(60)
    mask = orc.voxelise(shape, spheres)
    cfg = orc.Config(shape=shape, tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, periodic=(1, 1, 0))
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 60)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


@pytest.mark.parametrize("kernel", ["staged", "tma", "split", "staged2", "push", "push_resident"])
def test_unequal_tau_and_body_force_every_kernel(lbm, orc, kernel):
    """tau = (0.8, 1.2) with a body force (weakly damped, the most rounding
    sensitive case of the suite) for every FP32 kernel."""
    shape = (41, 16, 36)
    spheres = np.array([[18.0, 8.0, 10.0, 4.5]])
    rho0 = W.droplet_densities(shape, (9, 8, 25), 4.0, seed=3)
    nz, ny, nx = shape
    kw = dict(tau=(0.8, 1.2))
    dom = lbm.Domain(_params(lbm, body_force=(1e-5, 0, -2e-5), **kw), spheres, (nx, ny, nz))
    if kernel == "tma":
        dom.set_step_kernel(lbm.KERNEL_TMA, 8)
    elif kernel == "split":
        dom.set_step_kernel(lbm.KERNEL_SPLIT)
    elif kernel == "staged2":
        dom.set_step_kernel(lbm.KERNEL_STAGED2, 8)
    elif kernel == "push":
        dom.set_push_shape(1, 9)
    elif kernel == "push_resident":
        dom.set_push_shape(9, 7)
    dom.set_densities(rho0)
    dom.step(80)
    mask = orc.voxelise(shape, spheres)
    cfg = orc.Config(shape=shape, G=W.G_COHESION, G_ads=W.G_ADS, g=(1e-5, 0, -2e-5), **kw)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 80)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO


def test_staged_and_double_pull_bitwise(lbm, orc):
    """The staged kernel (pulls queued as asynchronous copies into shared memory)
    and the double-pull kernel (pulls from global memory twice) sum the
    densities in the same order and share the collision: the same state bit for
    bit."""
    flags, mask, cfg, rho0 = _case(lbm, orc, 0)
    a = _gpu_run(lbm, flags, rho0, 60, lbm.KERNEL_STAGED, lz=(6, 16, 2)).state()[0]
    b = _gpu_run(lbm, flags, rho0, 60, lbm.KERNEL_STAGED, lz=(6, 16, 0)).state()[0]
    assert np.array_equal(a, b)


def test_bounded_wait_gives_up_and_reports(lbm):
    """The TMA kernel's waits are bounded: a wait on an mbarrier that nothing
    completes (a flag nobody sets) gives up after its limit and reports it, and
    the context stays usable for the next domain."""
    import time
    t0 = time.perf_counter()
    assert lbm.lbm_selftest_bounded_wait(20000)  # 20 ms
    assert time.perf_counter() - t0 < 30.0
    nz, ny, nx = SHAPE
    dom = lbm.Domain(_params(lbm, periodic=(0, 0, 1)), SPHERES, (nx, ny, nz))
    dom.set_step_kernel(lbm.KERNEL_TMA, 8)
    dom.step(3)
    assert dom.measure()["n_nonfinite"] == 0


# ------------------------------------------------------- paired push kernel
def _push_run(lbm, flags, rho0, steps, shape, lz, prefetch=0, order=0):
    nz, ny, nx = SHAPE
    dom = lbm.Domain(_params(lbm, **flags), SPHERES, (nx, ny, nz))
    dom.set_push_shape(shape, lz)
    dom.set_push_prefetch(prefetch)
    dom.set_push_order(order)
    assert dom.step_kernel() == (lbm.KERNEL_PUSH, lz)
    dom.set_densities(rho0)
    if not flags.get("periodic"):
        dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    dom.step(steps)
    return dom


@pytest.mark.parametrize("shape,lz,prefetch,order", [
    (0, 13, 0, 0), (1, 7, 2, 1), (1, 45, 4, 0), (2, 16, 1, 1), (3, 11, 2, 0), (4, 9, 3, 1), (5, 20, 0, 0), (0, 5, 2, 1),
    (6, 13, 2, 0), (7, 9, 0, 1), (8, 20, 1, 0), (9, 11, 3, 1), (10, 7, 2, 0), (11, 45, 0, 1), (9, 1, 2, 1),
    (6, 2, 0, 1), (3, 4, 2, 1), (11, 6, 0, 1)])
@pytest.mark.parametrize("periodic_z", [0, 1])
def test_push_kernel_equals_staged_bitwise(lbm, orc, shape, lz, prefetch, order, periodic_z):
    """The push kernel reads each cell's own populations and streams at the
    store, the staged kernel pulls; both sum the densities in the same order and
    share the collision, so after 60 steps the states (read back in the pull
    layout) are the same bit for bit -- every shape, ragged x, y and z tiles,
    reservoirs and a membrane (closed z) or a wrapped z axis, with and without
    the L2 prefetch (a hint that changes nothing), with the pairs re-read from
    shared memory or held in registers, down to one- and two-plane segments,
    every segment marching +z or alternate segments marching -z."""
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    a = _push_run(lbm, flags, rho0, 60, shape, lz, prefetch, order).state()[0]
    b = _gpu_run(lbm, flags, rho0, 60, lbm.KERNEL_STAGED).state()[0]
    assert np.array_equal(a, b)


@pytest.mark.parametrize("periodic_z", [0, 1])
def test_push_kernel_matches_oracle(lbm, orc, periodic_z):
    flags, mask, cfg, rho0 = _case(lbm, orc, periodic_z)
    dom = _push_run(lbm, flags, rho0, 70, 0, 13)
    assert np.array_equal(dom.mask(), mask)
    f = orc.init(cfg, mask, rho0)
    orc.step(cfg, mask, f, 70)
    assert _rel_err(dom.density(), orc.density(cfg, mask, f), mask, orc) <= RTOL_RHO
    m, mo = dom.measure(), orc.measure(cfg, mask, f)
    for key in ("n_fluid", "n_w", "n_in", "n_out"):
        assert m[key] == mo[key], key
    for s in range(2):
        assert abs(m["mass"][s] - mo["mass"][s]) <= 1e-6 * mo["mass"][s]


def test_push_kernel_switches_and_checkpoints_bitwise(lbm, orc):
    """The state changes layout when the kernel kind changes and when it is read
    out; neither changes a bit: push 25 steps, read the density (a converted
    copy), staged 20, push 15 more, checkpoint, resume on a new domain with the
    push kernel, equals 60 staged steps."""
    flags, mask, cfg, rho0 = _case(lbm, orc, 0)
    nz, ny, nx = SHAPE
    ref = _gpu_run(lbm, flags, rho0, 60, lbm.KERNEL_STAGED).state()[0]
    dom = _push_run(lbm, flags, rho0, 25, 0, 8)
    dom.density()
    dom.set_tile(6, 16, 2)
    dom.step(20)
    dom.set_push_shape(2, 11)
    dom.step(10)
    f, st = dom.state()
    assert st == 55
    dom2 = lbm.Domain(_params(lbm, **flags), SPHERES, (nx, ny, nz))
    dom2.set_push_shape(1, 0)
    dom2.set_pressure_bc(2.08, W.RHO_MAJOR)
    dom2.set_state(f, st)
    dom2.step(5)
    got, st2 = dom2.state()
    assert st2 == 60
    assert np.array_equal(got, ref)


def test_push_kernel_applicability(lbm):
    nz, ny, nx = SHAPE
    d1 = lbm.Domain(_params(lbm, periodic=(1, 0, 0)), SPHERES, (nx, ny, nz))
    with pytest.raises(lbm.LbmError):
        d1.set_step_kernel(lbm.KERNEL_PUSH)
    d2 = lbm.Domain(_params(lbm), SPHERES, (nx - 1, ny, nz))  # odd nx
    with pytest.raises(lbm.LbmError):
        d2.set_push_shape(0)
    d3 = lbm.Domain(_params(lbm), SPHERES, (nx, ny, nz))
    with pytest.raises(lbm.LbmError):
        d3.set_push_shape(lbm.PUSH_SHAPES)
    for bad in (-1, 5):
        with pytest.raises(lbm.LbmError):
            d3.set_push_prefetch(bad)
    for bad in (-1, 2):
        with pytest.raises(lbm.LbmError):
            d3.set_push_order(bad)
    d3.set_step_kernel(lbm.KERNEL_PUSH, 9)
    assert d3.step_kernel() == (lbm.KERNEL_PUSH, 9)
