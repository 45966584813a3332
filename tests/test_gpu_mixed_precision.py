"""16-bit population storage (FP16 / BF16 deviations, FP32 collision) against
the FP64 oracle on the single-throat workload.

No precision bound is set for 16-bit storage; the errors are printed and held to
sanity bars: density within 1 % (FP16) / 5 % (BF16) of the oracle after 500
steps (300 at tau = 0.8), S_w within 2 %, and per-component mass conserved to 1e-4 with closed walls
(the rounding of each cell's 18 moving deviations is fed into its rest value).
"""
import json
import os

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
# reports (JSON) go to the directory named by LBM_REPORT_DIR, when it is set
OUT = os.environ.get("LBM_REPORT_DIR", "")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def _rel(rho_g, rho_o, mask, orc):
    fl = (mask & orc.M_SOLID) == 0
    return max(float((np.abs(rho_g[s][fl] - rho_o[s][fl]) / np.maximum(np.abs(rho_o[s][fl]), W.RHO_MINOR)).max())
               for s in range(2))


@pytest.mark.parametrize("precision,bound", [(1, 1e-2), (2, 5e-2)])
@pytest.mark.parametrize("tau", [1.0, 0.8])
def test_16bit_throat32_vs_oracle(lbm, orc, precision, bound, tau):
    shape = (32, 32, 32)
    spheres = W.throat32_spheres()
    params = lbm.make_params(tau=(tau, tau), G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, reservoirs=True, prism_clip=True, precision=precision)
    rho0 = W.initial_densities(shape, noise=1e-3, seed=1)
    dom = lbm.Domain(params, spheres, (32, 32, 32))
    dom.set_densities(rho0)
    dom32 = lbm.Domain(lbm.make_params(tau=(tau, tau), G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                                       rho_minor=W.RHO_MINOR, reservoirs=True, prism_clip=True), spheres, (32, 32, 32))
    dom32.set_densities(rho0)
    mask = orc.voxelise(shape, spheres, prism=True, reservoirs=True)
    f = orc.init(orc.Config(shape=shape, tau=(tau, tau)), mask, rho0)
    # at tau = 0.8 this throat ladder diverges after about 400 steps in the FP64
    # oracle as well (the Shan-Chen model at G = 0.9 is less stable below tau = 1),
    # so that case is compared after 300 steps
    n_incr = 20 if tau == 1.0 else 12
    for rin in W.throat32_ladder(n_incr):
        cfg = orc.Config(shape=shape, tau=(tau, tau), G=W.G_COHESION, G_ads=W.G_ADS, rho_in=(W.RHO_MINOR, rin))
        for d in (dom, dom32):
            d.set_pressure_bc(rin, W.RHO_MAJOR)
            d.step(25)
        orc.step(cfg, mask, f, 25)
    ro = orc.density(cfg, mask, f)
    e16 = _rel(dom.density(), ro, mask, orc)
    e32 = _rel(dom32.density(), ro, mask, orc)
    # at tau = 0.8 the minor component goes slightly negative in interface cells
    # (the FP64 oracle shows the same), which lbm_measure reports as a status
    mg, mo = dom.measure(allow_nonfinite=True), orc.measure(cfg, mask, f)
    assert mg["n_nonfinite"] == 0 and mo["n_nonfinite"] == 0
    rep = {"precision": {1: "fp16", 2: "bf16"}[precision], "tau": tau, "max_rel_density_err": e16,
           "fp32_max_rel_density_err": e32, "S_w": mg["S_w"], "S_w_oracle": mo["S_w"],
           "p_c_res": mg["p_c_res"], "p_c_res_oracle": mo["p_c_res"],
           "mass_rel_err": [abs(mg["mass"][s] - mo["mass"][s]) / mo["mass"][s] for s in range(2)],
           "n_negative": mg["n_negative"], "n_negative_oracle": mo["n_negative"]}
    print(json.dumps(rep))
    if OUT:
        os.makedirs(OUT, exist_ok=True)
        with open(os.path.join(OUT, "mixed_precision_errors.jsonl"), "a") as fh:
            fh.write(json.dumps(rep) + "\n")
    assert e16 <= bound
    assert abs(mg["S_w"] - mo["S_w"]) <= 2e-2 * mo["S_w"]


@pytest.mark.parametrize("precision", [1, 2])
def test_16bit_mass_conservation(lbm, precision):
    shape = (40, 36, 44)
    spheres = np.array([[10.0, 10.0, 10.0, 6.0], [30.0, 25.0, 28.0, 7.5]])
    params = lbm.make_params(tau=(0.9, 0.9), G=W.G_COHESION, G_ads=W.G_ADS, precision=precision)
    nz, ny, nx = shape
    dom = lbm.Domain(params, spheres, (nx, ny, nz))
    dom.set_densities(W.droplet_densities(shape, (22, 18, 20), 8.0, seed=6))
    m0 = dom.measure()["mass"]
    dom.step(300)
    m1 = dom.measure()["mass"]
    for s in range(2):
        assert abs(m1[s] - m0[s]) <= 1e-4 * m0[s], (s, m0[s], m1[s])


@pytest.mark.parametrize("kernel", ["push", "staged"])
@pytest.mark.parametrize("precision,bound", [(1, 2e-3), (2, 2e-2)])
def test_16bit_sample192_sampled_cells(lbm, orc, precision, bound, kernel):
    """The 192^3 drainage sample with 16-bit storage in the launch shapes the
    autotuner picks for it: the push kernel's 10-row shape with 24-plane z
    segments, and the staged kernel with 32 x 8 threads and 32-plane segments.
    Two steps from a seeded noisy state, sampled cells against the oracle run on
    crops that hold their whole dependency cone (2 cells per step)."""
    shape = (192, 192, 192)
    spheres = W.sample192_spheres()
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR, rho_minor=W.RHO_MINOR,
                             reservoirs=True, membrane_layers=3, precision=precision)
    dom = lbm.Domain(params, spheres, (192, 192, 192))
    if kernel == "push":
        dom.set_push_shape(3, 24)
        assert dom.step_kernel() == (lbm.KERNEL_PUSH, 24)
    else:
        dom.set_tile(8, 32, 2)
        assert dom.tile() == (8, 32, 2)
    mask = orc.voxelise(shape, spheres, reservoirs=True, membrane_layers=3)
    assert np.array_equal(dom.mask(), mask)
    rho0 = W.initial_densities(shape, noise=2e-2, seed=8)
    dom.set_densities(rho0)
    K = 2
    dom.step(K)
    rho_g = dom.density()
    rng = np.random.default_rng(14)
    R = 2 * K + 2
    fluid = np.argwhere(mask == 0)
    picks = list(fluid[rng.choice(len(fluid), 24, replace=False)]) + [(0, 95, 1), (191, 100, 190), (188, 50, 60)]
    worst = 0.0
    for z, y, x in picks:
        if mask[z, y, x] & orc.M_SOLID:
            continue
        zs, ys, xs = [slice(max(0, v - R), min(192, v + R + 1)) for v in (z, y, x)]
        sub = mask[zs, ys, xs].copy()
        cfg = orc.Config(shape=sub.shape, tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS,
                         rho_in=(W.RHO_MINOR, W.RHO_MAJOR), rho_out=(W.RHO_MAJOR, W.RHO_MINOR))
        f = orc.init(cfg, sub, np.ascontiguousarray(rho0[:, zs, ys, xs]))
        orc.step(cfg, sub, f, K)
        ro = orc.density(cfg, sub, f)[:, z - zs.start, y - ys.start, x - xs.start]
        for s in range(2):
            if s == 1 and mask[z, y, x] & orc.M_MEMBRANE:
                continue
            worst = max(worst, abs(rho_g[s, z, y, x] - ro[s]) / max(abs(ro[s]), W.RHO_MINOR))
    print(json.dumps({"precision": {1: "fp16", 2: "bf16"}[precision], "kernel": kernel,
                      "sample192_max_rel_density_err_2_steps": worst}))
    assert worst <= bound, worst
