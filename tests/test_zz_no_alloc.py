"""lbm_measure_state_noalloc: measurements for callers that must not allocate
device memory (a host application that owns every device byte through its own
pool, loops that cannot absorb cudaMalloc's synchronisation).  The state lives
in caller-owned device buffers (torch tensors here); the entry point's only
scratch is a fixed device array inside the library.  Its results must equal
those of lbm_measure on the same state, call after call: a smaller state
measured after a larger one must not pick up the larger one's leftovers in the
shared array.

This file is collected last on purpose: a run that stops at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

COUNTS = ("n_fluid", "n_w", "n_interface", "n_bulk_w", "n_bulk_nw", "n_in", "n_out", "n_nonfinite", "n_negative")
VALUES = ("p_w", "p_nw", "p_c", "p_in", "p_out", "p_c_res", "S_w")


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04722_gb300 as lbm
    lbm.load()
    return torch, lbm


def _same(a, b):
    for k in COUNTS:
        assert a[k] == b[k], k
    for k in VALUES:
        if np.isnan(b[k]):
            assert np.isnan(a[k]), k
            continue
        assert abs(a[k] - b[k]) <= 1e-9 * max(1.0, abs(b[k])), (k, a[k], b[k])
    for s in range(2):
        assert abs(a["mass"][s] - b["mass"][s]) <= 1e-9 * abs(b["mass"][s])
    assert a["status_flags"] == b["status_flags"]


def _measure_both(torch, lbm, dom, params, box, mask_dev, stream=None):
    """lbm_measure of the domain, and the no-alloc call on a device copy of its state."""
    ref = dom.measure()
    f, _ = dom.state()
    f_dev = torch.from_numpy(f).cuda()
    torch.cuda.synchronize()
    if stream is None:
        got = lbm.lbm_measure_state_noalloc(params, box, f_dev.data_ptr(), mask_dev.data_ptr())
    else:
        with torch.cuda.stream(stream):
            got = lbm.lbm_measure_state_noalloc(params, box, f_dev.data_ptr(), mask_dev.data_ptr(),
                                                stream=lbm.ctypes.c_void_p(stream.cuda_stream))
    return got, ref


def test_noalloc_measure_matches_lbm_measure_twice(env):
    torch, lbm = env
    shape = (44, 36, 40)
    nz, ny, nx = shape
    spheres = np.array([[12.0, 10.0, 14.0, 6.0], [28.0, 25.0, 30.0, 7.0]])
    params = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=W.G_ADS, rho_major=W.RHO_MAJOR,
                             rho_minor=W.RHO_MINOR, reservoirs=True, membrane_layers=2)
    dom = lbm.Domain(params, spheres, (nx, ny, nz))
    rho = W.droplet_densities(shape, (20, 18, 22), 8.0, seed=21)  # a non-wetting drop in the pores
    rho[0, 0], rho[1, 0] = W.RHO_MINOR, W.RHO_MAJOR                 # and the inlet reservoir layer
    dom.set_densities(rho)
    dom.set_pressure_bc(2.08, W.RHO_MAJOR)
    mask_dev = torch.from_numpy(dom.mask()).cuda()
    for n_steps in (30, 20):
        dom.step(n_steps)
        got, ref = _measure_both(torch, lbm, dom, params, (nx, ny, nz), mask_dev)
        _same(got, ref)
        assert got["n_bulk_nw"] > 0 and got["n_interface"] > 0
    dom.close()

    # a smaller, periodic state right after: fewer blocks write partials, so any
    # slot of the shared array that the larger call left behind and this call
    # reads would show; measured on a non-default stream
    shape2 = (10, 12, 14)
    nz2, ny2, nx2 = shape2
    params2 = lbm.make_params(tau=W.TAU, G=W.G_COHESION, G_ads=(0.0, 0.0), rho_major=W.RHO_MAJOR,
                              rho_minor=W.RHO_MINOR, periodic=(1, 1, 1))
    dom2 = lbm.Domain(params2, np.zeros((0, 4)), (nx2, ny2, nz2))
    dom2.set_densities(W.droplet_densities(shape2, (7, 6, 5), 3.5, seed=22))
    dom2.step(15)
    mask2 = torch.from_numpy(dom2.mask()).cuda()
    side = torch.cuda.Stream()
    got, ref = _measure_both(torch, lbm, dom2, params2, (nx2, ny2, nz2), mask2, stream=side)
    _same(got, ref)
    assert got["n_fluid"] == nx2 * ny2 * nz2 and got["n_bulk_nw"] > 0
    dom2.close()


def test_noalloc_rejects_states_beyond_its_maximum(env):
    torch, lbm = env
    params = lbm.make_params()
    buf = torch.zeros(16, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_measure_state_noalloc(params, (4096, 4096, 4), buf.data_ptr(), buf.data_ptr())
    assert e.value.code == lbm.LBM_ERR_ARG
    assert "maximum" in lbm.lbm_last_error()
