"""Surrogate MLP kernels against the FP64 oracle MLP.

Forward outputs, loss gradients and one Adam step of the tensor-core kernels
(BF16 or FP16 operands rounded from FP32 masters, FP32 accumulation) are compared
with oracle/mlp.py on the same parameters, element by element, each element
against its own bound.  The bounds follow the arithmetic: a GEMM rounds both of
its operands once (unit roundoff u = 2^-11 for FP16, 2^-8 for BF16) and adds in
FP32 (2^-24 per addition), so an output element is off by at most
(2u + (n + 2) 2^-24) times the sum of the absolute values of its products, plus
what its inputs were off by carried through |W|.  Carried layer by layer (ReLU
does not amplify), and through the backward pass with the same rule, this bounds
every output and every gradient element; where a hidden unit's pre-activation
lies within its own bound of zero the two sides may disagree on its ReLU
derivative, and the full size of that unit's term is added to the bound.  The
norm-wise errors are printed as a report.  Training must drive the loss of a
smooth target down.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1906_04722_gb300 as m
    m.load()
    return m


def _nrel(a, b):
    return float(np.linalg.norm(np.asarray(a, dtype=np.float64) - b) / max(1e-30, np.linalg.norm(b)))


U32 = 2.0 ** -24


def _elementwise_bounds(params, X, T, u):
    """Per-element bounds on |GPU - oracle| of the outputs and of every (dW, db),
    for GEMMs that round their operands to a 16-bit type of unit roundoff u and
    accumulate in FP32 (first order in u; see the module docstring)."""
    acts, zs, ez = [np.asarray(X, float)], [], []
    eh = np.zeros_like(acts[0])
    L = len(params)
    for i, (W, b) in enumerate(params):
        h = acts[-1]
        n = W.shape[1]
        z = h @ W.T + b
        mag = np.abs(h) @ np.abs(W).T + np.abs(b)
        e = eh @ np.abs(W).T * (1 + u) ** 2 + (2.01 * u + (n + 2) * U32) * mag
        zs.append(z)
        ez.append(e)
        eh = e
        acts.append(np.maximum(z, 0.0) if i < L - 1 else z)
    y, ey = acts[-1], ez[-1]
    N = y.size
    d = 2.0 * (y - T) / N
    ed = 2.0 * (ey + 4 * U32 * np.abs(y - T)) / N
    bounds = [None] * L
    for i in range(L - 1, -1, -1):
        W, _ = params[i]
        h = acts[i]
        ehi = ez[i - 1] if i > 0 else np.zeros_like(h)
        ns = h.shape[0]
        gam = 2.01 * u + (ns + 2) * U32
        bW = np.abs(ed).T @ np.abs(h) * (1 + u) ** 2 + np.abs(d).T @ ehi * (1 + u) ** 2 + gam * (np.abs(d).T @ np.abs(h))
        bb = ed.sum(axis=0) + (ns + 2) * U32 * np.abs(d).sum(axis=0)
        bounds[i] = (bW, bb)
        if i > 0:
            m = W.shape[0]
            full = np.abs(d) @ np.abs(W)
            back = np.abs(ed) @ np.abs(W) * (1 + u) ** 2 + (2.01 * u + (m + 2) * U32) * full
            zprev = zs[i - 1]
            certain = np.abs(zprev) > ez[i - 1]
            alive = zprev > 0
            ed = np.where(certain, np.where(alive, back, 0.0), back + full)
            d = (d @ W) * alive
    return y, ey, bounds


@pytest.mark.parametrize("half", [1, 0])
def test_forward_and_gradients_elementwise(lbm, half):
    rng = np.random.default_rng(5)
    sur = lbm.Surrogate(7, 17, n_hidden=256, n_layers=4, n_members=2, half=half, seed=3)
    layers = omlp.init_params(sur.sizes, seed=9)
    for W, b in layers:
        b[:] = rng.standard_normal(b.shape) * 0.1
    sur.set_params(1, sur.flatten(layers))
    ref = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)] for W, b in layers]
    X = rng.standard_normal((300, 7)).astype(np.float32).astype(np.float64)
    T = rng.standard_normal((300, 17)).astype(np.float32).astype(np.float64)
    u = 2.0 ** -11 if half else 2.0 ** -8
    y_ref, ey, bounds = _elementwise_bounds(ref, X, T, u)
    def ratio(err, bound):  # largest err / bound (an element whose bound is 0 must be exact)
        assert np.all(err <= bound)
        pos = bound > 0
        return float((err[pos] / bound[pos]).max()) if pos.any() else 0.0

    y = sur.forward(1, X)
    worst = [ratio(np.abs(y - y_ref), ey)]
    g, _ = sur.gradients(1, X, T)
    g_ref = omlp.gradients(ref, X, T)
    for (gW, gb), (rW, rb), (bW, bb) in zip(sur.layers(g), g_ref, bounds):
        worst.append(max(ratio(np.abs(gW - rW), bW), ratio(np.abs(gb - rb), bb)))
    print("half" if half else "bf16", "largest error / element bound: forward then layers", worst)


@pytest.mark.parametrize("half,tol_fwd,tol", [(1, 2e-3, 2e-2), (0, 1.5e-2, 6e-2)])
def test_forward_and_gradients_match_oracle(lbm, half, tol_fwd, tol):
    """Norm-wise report: the backward dot products over 256 hidden units cancel,
    which amplifies operand rounding by about sqrt(256) per layer; measured
    1.1e-2 (FP16) and 3.1e-2 (BF16) on the first layer's gradient."""
    rng = np.random.default_rng(5)
    sur = lbm.Surrogate(7, 17, n_hidden=256, n_layers=4, n_members=2, half=half, seed=3)
    layers = omlp.init_params(sur.sizes, seed=9)
    for W, b in layers:
        b[:] = rng.standard_normal(b.shape) * 0.1
    sur.set_params(1, sur.flatten(layers))
    ref = [[W.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)] for W, b in layers]
    X = rng.standard_normal((300, 7))
    T = rng.standard_normal((300, 17))
    y = sur.forward(1, X)
    y_ref, _ = omlp.forward(ref, X.astype(np.float32).astype(np.float64))
    assert _nrel(y, y_ref) <= tol_fwd, _nrel(y, y_ref)
    g, loss = sur.gradients(1, X, T)
    g_ref = omlp.gradients(ref, X.astype(np.float32).astype(np.float64), T.astype(np.float32).astype(np.float64))
    gl = sur.layers(g)
    errs = [(_nrel(gW, rW), _nrel(gb, rb)) for (gW, gb), (rW, rb) in zip(gl, g_ref)]
    print("half" if half else "bf16", "forward", _nrel(y, y_ref), "gradients per layer", errs)
    for i, (eW, eb) in enumerate(errs):
        assert eW <= tol and eb <= tol, (i, eW, eb)
    assert abs(loss - omlp.loss(ref, X, T)) <= tol * omlp.loss(ref, X, T)


def test_adam_step_matches_oracle(lbm):
    """One full-batch training step: new parameters equal the oracle's Adam
    update applied with the GPU's own gradient (so only the update is tested)."""
    rng = np.random.default_rng(6)
    sur = lbm.Surrogate(7, 17, n_hidden=64, n_layers=2, n_members=1, half=1, seed=4)
    p0 = sur.get_params(0)
    X = rng.standard_normal((128, 7))
    T = rng.standard_normal((128, 17))
    g, _ = sur.gradients(0, X, T)
    sur.train(X, T, epochs=1, batch=128, lr=1e-3, seed=1)
    p1 = sur.get_params(0)
    params = [[W.astype(np.float64), b.astype(np.float64)] for W, b in sur.layers(p0.copy())]
    grads = [[W.astype(np.float64), b.astype(np.float64)] for W, b in sur.layers(g)]
    omlp.adam_step(params, grads, {}, lr=1e-3)
    want = sur.flatten(params)
    assert np.allclose(p1, want, rtol=0, atol=2e-6), np.abs(p1 - want).max()


def test_training_reduces_loss_and_ensemble_spread(lbm):
    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (4096, 7)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0] * 2) + X[:, 1] * X[:, 2], np.cos(X[:, 3]) - 0.5 * X[:, 6]], axis=1)
    sur = lbm.Surrogate(7, 2, n_hidden=128, n_layers=3, n_members=3, half=0, seed=8)
    losses = sur.train(X, T, epochs=30, batch=256, lr=2e-3, seed=2)
    assert np.all(losses[:, -1] < 0.05 * losses[:, 0]), losses[:, [0, -1]]
    Xt = rng.uniform(-1, 1, (512, 7)).astype(np.float32)
    Tt = np.stack([np.sin(Xt[:, 0] * 2) + Xt[:, 1] * Xt[:, 2], np.cos(Xt[:, 3]) - 0.5 * Xt[:, 6]], axis=1)
    mean, spread = sur.predict(Xt)
    assert np.sqrt(np.mean((mean - Tt) ** 2)) < 0.1
    members = np.stack([sur.forward(m, Xt) for m in range(3)])
    assert np.allclose(mean, members.mean(axis=0), atol=1e-5)
    assert np.allclose(spread, members.std(axis=0, ddof=1), atol=1e-5)


def test_members_train_independently(lbm):
    """All members step together, one launch per layer: member 0 of a two-member
    ensemble ends bit for bit where the same member trained alone ends (same
    initialisation seed, same shuffle seed)."""
    rng = np.random.default_rng(11)
    X = rng.uniform(-1, 1, (700, 7)).astype(np.float32)
    T = np.stack([np.sin(X[:, 0]), X[:, 1] * X[:, 2]], axis=1)
    alone = lbm.Surrogate(7, 2, n_hidden=96, n_layers=2, n_members=1, half=0, seed=21)
    pair = lbm.Surrogate(7, 2, n_hidden=96, n_layers=2, n_members=2, half=0, seed=21)
    assert np.array_equal(alone.get_params(0), pair.get_params(0))
    la = alone.train(X, T, epochs=3, batch=128, lr=1e-3, seed=5)
    lp = pair.train(X, T, epochs=3, batch=128, lr=1e-3, seed=5)
    assert np.array_equal(alone.get_params(0), pair.get_params(0))
    assert not np.array_equal(pair.get_params(0), pair.get_params(1))
    assert np.allclose(la[0], lp[0], rtol=1e-12, atol=0)


def test_gemm_wait_gives_up_and_context_survives(lbm):
    """The surrogate GEMM's bounded wait for its MMAs, run with no MMA issued
    (a completion barrier nothing completes, limit 20 ms): the kernel gives up,
    reports it, frees its tensor memory, and the context runs a forward pass
    afterwards."""
    assert lbm.lbm_surrogate_selftest_wait(20000)
    rng = np.random.default_rng(12)
    sur = lbm.Surrogate(7, 3, n_hidden=64, n_layers=2, n_members=1, half=0, seed=5)
    y = sur.forward(0, rng.standard_normal((50, 7)))
    assert y.shape == (50, 3) and np.all(np.isfinite(y))
