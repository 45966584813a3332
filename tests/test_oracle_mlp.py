"""Pins of the FP64 MLP oracle: central finite differences of the loss, a
hand-worked two-layer case, ReLU's kink handling and the first Adam step's
closed form (|update| = lr for every parameter with a non-zero gradient)."""
import numpy as np

from oracle import mlp


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    sizes = [7, 16, 16, 5]
    params = mlp.init_params(sizes, seed=3)
    X = rng.standard_normal((9, 7))
    Y = rng.standard_normal((9, 5))
    grads = mlp.gradients(params, X, Y)
    h = 1e-6
    worst = 0.0
    for i in range(len(params)):
        for j in range(2):
            P = params[i][j]
            flat = P.reshape(-1)
            for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = mlp.loss(params, X, Y)
                flat[idx] = old - h
                lm = mlp.loss(params, X, Y)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[i][j].reshape(-1)[idx]
                worst = max(worst, abs(fd - an) / max(1e-8, abs(fd) + abs(an)))
    assert worst <= 1e-6, worst


def test_hand_worked_two_layer():
    """x = [1, 2], W0 = [[1, -1], [0.5, 0.5]], b0 = [1.5, 0] -> z0 = h = [0.5, 1.5];
    W1 = [[2, -1]], b1 = [0.25] -> y = 1 - 1.5 + 0.25 = -0.25; target 0.75 ->
    loss 1, dL/dy = -2, worked by hand below."""
    params = [[np.array([[1.0, -1.0], [0.5, 0.5]]), np.array([1.5, 0.0])],
              [np.array([[2.0, -1.0]]), np.array([0.25])]]
    X = np.array([[1.0, 2.0]])
    Y = np.array([[0.75]])
    y, _ = mlp.forward(params, X)
    assert y[0, 0] == -0.25
    assert mlp.loss(params, X, Y) == 1.0
    g = mlp.gradients(params, X, Y)
    assert np.array_equal(g[1][0], np.array([[-1.0, -3.0]]))  # dy * h
    assert np.array_equal(g[1][1], np.array([-2.0]))
    # dh = dy * W1 = [-4, 2]; both units active -> dz0 = [-4, 2]
    assert np.array_equal(g[0][0], np.array([[-4.0, -8.0], [2.0, 4.0]]))
    assert np.array_equal(g[0][1], np.array([-4.0, 2.0]))


def test_relu_blocks_gradient_of_inactive_units():
    params = [[np.array([[1.0], [-1.0]]), np.array([0.0, 0.0])], [np.array([[1.0, 1.0]]), np.array([0.0])]]
    X = np.array([[2.0]])
    g = mlp.gradients(params, X, np.array([[0.0]]))
    assert g[0][0][1, 0] == 0.0 and g[0][1][1] == 0.0  # unit 2 is inactive (z = -2)
    assert g[0][0][0, 0] != 0.0


def test_first_adam_step_has_size_lr():
    rng = np.random.default_rng(4)
    params = mlp.init_params([3, 4, 2], seed=5)
    before = [[W.copy(), b.copy()] for W, b in params]
    X = rng.standard_normal((6, 3))
    Y = rng.standard_normal((6, 2))
    grads = mlp.gradients(params, X, Y)
    state = {}
    mlp.adam_step(params, grads, state, lr=0.01)
    for i in range(len(params)):
        for j in range(2):
            step = np.abs(params[i][j] - before[i][j])
            nz = np.abs(grads[i][j]) > 1e-12
            assert np.allclose(step[nz], 0.01, rtol=1e-6)
