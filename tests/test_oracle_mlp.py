"""Pin of the oracle's FP64 sampler network: its hand-written backward pass
agrees with central finite differences of its own loss, parameter by
parameter, and the packing is a bijection.  CPU only."""
import numpy as np

from oracle import mlp


def test_parameter_count_and_packing():
    assert mlp.N_PARAMS == 8577
    th = mlp.init(3)
    assert th.shape == (8577,)
    np.testing.assert_array_equal(mlp.pack(mlp.unpack(th)), th)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    th = mlp.init(1)
    v = mlp.inputs(rng.uniform(-2, 2, 32), rng.uniform(0, 1, 32))
    t = rng.uniform(0.05, 0.95, 32)
    wt = rng.uniform(0.5, 2.0, 32)
    loss, g = mlp.loss_and_grad(th, v, t, wt)
    # every bias and output weight, and a sample of the matrix entries
    idx = np.concatenate([np.arange(8577 - 129, 8577), rng.choice(8577 - 129, 200, replace=False)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        lp, _ = mlp.loss_and_grad(th + e, v, t, wt)
        lm, _ = mlp.loss_and_grad(th - e, v, t, wt)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_forward_is_logistic_of_a_silu_network():
    # zero weights give sigmoid(b4 + logit u) = u e^b4 / (1 - u + u e^b4)
    th = np.zeros(mlp.N_PARAMS)
    th[-1] = 0.3
    u = np.array([0.2, 0.9])
    x, _ = mlp.forward(th, mlp.inputs([0.5, -1.0], u))
    e = np.exp(0.3)
    np.testing.assert_allclose(x, u * e / (1 - u + u * e), rtol=1e-14)
    # and b4 = 0 is the identity u -> x, with the end points fixed
    th[-1] = 0.0
    u = np.array([1e-9, 0.37, 1 - 1e-9])
    x, _ = mlp.forward(th, mlp.inputs(np.zeros(3), u))
    np.testing.assert_allclose(x, u, rtol=1e-6)
