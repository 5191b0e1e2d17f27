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
    loss, g = mlp.loss_and_grad(th, v, t)
    # every bias and output weight, and a sample of the matrix entries
    idx = np.concatenate([np.arange(8577 - 129, 8577), rng.choice(8577 - 129, 200, replace=False)])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(th)
        e[i] = h
        lp, _ = mlp.loss_and_grad(th + e, v, t)
        lm, _ = mlp.loss_and_grad(th - e, v, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])


def test_forward_is_logistic_of_a_silu_network():
    # output in (0, 1); zero weights give sigmoid(b4)
    th = np.zeros(mlp.N_PARAMS)
    th[-1] = 0.3
    x, _ = mlp.forward(th, mlp.inputs([0.5, -1.0], [0.2, 0.9]))
    np.testing.assert_allclose(x, 1 / (1 + np.exp(-0.3)), rtol=1e-15)
