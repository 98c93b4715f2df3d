"""Pins of the double-precision scheduler-MLP reference (CPU): central finite
differences of the loss, closed forms of special parameter settings, and the
Adam update written out for one step."""
import numpy as np

from oracle import mlp_ref as R


def random_problem(seed=0, N=64, scale=0.5):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, scale, R.NPARAMS)
    X = rng.normal(0, 1, (N, R.NIN))
    y = rng.integers(0, 3, N)
    return theta, X, y


def test_parameter_count_matches_the_abi():
    assert R.NPARAMS == 1571


def test_gradient_matches_central_differences():
    theta, X, y = random_problem(1)
    L, g = R.loss_grad(theta, X, y)
    assert abs(L - R.loss(theta, X, y)) < 1e-12
    fd = R.finite_difference_grad(theta, X, y)
    err = np.abs(fd - g).max() / max(1e-12, np.abs(g).max())
    assert err < 1e-6, err


def test_zero_network_is_uniform():
    """All-zero parameters: every logit is 0, p = 1/3, loss = ln 3; only the
    output bias gets a gradient, mean(p - onehot(y))."""
    theta = np.zeros(R.NPARAMS)
    _, X, y = random_problem(2)
    L, g = R.loss_grad(theta, X, y)
    assert abs(L - np.log(3.0)) < 1e-12
    P = R.unpack(g)
    onehot = np.eye(3)[y]
    np.testing.assert_allclose(P["b3"], (1 / 3 - onehot).mean(axis=0), atol=1e-12)
    for k in ["W1", "b1", "W2", "b2", "W3"]:
        assert np.abs(P[k]).max() == 0.0


def test_bias_only_network_is_multinomial_regression():
    """With W3 = 0 the logits are b3 for every row: the loss is the cross-entropy
    of the label histogram against softmax(b3)."""
    theta, X, y = random_problem(3)
    P = R.unpack(theta)
    P["W3"] = np.zeros_like(P["W3"])
    theta = R.pack(P)
    b3 = P["b3"]
    logp = b3 - np.log(np.exp(b3).sum())
    counts = np.bincount(y, minlength=3) / len(y)
    assert abs(R.loss(theta, X, y) - float(-(counts * logp).sum())) < 1e-12


def test_relu_dead_units_get_no_gradient():
    """Hidden units whose pre-activation is negative on every row pass no gradient."""
    theta, X, y = random_problem(4)
    P = R.unpack(theta)
    P["b1"][:5] = -1e6  # units 0..4 of layer 1 never fire
    theta = R.pack(P)
    _, g = R.loss_grad(theta, X, y)
    G = R.unpack(g)
    assert np.abs(G["W1"][:5]).max() == 0 and np.abs(G["b1"][:5]).max() == 0
    assert np.abs(G["W2"][:, :5]).max() == 0


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 the bias-corrected moments are g and g^2: the step is
    lr * g / (|g| + eps), i.e. lr * sign(g) for |g| >> eps."""
    theta, X, y = random_problem(5)
    _, g = R.loss_grad(theta, X, y)
    new, m, v = R.adam_step(theta, g, np.zeros_like(g), np.zeros_like(g), 1, lr=1e-3)
    big = np.abs(g) > 1e-4
    np.testing.assert_allclose((theta - new)[big], 1e-3 * np.sign(g[big]), rtol=1e-3)
