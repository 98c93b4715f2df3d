"""Host-side pieces of the learned scheduler (no GPU): how judged rounds
become training labels, the initial weights, the input normalisation, and the
model blob layout that trim_set_model reads (parameters, mean, inverse std,
and the feature range in which the kernel trusts the model)."""
import numpy as np

from paper_2107_12720_gb300 import scheduler
from paper_2107_12720_gb300.abi import TRIM_MLP_NBLOB, TRIM_MLP_NIN, TRIM_MLP_NPARAMS


def test_judged_rounds_become_labels_and_ambiguous_ones_are_dropped():
    f = [float(i) for i in range(TRIM_MLP_NIN)]
    rows = [(f, {0: 1.0, 1: 2.0, 2: 3.0}),      # AC-4 best by 100%
            (f, {0: 1.00, 1: 1.02, 2: 5.0}),    # within 5%: ambiguous, dropped
            (f, {0: 4.0, 1: 3.0, 2: 1.5}),      # AC-3 best
            (f, {1: 2.0})]                      # one variant only: kept
    X, y, w = scheduler.rows_to_xy(rows)
    assert X.shape == (3, TRIM_MLP_NIN) and X.dtype == np.float32
    assert y.tolist() == [0, 2, 1]
    assert np.allclose(w[:2], [1.0, 1.5]) and np.isinf(w[2])


def test_initial_weights():
    theta = scheduler.he_init(0)
    assert theta.shape == (TRIM_MLP_NPARAMS,) and theta.dtype == np.float32
    W1, b1 = theta[:32 * 12], theta[32 * 12:32 * 13]
    W2, b2 = theta[32 * 13:32 * 13 + 32 * 32], theta[32 * 13 + 32 * 32:32 * 14 + 32 * 32]
    W3, b3 = theta[32 * 14 + 32 * 32:32 * 14 + 32 * 32 + 96], theta[-3:]
    assert not b1.any() and not b2.any() and not b3.any()
    for W, fan_in in ((W1, 12), (W2, 32), (W3, 32)):  # He-normal: std sqrt(2 / fan_in)
        assert abs(W.std() / np.sqrt(2.0 / fan_in) - 1.0) < 0.25
    assert np.array_equal(theta, scheduler.he_init(0))
    assert not np.array_equal(theta, scheduler.he_init(1))


def test_normalisation_keeps_constant_features():
    X = np.array([[1.0, 5.0], [3.0, 5.0]], np.float32)
    mean, istd = scheduler.normalisation(X)
    assert np.allclose(mean, [2.0, 5.0]) and np.allclose(istd, [1.0, 1.0])
    X = np.array([[0.0, 5.0], [4.0, 5.0]], np.float32)
    mean, istd = scheduler.normalisation(X)
    assert np.allclose(istd, [0.5, 1.0])


def test_blob_layout_and_trusted_range():
    rng = np.random.default_rng(0)
    X = rng.uniform(0, 10, (50, TRIM_MLP_NIN)).astype(np.float32)
    theta = scheduler.he_init(2)
    mean, istd = scheduler.normalisation(X)
    blob = scheduler.make_blob(theta, mean, istd, X, margin=0.25)
    assert blob.shape == (TRIM_MLP_NBLOB,) and blob.dtype == np.float32
    k = TRIM_MLP_NPARAMS
    assert np.array_equal(blob[:k], theta)
    assert np.array_equal(blob[k:k + 12], mean) and np.array_equal(blob[k + 12:k + 24], istd)
    lo, hi = blob[k + 24:k + 36], blob[k + 36:k + 48]
    span = X.max(axis=0) - X.min(axis=0)
    for i in range(TRIM_MLP_NIN):
        extra = scheduler.LOG2_MARGIN if i in scheduler.LOG2_FEATURES else 0.0
        assert np.isclose(lo[i], X[:, i].min() - 0.25 * span[i] - extra, atol=1e-4)
        assert np.isclose(hi[i], X[:, i].max() + 0.25 * span[i] + extra, atol=1e-4)


def test_committed_model_blob():
    blob = scheduler.load_blob()
    assert blob.shape == (TRIM_MLP_NBLOB,) and np.isfinite(blob).all()
    k = TRIM_MLP_NPARAMS
    istd = blob[k + 12:k + 24]
    lo, hi = blob[k + 24:k + 36], blob[k + 36:k + 48]
    assert (istd > 0).all() and (lo < hi).all()
