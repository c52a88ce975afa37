"""The surrogate's CUDA training and inference kernels against the FP64
perceptron oracle (FP32 accumulation: gradients within 1e-4 of the largest
component, outputs within 1e-5 relative)."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_7228_gb300 import lbm
    lbm.lib()
    return lbm


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.uniform(0.6, 0.85, n), rng.uniform(-0.9, -0.8, n), rng.uniform(0, 0.6, n)], 1)
    Y = np.stack([(1 - X[:, 2]) * (0.9 - X[:, 0]) * 0.05, 0.3 + 0.2 * (0.85 - X[:, 0]),
                  0.02 * X[:, 0] ** 3, 1e-3 * (1 + X[:, 1])], 1)
    return X, Y


def _std(X, Y):
    return X.mean(0), X.std(0), Y.mean(0), Y.std(0)


@pytest.mark.parametrize("n", [200, 64, 13])
def test_loss_and_gradient_match_oracle(L, n):
    X, Y = _data(n, n)
    mlp = L.Mlp(max_samples=512, seed=11)
    im, isd, om, osd = _std(X, Y)
    mlp.set_normalization(im, isd, om, osd)
    p = mlp.get_params().astype(np.float64)
    Xs = ((X - im) / isd).astype(np.float32).astype(np.float64)
    Ys = ((Y - om) / osd).astype(np.float32).astype(np.float64)
    loss_g, g_g = mlp.loss_grad(X, Y)
    loss_o, g_o = M.loss_grad(p, Xs, Ys)
    assert abs(loss_g / loss_o - 1) < 1e-5
    assert np.abs(g_g - g_o).max() <= 1e-4 * np.abs(g_o).max()
    mlp.close()


def test_predict_matches_oracle(L):
    X, Y = _data(300, 5)
    mlp = L.Mlp(max_samples=512, seed=2)
    im, isd, om, osd = _std(X, Y)
    mlp.set_normalization(im, isd, om, osd)
    p = mlp.get_params().astype(np.float64)
    ys = M.forward(p, (X - im) / isd)[0] * osd + om
    got = mlp.predict(X)
    assert np.abs(got - ys).max() <= 1e-5 * np.abs(ys).max() + 1e-7
    mlp.close()


def test_adam_steps_match_oracle(L):
    """Three Adam steps.  Where a gradient component is near zero its
    normalised step m/sqrt(v) is ill-conditioned (FP32 may even flip its
    sign), so the comparison covers components with |g| > 1e-3 max|g|."""
    X, Y = _data(150, 8)
    mlp = L.Mlp(max_samples=256, seed=3)
    im, isd, om, osd = _std(X, Y)
    mlp.set_normalization(im, isd, om, osd)
    p = mlp.get_params().astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    Xs = ((X - im) / isd).astype(np.float32).astype(np.float64)
    Ys = ((Y - om) / osd).astype(np.float32).astype(np.float64)
    mask = None
    for t in range(1, 4):
        mlp.adam_step(X, Y, lr=1e-3)
        _, g = M.loss_grad(p, Xs, Ys)
        ok = np.abs(g) > 1e-3 * np.abs(g).max()
        mask = ok if mask is None else (mask & ok)
        p, m, v = M.adam(p, m, v, t, g, 1e-3)
    assert mask.sum() > 0.9 * mask.size
    assert np.abs(mlp.get_params()[mask] - p[mask]).max() <= 2e-6
    mlp.close()


def test_training_fits_and_inverse_hits_targets(L):
    """Train on a smooth sigma(T, A, kappa) decreasing in kappa; the GPU
    bisection returns kappas whose FP64-oracle prediction hits each target."""
    X, Y = _data(2000, 21)
    mlp = L.Mlp(max_samples=2048, seed=4)
    im, isd, om, osd = _std(X, Y)
    mlp.set_normalization(im, isd, om, osd)
    losses = mlp.train(X, Y, epochs=150, batch=128, lr=3e-3, seed=1)
    assert losses[-1] < 0.02 * losses[0]
    rng = np.random.default_rng(9)
    tr = rng.uniform(0.62, 0.83, 16)
    A = rng.uniform(-0.88, -0.82, 16)
    kt = rng.uniform(0.05, 0.55, 16)
    sig = (1 - kt) * (0.9 - tr) * 0.05
    k = mlp.invert_kappa(tr, A, sig, 0.0, 0.6)
    assert np.all(np.isfinite(k))
    p = mlp.get_params().astype(np.float64)
    x = np.stack([tr, A, k], 1)
    pred = M.forward(p, (x - im) / isd)[0][:, 0] * osd[0] + om[0]
    assert np.abs(pred / sig - 1).max() < 1e-3
    assert np.abs(k - kt).max() < 0.05          # and the function was learnt well
    mlp.close()
