"""Pins of the learned-alpha oracle: backpropagation against central finite differences, and the
first Adam step against its closed form (each parameter moves by lr * sign(g))."""
import numpy as np

from oracle import mlp


def _model(seed=0):
    rng = np.random.default_rng(seed)
    m = np.zeros(mlp.MODEL_FLOATS)
    m[:mlp.NPARAM] = rng.normal(0, 0.3, mlp.NPARAM)
    m[mlp.NPARAM:mlp.NPARAM + 4] = rng.normal(0, 1, 4)           # mean
    m[mlp.NPARAM + 4:mlp.NPARAM + 8] = rng.uniform(0.5, 2, 4)    # std
    m[-2], m[-1] = -3.0, 1.5
    return m


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    model = _model()
    X = rng.normal(0, 1, (37, 4))
    t = rng.normal(-3, 1.5, 37)
    L, g = mlp.loss_and_grad(model, X, t)
    assert g.shape == (mlp.NPARAM,)
    idx = rng.choice(mlp.NPARAM, 60, replace=False).tolist() + [0, mlp.NPARAM - 1]
    h = 1e-6
    for k in idx:
        mp, mm = model.copy(), model.copy()
        mp[k] += h
        mm[k] -= h
        fd = (mlp.loss_and_grad(mp, X, t)[0] - mlp.loss_and_grad(mm, X, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(g[k])), k


def test_first_adam_step_is_lr_sign_g():
    rng = np.random.default_rng(2)
    model = _model(3)
    X = rng.normal(0, 1, (20, 4))
    t = rng.normal(-3, 1.5, 20)
    _, g = mlp.loss_and_grad(model, X, t)
    new, hist = mlp.adam_train(model, X, t, epochs=1, lr=1e-3, eps=0.0)
    step = model[:mlp.NPARAM] - new[:mlp.NPARAM]
    nz = np.abs(g) > 0
    assert np.allclose(step[nz], 1e-3 * np.sign(g[nz]), rtol=1e-12, atol=0)
    assert np.array_equal(new[mlp.NPARAM:], model[mlp.NPARAM:])   # normalisation untouched


def test_training_reduces_loss():
    rng = np.random.default_rng(4)
    model = _model(5)
    X = rng.normal(0, 1, (64, 4))
    t = -2.0 + np.tanh(X[:, 0]) - 0.5 * X[:, 1]
    _, hist = mlp.adam_train(model, X, t, epochs=200, lr=1e-2)
    assert hist[-1] < 0.2 * hist[0]
