"""Learned alpha: the CUDA forward/backward/Adam kernels against the FP64 oracle, and the gain of
the trained network over the paper's alpha rule and over a fixed alpha on held-out problems."""
import numpy as np
import pytest

from oracle import mlp
from workloads import fractional_problem, rhs_uniform
from _gpu_helpers import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_07749_gb300 import build
    build.build()
    import paper_2307_07749_gb300 as mod
    return mod


def _data(seed, n=300):
    rng = np.random.default_rng(seed)
    X = np.stack([rng.uniform(3, 7, n), rng.uniform(3, 10, n), rng.uniform(0.2, 1, n),
                  rng.uniform(-2, 6, n)], 1)
    t = -2.5 + 0.4 * np.tanh(X[:, 3] - 2) - 0.3 * (X[:, 2] - 0.5) + 0.05 * rng.normal(size=n)
    return X, t


def _model(B, X, t, seed):
    from paper_2307_07749_gb300 import learned_alpha as LA
    return LA.init_model(X, t, seed)


def test_grad_matches_oracle(B):
    X, t = _data(1)
    model = _model(B, X, t, 3)
    g, loss = B.bltt_alpha_grad(model, X, t)
    L, gref = mlp.loss_and_grad(model.astype(np.float64), X.astype(np.float32), t.astype(np.float32))
    assert abs(loss - L) <= 1e-5 * max(1.0, L)
    assert np.linalg.norm(g - gref) <= 1e-4 * np.linalg.norm(gref)


def test_train_matches_oracle(B):
    X, t = _data(2)
    model = _model(B, X, t, 4)
    gm, gh = B.bltt_alpha_train(model, X, t, epochs=20, lr=3e-3)
    rm, rh = mlp.adam_train(model.astype(np.float64), X.astype(np.float32), t.astype(np.float32),
                            epochs=20, lr=3e-3)
    assert np.allclose(gh, rh, rtol=2e-4, atol=1e-6)
    # Adam normalises each step, so a parameter whose gradient is near zero may move by a few
    # lr in either precision: compare the parameter vectors normwise with that slack
    p = mlp.NPARAM
    assert np.linalg.norm(gm[:p] - rm[:p]) <= 5e-3 * np.linalg.norm(rm[:p])


def test_predict_matches_oracle(B):
    X, t = _data(3)
    model, _ = B.bltt_alpha_train(_model(B, X, t, 5), X, t, epochs=200, lr=3e-3)
    a = B.bltt_alpha_predict(model, X)
    aref = mlp.predict(model.astype(np.float64), X.astype(np.float32))
    assert np.max(np.abs(np.log10(a) - np.log10(aref))) <= 1e-4


def _family(seed, count):
    rng = np.random.default_rng(seed)
    out = []
    for j in range(count):
        m = int(rng.choice([15, 31, 63]))
        N = int(rng.choice([32, 64, 128]))
        p = fractional_problem(1, m, N, float(rng.uniform(0.2, 0.9)))
        sd = int(rng.integers(1 << 30))
        out.append((p, (lambda p=p, sd=sd: rhs_uniform(p.n, sd))))
    return out


def test_learned_alpha_beats_the_fixed_rules(B):
    """FP32-preconditioner form: on held-out problems the network trained on this solver's own
    sweeps needs no more iterations in total than the best fixed alpha, which is picked with
    hindsight on the held-out set itself, and far fewer than the paper's alpha = 1e-8, with which
    the FP32 form does not converge."""
    from paper_2307_07749_gb300 import learned_alpha as LA
    train_set, held = _family(11, 80), _family(12, 16)
    X, t, _ = LA.build_dataset(train_set)
    assert len(t) >= 60
    model, hist = LA.train(X, t, epochs=3000, lr=3e-3, seed=0)
    assert hist[-1] < hist[0]
    probs = [p for p, _ in held]
    alphas = LA.predict(model, probs)

    def iters(alpha_of):
        tot = []
        for (p, rf), a in zip(held, alpha_of):
            s = B.Solver(p)
            _, info = s.solve(to_dev(rf()), alpha=a, tol=1e-8, maxit=60, precision=32, basis=1,
                              matvec_arith=2, raise_on_error=False)
            tot.append(info["iters"] if info["status"] == 0 else 60)
        return np.array(tot)

    learned = iters(alphas)
    best_fixed = min((iters([a] * len(held)).sum(), a) for a in (1e-2, 3e-3, 1e-3, 1e-4))
    paper = iters([1e-8] * len(held))
    assert learned.sum() <= best_fixed[0], (learned.sum(), best_fixed)
    assert learned.sum() < paper.sum()
