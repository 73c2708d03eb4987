"""Pins of the CPU reference of the selector network: its analytic gradient
against central finite differences (plain float64 network), the BF16
rounding against its definition, and a closed-form case."""
import numpy as np

from oracle import mlp_oracle as R


def random_problem(n=64, seed=0):
    rng = np.random.default_rng(seed)
    p = rng.normal(size=R.NPARAM) * 0.2
    X = rng.normal(size=(n, R.NF))
    y = (rng.random(n) < 0.4).astype(float)
    w = rng.uniform(0.5, 2.0, n)
    return p, X, y, w


def test_gradient_matches_central_differences():
    p, X, y, w = random_problem()
    _, g = R.loss_and_grad(p, X, y, w, quantise=False)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(R.P_B1, 40, replace=False),                 # W1
                          R.P_B1 + rng.choice(R.NH, 10, replace=False),           # b1
                          R.P_W2 + rng.choice(R.NH * R.NH, 40, replace=False),    # W2
                          R.P_B2 + rng.choice(R.NH, 10, replace=False),           # b2
                          R.P_W3 + rng.choice(R.NH, 10, replace=False), [R.P_B3]])
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (R.loss_and_grad(pp, X, y, w, quantise=False)[0] - R.loss_and_grad(pm, X, y, w, quantise=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-8, (i, fd, g[i])


def test_bf16_rounding():
    # exactly representable values are kept; ties go to even; 1 + 2^-9 rounds to 1
    v = np.array([1.0, 1.5, -2.0, 1.0 + 2.0 ** -8, 1.0 + 2.0 ** -9, 1.0 + 3 * 2.0 ** -9], dtype=np.float32)
    out = R.bf16(v)
    assert out[0] == 1.0 and out[1] == 1.5 and out[2] == -2.0
    assert out[3] == 1.0          # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even, 1
    assert out[4] == 1.0
    assert out[5] == 1.0 + 2.0 ** -7
    x = np.random.default_rng(2).normal(size=1000).astype(np.float32)
    assert np.all(np.abs(R.bf16(x) - x) <= np.abs(x) * 2.0 ** -8 + 1e-30)


def test_zero_weights_give_log2_loss():
    p = np.zeros(R.NPARAM)
    X = np.random.default_rng(3).normal(size=(10, R.NF))
    y = np.array([0, 1] * 5, dtype=float)
    loss, g = R.loss_and_grad(p, X, y)
    assert abs(loss - np.log(2.0)) < 1e-15
    assert abs(g[R.P_B3] - 0.0) < 1e-15           # sigmoid(0) - y averages to zero
    assert np.all(g[:R.P_W3] == 0.0)              # dead ReLUs pass no gradient
