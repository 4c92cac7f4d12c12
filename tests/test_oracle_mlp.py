"""Pins of the warm-start oracle (oracle/mlp.py) against mathematics and
hand-worked values, independent of the oracle's own formulas."""
import math

import numpy as np

from oracle import mlp


def test_gelu_closed_form_and_derivative():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    # Phi(1) = 0.841344746...: GELU(1) = Phi(1), GELU(-1) = -(1 - Phi(1))
    assert abs(mlp.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-12
    assert abs(mlp.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-12
    assert abs(mlp.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    x = np.linspace(-4, 4, 17)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.max(np.abs(fd - mlp.gelu_grad(x))) < 1e-8


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    p = mlp.init_params(seed=5)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)   # nonzero biases too
    X = rng.standard_normal((9, mlp.NF))
    t = rng.standard_normal(9)
    y, cache = mlp.forward(p, X)
    g = mlp.backward(p, cache, y, t)
    h = 1e-6
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(mlp.forward(p, X)[0], t)
            flat[idx] = old - h
            lm = mlp.loss(mlp.forward(p, X)[0], t)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)


def test_adam_first_step_is_signed_lr():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    opt = mlp.Adam(p, lr=0.01, eps=1e-12)
    opt.step(p, {"w": np.array([0.5, -4.0, 1e-3])})
    assert np.allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], atol=1e-9)


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -3.0, 65504.0, 1.0 + 2.0 ** -7], dtype=np.float32)
    out = mlp.bf16(vals)
    # 8 significant bits: ulp(1) = 2^-7; exact half-ulp ties go to even
    assert out[0] == 1.0
    assert out[1] == 1.0
    assert out[2] == np.float32(1.0 + 2.0 ** -6)
    assert out[3] == -3.0
    assert out[4] == 65536.0
    assert out[5] == np.float32(1.0 + 2.0 ** -7)


def test_features_of_a_hand_built_3x3_state():
    # every bond at chi 2 with lam = (cos a, sin a); bond 0 at chi 1
    Lx = Ly = 3
    nb = 12
    a = 0.3
    chi = np.full(nb, 2)
    chi[0] = 1
    lam = np.zeros((nb, 2))
    lam[:, 0] = math.cos(a)
    lam[:, 1] = math.sin(a)
    lam[0] = [1.0, 0.0]
    X, idx = mlp.features(Lx, Ly, (1, 1), chi, lam, step=3, dt=0.05, h=2.0, J=1.0)
    # rows: bond 0 has one row per direction, the other 11 bonds two per direction
    assert X.shape == (2 * 1 + 11 * 4, mlp.NF)
    p = np.array([math.cos(a) ** 2, math.sin(a) ** 2])
    s = -(p * np.log(p)).sum() / math.log(2)
    # bond 1 = (1,0)-(2,0), direction 0: source site 1 (edge, deg 3), target 2 (corner)
    r = [i for i in range(len(idx)) if tuple(idx[i]) == (1, 0, 1)][0]
    row = X[r]
    assert abs(row[0] - math.log(math.sin(a))) < 1e-12
    assert row[1] == 0.5
    assert abs(row[2] - s) < 1e-12
    assert row[3] == 0.75 and row[4] == 0.5
    assert row[5] == 1 / 6 and row[6] == 2 / 6          # |1-1|+|0-1| = 1, |2-1|+|0-1| = 2
    assert abs(row[7] - 0.15) < 1e-15 and row[8] == 2.0 and row[9] == 1.0
    # other bonds of site 1: bond 0 (chi 1, fraction 0) and the vertical bond below it (fraction s)
    assert abs(row[10] - s / 2) < 1e-12 and abs(row[11] - s) < 1e-12
    # bond 0 at chi 1: log lam = 0, fraction 0
    r0 = [i for i in range(len(idx)) if tuple(idx[i]) == (0, 1, 0)][0]
    assert X[r0][0] == 0.0 and X[r0][2] == 0.0
    # centre site has degree 4
    rc = [i for i in range(len(idx)) if tuple(idx[i]) == (3, 1, 0)][0]   # bond 3 = (1,1)-(2,1), dir 1: source 5
    assert X[rc][3] == 0.75 and X[rc][4] == 1.0


def test_warm_message_is_trace_one_diagonal():
    M = mlp.warm_message(np.log(np.array([4.0, 2.0, 2.0])))
    assert np.allclose(M, np.diag([0.5, 0.25, 0.25]))


def test_warm_message_blend():
    M = mlp.warm_message(np.log(np.array([4.0, 2.0, 2.0])), plain_diag=np.array([1.0, 1.0, 0.0]), gamma=0.5)
    assert np.allclose(np.diag(M), [0.5 * 0.5 + 0.5 * 0.5, 0.5 * 0.5 + 0.5 * 0.25, 0.5 * 0.25])
    assert abs(np.trace(M) - 1.0) < 1e-15
