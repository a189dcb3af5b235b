"""Pins for the FP64 reference of the learned opening-angle network:
finite differences, closed forms of GELU, the loss and Adam, BF16 rounding
against torch's conversion, and the zero-weight special case."""
import math

import numpy as np
import pytest

import nbsynth
from oracle import mlp


def params(seed=3, scale=1.0):
    w = nbsynth.mlp_initial_weights(seed)
    rng = np.random.default_rng(seed + 100)
    return mlp.pack_params(w["W1"] * scale, rng.normal(0, 0.1, 64), w["W2"] * scale,
                           rng.normal(0, 0.1, 64), w["W3"] * scale, rng.normal(0, 0.1, 64),
                           w["w4"], 0.2, rng.normal(0, 1, 12), rng.uniform(0.5, 2, 12))


def data(n=40, seed=4):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 1.5, (n, 12)), rng.uniform(0.3, 1.2, n)


def test_gradient_matches_finite_differences():
    p = params().astype(np.float64)
    x, y = data()
    L, g = mlp.backward(p, x, y)
    rng = np.random.default_rng(0)
    trainable = np.flatnonzero(g != 0)
    idx = rng.choice(trainable, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss(mlp.forward(pp, x)[0], y) - mlp.loss(mlp.forward(pm, x)[0], y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-9


def test_gradient_zero_on_padding_and_normalisation():
    p = params().astype(np.float64)
    x, y = data()
    _, g = mlp.backward(p, x, y)
    W1g = g[mlp.OFF["W1"]:mlp.OFF["W1"] + 64 * 16].reshape(64, 16)
    assert np.all(W1g[:, 12:] == 0)
    assert np.all(g[mlp.OFF["mu"]:] == 0)
    assert np.all(g[mlp.OFF["w4"] + 64:mlp.OFF["b4"]] == 0)


def test_gelu_closed_forms():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu(np.array([10.0]))[0] == pytest.approx(10.0, rel=1e-15)
    assert abs(mlp.gelu(np.array([-10.0]))[0]) < 1e-20
    assert mlp.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    # gelu(1) = Phi(1) = 0.841344746...
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, rel=1e-14)


def test_zero_weights_give_sigmoid_of_bias():
    z = np.zeros((64, 64))
    p = mlp.pack_params(np.zeros((64, 12)), np.zeros(64), z, np.zeros(64), z, np.zeros(64),
                        np.zeros(64), 0.7, np.zeros(12), np.ones(12))
    th, _ = mlp.forward(p, np.random.default_rng(1).normal(size=(5, 12)))
    assert np.allclose(th, 0.3 + 0.9 / (1 + math.exp(-0.7)), rtol=1e-7)


def test_loss_penalises_overprediction_five_fold():
    assert mlp.loss(np.array([0.6]), np.array([0.5])) == pytest.approx(5 * 0.01)
    assert mlp.loss(np.array([0.4]), np.array([0.5])) == pytest.approx(0.01)


def test_first_adam_step_is_lr_times_sign():
    g = np.array([0.3, -2.0, 0.0, 1e-3])
    p1, m, v = mlp.adam(np.zeros(4), np.zeros(4), np.zeros(4), g, 1, 0.01)
    assert np.allclose(p1, -0.01 * np.sign(g), atol=1e-10)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    x = np.random.default_rng(2).normal(0, 3, 10000).astype(np.float32)
    x[:4] = [1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -0.0]
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_bf16_forward_close_to_fp64_forward():
    p = params()
    x, _ = data(200)
    t64, _ = mlp.forward(p, x)
    t16, _ = mlp.forward(p, x, bf=True)
    assert np.max(np.abs(t64 - t16)) < 0.02
    assert not np.array_equal(t64, t16)


def test_features_closed_form_two_clumps(oracle_lib):
    # two tight clumps far apart: each is a group whose probe list is the
    # other clump's cell, so every feature has a closed form
    from oracle import features
    rng = np.random.default_rng(0)
    a = 0.001 * rng.normal(size=(20, 3)) + [-1.0, -1.0, -1.0]   # octant 0
    b = 0.001 * rng.normal(size=(20, 3)) + [1.0, 1.0, 1.0]      # octant 7
    pos = np.vstack([a, b])
    mass = np.full(40, 0.025, np.float32)
    T = oracle_lib.Tree(pos, mass)
    f = features.group_features(T, 20)
    gnode = T.groups(20)
    assert len(gnode) == 2
    box = T.group_boxes(gnode)
    e = T.export()
    for k, other in ((0, b), (1, a)):
        lo, hi = box[k, :3].astype(np.float64), box[k, 3:6].astype(np.float64)
        side = (hi - lo) / T.L
        assert f[k, 0] == pytest.approx(np.log(20))
        assert np.allclose(f[k, 1:4], np.log(side + 1e-7))
        assert f[k, 6] == pytest.approx(np.log(2.0)) and f[k, 7] == 1.0
        com = other.mean(0)
        d = np.linalg.norm(com - box[k, 6:9].astype(np.float64)) / T.L
        assert np.allclose(f[k, 8:11], np.log(d + 1e-7), atol=1e-6)
