"""Tensor-core MLP kernels (forward, backward, Adam) against the FP64 oracle
with the same BF16 operand rounding."""
import numpy as np
import pytest

import nbsynth
from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

BLOCKS = [("W1", 0, 1024), ("b1", 1024, 1088), ("W2", 1088, 5184), ("b2", 5184, 5248),
          ("W3", 5248, 9344), ("b3", 9344, 9408), ("w4", 9408, 9472), ("b4", 9920, 9921)]


def params(seed=3):
    w = nbsynth.mlp_initial_weights(seed)
    rng = np.random.default_rng(seed + 100)
    return mlp.pack_params(w["W1"], rng.normal(0, 0.1, 64), w["W2"], rng.normal(0, 0.1, 64),
                           w["W3"], rng.normal(0, 0.1, 64), w["w4"], 0.2,
                           rng.normal(0, 1, 12), rng.uniform(0.5, 2, 12))


def data(n, seed=4):
    rng = np.random.default_rng(seed)
    f = np.zeros((n, 16), np.float32)
    f[:, :12] = rng.normal(0, 1.5, (n, 12))
    return f, rng.uniform(0.3, 1.2, n).astype(np.float32)


@pytest.mark.parametrize("n", [16, 100, 1000])
def test_forward_and_gradient(n):
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    p = params()
    f, y = data(n)
    P = torch.from_numpy(p).to(dev)
    F = torch.from_numpy(f).to(dev)
    Y = torch.from_numpy(y).to(dev)
    th = nb.mlp_forward(P, F).cpu().numpy()
    th_or, _ = mlp.forward(p, f[:, :12], bf=True)
    assert np.max(np.abs(th - th_or)) < 2e-3
    g, loss = nb.mlp_grad(P, F, Y)
    g = g.cpu().numpy()
    L_or, g_or = mlp.backward(p, f[:, :12], y, bf=True)
    assert abs(loss.item() / n - L_or) <= 1e-3 * L_or
    for name, a, b in BLOCKS:
        ref = g_or[a:b]
        err = np.linalg.norm(g[a:b] - ref) / max(np.linalg.norm(ref), 1e-12)
        assert err < 2e-2, (name, err)


def test_first_adam_step_and_training():
    import paper_0909_0541_gb300 as nb
    dev = torch.device("cuda")
    p = params(7)
    f, y = data(256, 9)
    P = torch.from_numpy(p).to(dev)
    F = torch.from_numpy(f).to(dev)
    Y = torch.from_numpy(y).to(dev)
    order = torch.arange(256, dtype=torch.int32, device=dev).reshape(1, 256)
    lr = 1e-3
    nb.mlp_train(P, F, Y, order, epochs=1, batch=256, lr=lr)
    step = P.cpu().numpy().astype(np.float64) - p
    _, g_or = mlp.backward(p, f[:, :12], y, bf=True)
    p1, _, _ = mlp.adam(p, np.zeros_like(g_or), np.zeros_like(g_or), g_or, 1, lr)
    ref = p1 - p
    big = np.abs(g_or) > 1e-4 * np.abs(g_or).max()
    agree = np.isclose(step[big], ref[big], rtol=1e-3, atol=1e-9)
    assert agree.mean() > 0.98
    # training on a learnable target lowers the loss by an order of magnitude
    rng = np.random.default_rng(12)
    n = 4096
    f2 = np.zeros((n, 16), np.float32)
    f2[:, :12] = rng.normal(0, 1, (n, 12))
    wt = rng.normal(0, 1, 12)
    y2 = (0.3 + 0.9 / (1 + np.exp(-(f2[:, :12] @ wt) / 3))).astype(np.float32)
    P2 = torch.from_numpy(params(8)).to(dev)
    P2[mlp.OFF["mu"]:mlp.OFF["mu"] + 16] = 0
    P2[mlp.OFF["sigma"]:mlp.OFF["sigma"] + 16] = 1
    epochs = 40
    order = torch.stack([torch.from_numpy(rng.permutation(n).astype(np.int32))
                         for _ in range(epochs)]).to(dev)
    hist = nb.mlp_train(P2, torch.from_numpy(f2).to(dev), torch.from_numpy(y2).to(dev),
                        order, epochs=epochs, batch=256, lr=3e-3).cpu().numpy()
    assert hist[-1] < 0.1 * hist[0]
