"""The learned per-group opening angle on the GPU: probe features against
the oracle's, per-group theta walks bit-exact against the oracle, network
inference against the BF16-emulated oracle on the oracle's features, and an
end-to-end train/evaluate run showing what the network saves at equal
median error."""
import numpy as np
import pytest

import nbsynth
from oracle import features as ofeat
from oracle import mlp

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def setup(n=40000, seed=61, n_halos=60):
    import paper_0909_0541_gb300 as nb
    ps = nbsynth.halo_mix(n, seed, n_halos=n_halos)
    dev = torch.device("cuda")
    pos = torch.from_numpy(ps.pos).to(dev)
    mass = torch.from_numpy(ps.mass).to(dev)
    ctx = nb.NBody(ps.n, eps=5e-4, n_crit=64)
    ctx.build_tree(pos, mass)
    return nb, ps, pos, mass, ctx


def test_probe_features_match_oracle(oracle_lib):
    nb, ps, pos, mass, ctx = setup()
    feat = ctx.group_features(64).cpu().numpy()
    T = oracle_lib.Tree(ps.pos, ps.mass)
    sel = np.random.default_rng(3).choice(feat.shape[0], 200, replace=False)
    ref = ofeat.group_features(T, 64, sel)
    assert feat.shape[0] == len(T.groups(64))
    assert np.all(feat[:, 12:] == 0)
    assert np.allclose(feat[sel, :12], ref, rtol=0, atol=2e-5)


def test_tree_features_match_oracle(oracle_lib):
    """Feature mode 1: the features that need no walk, for every group,
    against the oracle's tree_features; the walk-based slots are zero."""
    nb, ps, pos, mass, ctx = setup()
    ctx.set_feature_mode(1)
    feat = ctx.group_features(64).cpu().numpy()
    T = oracle_lib.Tree(ps.pos, ps.mass)
    ref = ofeat.tree_features(T, 64)
    assert feat.shape[0] == ref.shape[0]
    assert np.all(feat[:, 6:11] == 0) and np.all(feat[:, 12:] == 0)
    assert np.allclose(feat[:, :12], ref, rtol=0, atol=2e-5)


def test_per_group_theta_lists_bit_exact(oracle_lib):
    nb, ps, pos, mass, ctx = setup(20000, 62, 30)
    T = oracle_lib.Tree(ps.pos, ps.mass)
    G = len(T.groups(64))
    th = np.random.default_rng(4).uniform(0.3, 1.2, G).astype(np.float32)
    ctx.walk_groups(0.6, 64, torch.from_numpy(th).cuda())
    gg = ctx.copy_groups()
    assert np.array_equal(gg["invtheta"], (1.0 / th.astype(np.float64)).astype(np.float32))
    e = T.export()
    leaf_of_slot = np.flatnonzero(e["is_cell"] == 0)
    gnode = T.groups(64)
    box = T.group_boxes(gnode)
    for k in np.random.default_rng(5).choice(G, 60, replace=False):
        ref = T.walk_group(gnode[k], box[k], float(th[k]))
        f, c = e["first"][gnode[k]], e["count"][gnode[k]]
        ref = ref[~np.isin(ref, leaf_of_slot[f:f + c])]
        ids, _ = ctx.copy_list(k)
        assert np.array_equal(np.sort(ids), ref)
    # forces with per-group theta against the oracle's per-group-theta sums
    acc = torch.empty((ps.n, 3), dtype=torch.float32, device="cuda")
    ctx.forces(5e-4, acc)
    a32, _, _, _, am = T.forces(64, 0.6, 5e-4, theta_g=th, with_amag=True, coords32=True)
    d = np.linalg.norm(acc.cpu().numpy().astype(np.float64) - a32, axis=1)
    assert np.all(d <= 1e-5 * am)


def test_inference_matches_oracle_on_oracle_features(oracle_lib):
    nb, ps, pos, mass, ctx = setup()
    T = oracle_lib.Tree(ps.pos, ps.mass)
    G = len(T.groups(64))
    sel = np.random.default_rng(6).choice(G, 100, replace=False)
    fo = ofeat.group_features(T, 64, sel)
    w = nbsynth.mlp_initial_weights(11)
    p = mlp.pack_params(w["W1"], w["b1"], w["W2"], w["b2"], w["W3"], w["b3"], w["w4"], 0.0,
                        fo.mean(0), fo.std(0) + 1e-3)
    P = torch.from_numpy(p).cuda()
    theta = torch.zeros(ps.n, dtype=torch.float32, device="cuda")
    ctx.walk_groups_learned(64, P, 0.6, theta)
    th_gpu = theta.cpu().numpy()[sel]
    th_or, _ = mlp.forward(p, fo, bf=True)
    assert np.max(np.abs(th_gpu - th_or)) < 5e-3
    assert np.all((th_gpu >= 0.3) & (th_gpu <= 1.2))


@pytest.mark.slow
def test_train_and_gain_at_equal_error():
    """Train on one halo mix, evaluate on another: report the network's
    interactions against the fixed theta with the same median error.  On
    these clustered sets the per-group allocation does not beat one fixed
    theta (measured within a few per cent either way), so the test bounds
    the learned form's cost and error rather than asserting a gain."""
    import paper_0909_0541_gb300 as nb
    from paper_0909_0541_gb300 import learn
    dev = torch.device("cuda")
    tr = nbsynth.halo_mix(300000, 71, n_halos=300)
    X, y, info = learn.make_dataset(torch.from_numpy(tr.pos).to(dev),
                                    torch.from_numpy(tr.mass).to(dev), 5e-4, 64, 10 ** 9, 1)
    assert float(y.min()) >= np.float32(0.3) and float(y.max()) <= np.float32(1.2)
    assert abs(info["labelled_error"] - 1e-3) < 2e-4
    params, hist = learn.train(X, y, epochs=120, batch=256, lr=2e-3)
    assert hist[-1] < hist[0]
    ev = nbsynth.halo_mix(300000, 72, n_halos=300)
    pos = torch.from_numpy(ev.pos).to(dev)
    mass = torch.from_numpy(ev.mass).to(dev)
    ctx = nb.NBody(ev.n, eps=5e-4, n_crit=64)
    ctx.build_tree(pos, mass)
    tg = torch.from_numpy(np.random.default_rng(8).choice(ev.n, 2048, replace=False)).to(dev)
    ref, _ = nb.direct_sum(pos, mass, 5e-4, tg)
    acc = torch.empty((ev.n, 3), dtype=torch.float32, device=dev)
    inter_l, _ = learn.step_cost(ctx, 64, 5e-4, acc, params=params)
    err_l = learn.median_error(acc, ref, tg)
    th = learn.matched_fixed_theta(ctx, 64, 5e-4, acc, ref, tg, err_l)
    inter_f, _ = learn.step_cost(ctx, 64, 5e-4, acc, theta=th)
    err_f = learn.median_error(acc, ref, tg)
    gain = 1.0 - inter_l / inter_f
    print(f"learned: err {err_l:.3e} interactions {inter_l}; fixed theta {th:.3f}: "
          f"err {err_f:.3e} interactions {inter_f}; gain {gain:+.3f}")
    assert err_l < 2.5e-3
    assert abs(err_f - err_l) < 0.1 * err_l
    assert gain > -0.15
    # a non-finite network output falls back to the fixed theta
    bad = params.clone()
    bad[9920] = float("nan")
    theta = torch.zeros(ev.n, dtype=torch.float32, device=dev)
    ctx.walk_groups_learned(64, bad, 0.6, theta)
    G = ctx.stats()["n_groups"]
    assert torch.all(theta[:G] == np.float32(0.6))
    ctx.close()
