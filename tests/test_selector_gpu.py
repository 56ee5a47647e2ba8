"""The learned selector: its MLP kernels against the fp64 oracle (forward,
soft targets, gradients, Adam), its features against closed forms and the
oracle, a training run that learns a rule it can be scored on, and labels
that never depend on the choice."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
import paper_2008_03909_gb300 as cc
from paper_2008_03909_gb300 import selector
import synth

pytestmark = pytest.mark.gpu


def _params(seed):
    p = torch.empty(cc.MLP_NPARAM, dtype=torch.float32, device="cuda")
    cc.mlp_init(p, seed)
    rng = np.random.default_rng(seed)
    h = p.cpu().numpy().astype(np.float64)
    h[:16] = rng.normal(0, 1, 16)
    h[16:32] = rng.uniform(0.5, 2.0, 16)
    return torch.from_numpy(h.astype(np.float32)).cuda()


def test_mlp_kernels_match_oracle():
    rng = np.random.default_rng(7)
    B = 257
    p = _params(3)
    X = torch.from_numpy(rng.normal(0, 1.5, (B, 16)).astype(np.float32)).cuda()
    T = torch.from_numpy(rng.uniform(1, 4, (B, 12)).astype(np.float32)).cuda()
    Q = torch.empty(B, 12, device="cuda")
    cc.mlp_soft_targets(T, 0.2, Q)
    qo = omlp.soft_targets(T.cpu().numpy(), 0.2)
    assert np.allclose(Q.cpu().numpy(), qo, rtol=1e-5, atol=1e-6)
    logits = torch.empty(B, 12, device="cuda")
    acts = torch.empty(B, 128, device="cuda")
    cc.mlp_forward(p, X, logits, acts)
    po = p.cpu().numpy().astype(np.float64)
    zo, _ = omlp.forward(po, X.cpu().numpy())
    # fp32 sums of <= 64 products of O(1) terms: relative error ~1e-6
    assert np.allclose(logits.cpu().numpy(), zo, rtol=1e-4, atol=1e-4)
    grads = torch.empty(cc.MLP_NPARAM, device="cuda")
    loss = torch.empty(1, device="cuda")
    cc.mlp_backward(p, X, acts, logits, Q, grads, loss)
    go, lo = omlp.backward(po, X.cpu().numpy(), qo)
    g = grads.cpu().numpy()
    scale = np.abs(go).max()
    assert np.allclose(g, go, rtol=1e-3, atol=1e-5 * scale)
    assert abs(float(loss.item()) - lo) < 1e-4 * max(1.0, lo)
    # deterministic: the same step twice gives the same bits
    g2 = torch.empty_like(grads)
    cc.mlp_backward(p, X, acts, logits, Q, g2)
    assert torch.equal(grads, g2)
    m = torch.zeros_like(grads)
    v = torch.zeros_like(grads)
    p2 = p.clone()
    cc.mlp_adam(p2, grads, m, v, 1, 0.01)
    po2, _, _ = omlp.adam(po, g.astype(np.float64), np.zeros_like(po), np.zeros_like(po), 1, 0.01)
    assert np.allclose(p2.cpu().numpy(), po2, rtol=1e-5, atol=1e-6)


def test_training_learns_a_rule():
    """Times follow a known rule of the features; the trained network picks
    the fastest class on held-out samples far better than a fixed choice."""
    rng = np.random.default_rng(11)
    N, Nt = 600, 300
    X = rng.normal(0, 1, (N + Nt, 16)).astype(np.float32)
    best = (np.argmax(X[:, :4] @ rng.normal(0, 1, (4, 12)), axis=1)).astype(np.int64)
    T = np.ones((N + Nt, 12), np.float32) * 2.0
    T[np.arange(N + Nt), best] = 1.0
    sel = selector.Selector(seed=5)
    hist = sel.fit(torch.from_numpy(X[:N]).cuda(), torch.from_numpy(T[:N]).cuda(), epochs=600, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    pred = sel.predict(torch.from_numpy(X[N:]).cuda()).cpu().numpy()
    acc = (pred == best[N:]).mean()
    assert acc > 0.8, acc
    r_sel = selector.regret(torch.from_numpy(T[N:]), torch.from_numpy(pred)).mean()
    r_fix = selector.regret(torch.from_numpy(T[N:]), torch.full((Nt,), selector.DEFAULT)).mean()
    assert r_sel < 0.3 * r_fix


def test_features_closed_form_path():
    # path 0 - 1 - ... - (n-1): two vertices of degree 1, the rest degree 2;
    # k-out joins everything into the cluster of vertex 0, nothing is left
    # for the finish
    n = 1000
    g = synth.path(n)
    f = cc.cc_features(g.offsets.cuda(), g.edges.cuda()).cpu().numpy()
    assert abs(f[0] - np.log2(n + 1)) < 1e-5 and abs(f[1] - np.log2(2 * (n - 1) + 1)) < 1e-5
    assert abs(f[2] - 2 * (n - 1) / n) < 1e-6 and abs(f[3] - np.log2(3)) < 1e-6
    assert f[5] == 0 and abs(f[6] - 2 / n) < 1e-7 and abs(f[7] - (n - 2) / n) < 1e-6
    assert f[11] == 1.0 and abs(f[12] - (n - 1) / n) < 1e-6 and f[13] == 0.0 and f[14] == 0.0
    assert f[15] >= 0.0


def _check_features(g, seed):
    off, edg = g.numpy()
    f = cc.cc_features(g.offsets.cuda(), g.edges.cuda(), seed=seed).cpu().numpy()
    deg = np.diff(off).astype(np.float64)
    n, m = g.n, max(1.0, deg.sum())
    assert abs(f[2] - deg.mean()) < 1e-4 * max(deg.mean(), 1e-9)
    if deg.mean() > 0:
        assert abs(f[4] - deg.var() / deg.mean() ** 2) < 1e-3 * max(deg.var() / deg.mean() ** 2, 1e-9)
    assert abs(f[3] - np.log2(deg.max() + 1)) < 1e-5
    assert abs(f[5] - (deg == 0).mean()) < 1e-6 and abs(f[9] - (deg > 64).mean()) < 1e-6
    assert abs(f[10] - deg[deg > 64].sum() / m) < 1e-5
    # from the k-out sample (the oracle's, same seed) and its IdentifyFrequent
    lab = oracle.kout_sample(off, edg, 2, seed)
    lm, cnt = oracle.identify_frequent(lab)
    out = lab != lm
    assert abs(f[11] - cnt / n) < 1e-6
    assert abs(f[12] - (lab != np.arange(n)).mean()) < 1e-6
    assert abs(f[13] - deg[out].sum() / m) < 1e-6
    assert abs(f[14] - (out & (deg > 0) & (deg <= 32)).mean()) < 1e-6
    return f


def test_features_match_numpy_and_oracle():
    f1 = _check_features(synth.rmat(16, 8, seed=4), 9)
    f2 = _check_features(synth.grid2d(200, 150, 0.2, seed=3), 2)
    _check_features(synth.erdos_renyi(40000, 1.5, seed=5), 4)
    _check_features(synth.cliques([7, 30, 2, 64, 5] * 20), 1)
    # the depth stand-in separates a power-law graph from a grid
    assert f2[15] > f1[15]


def test_selected_path_every_class_exact():
    """Every class the selected path can run (forced) gives the oracle's
    labels and reports the class it ran."""
    for i, g in enumerate((synth.rmat(13, 8, seed=2), synth.grid2d(90, 80, 0.3, seed=1),
                           synth.erdos_renyi(20000, 1.2, seed=3), synth.path(3000))):
        want, _ = oracle.cc_uf(*g.numpy())
        off, edg = g.offsets.cuda(), g.edges.cuda()
        for c in range(12):
            lab, ran = cc.cc_select_static(off, edg, None, c)
            assert ran == c
            assert np.array_equal(lab.cpu().numpy().view(np.uint32), want), (i, c)
    assert cc.device_error() == 0


def test_selected_path_features_equal_cc_features():
    g = synth.rmat(14, 8, seed=6)
    off, edg = g.offsets.cuda(), g.edges.cuda()
    feat = torch.empty(16, device="cuda")
    sel = selector.Selector(seed=4)
    lab, c = cc.cc_select_static(off, edg, sel.params, -1, feat_out=feat)
    assert torch.equal(feat, cc.cc_features(off, edg))
    # the class the network picks in the path is the one cc_mlp_predict picks
    assert c == int(sel.predict(feat).item())


def test_selector_never_changes_labels():
    for seed in (2, 3, 4):
        sel = selector.Selector(seed=seed)
        for i in range(8):
            g = synth.selector_graph(i, seed=3, scale_lo=10, scale_hi=13)
            want, _ = oracle.cc_uf(*g.numpy())
            lab, c = sel.run(g.offsets.cuda(), g.edges.cuda())
            assert 0 <= c < 12
            assert np.array_equal(lab.cpu().numpy().view(np.uint32), want)
