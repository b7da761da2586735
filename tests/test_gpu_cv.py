"""Learned control variate on the GPU against the FP64 oracle: neighbour
features, union attributions, the control-variate volume estimator (fixed
and adaptive), the network's forward and backward kernels and its Adam
step; and what a trained network gains over the plain estimator."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import cv, synth

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def mols():
    ms = synth.generate(61, [1, 5, 12, 18, 33, 60, 64])
    return ms, shp.shape_set_load(ms)


def test_features_match_oracle(mols):
    ms, S = mols
    np.testing.assert_allclose(shp.cv_features(S).cpu().numpy(), O.cv_features(ms), rtol=2e-6, atol=2e-6)


def test_attributions_match_oracle(mols):
    ms, S = mols
    om = shp.union_attributions(S, seed=3, M=512, stream_base=5).cpu().numpy()
    ref = O.attributions(ms, np.arange(ms.n_mol), seed=3, M=512, stream_base=5)
    np.testing.assert_allclose(om, ref, rtol=RTOL, atol=1e-7)


@pytest.mark.parametrize("n", [1000, 4096])
def test_cv_volume_matches_oracle(mols, n):
    ms, S = mols
    rng = np.random.default_rng(n)
    omega = rng.uniform(0.0, 1.1, ms.n_atoms)
    idx = np.array([1, 2, 3, 6, 5, 4], np.int32)
    vol, se, nu = shp.union_volume_cv(S, idx, torch.tensor(omega, dtype=torch.float32), seed=8, n_samples=n,
                                      stream_base=2)
    ref_v, ref_s = O.union_volume_cv(ms, idx, omega.astype(np.float32).astype(np.float64), seed=8, n=n,
                                     stream_base=2)
    np.testing.assert_allclose(vol.cpu().numpy(), ref_v, rtol=RTOL)
    np.testing.assert_allclose(se.cpu().numpy(), ref_s, rtol=1e-4)
    assert np.all(nu.cpu().numpy() == n)
    # without weights it is the plain estimator on the same samples
    v0, s0, _ = shp.union_volume_cv(S, idx, None, seed=8, n_samples=n, stream_base=2)
    vp, sp, _, _ = shp.union_volume_estimate(S, idx, seed=8, n_samples=n, stream_base=2)
    np.testing.assert_allclose(v0.cpu().numpy(), vp.cpu().numpy(), rtol=2e-6)


def test_adaptive_cv_volume_stop_rule(mols):
    ms, S = mols
    idx = np.array([2, 3, 4, 5, 6], np.int32)
    # weights from the oracle's own attributions, fed to both sides
    omega = O.attributions(ms, np.arange(ms.n_mol), seed=1, M=256).astype(np.float32).astype(np.float64)
    om = torch.tensor(omega, dtype=torch.float32)
    target, rnd, cap = 3e-3, 256, 65536
    vol, se, nu = shp.union_volume_cv(S, idx, om, seed=4, n_samples=cap, target_rel_se=target, round=rnd)
    nu = nu.cpu().numpy().astype(np.int64)
    for k, n in enumerate(nu):
        assert n % rnd == 0 and rnd <= n <= cap
        v, s = O.union_volume_cv(ms, idx[k:k + 1], omega, seed=4, n=int(n), stream_base=k)
        assert vol.cpu().numpy()[k] == pytest.approx(v[0], rel=RTOL)
        if n < cap:
            assert s[0] <= target * v[0] * (1 + 1e-4)
        if n > rnd:
            v2, s2 = O.union_volume_cv(ms, idx[k:k + 1], omega, seed=4, n=int(n - rnd), stream_base=k)
            assert s2[0] > target * v2[0] * (1 - 1e-4)


def test_mlp_forward_and_gradients_match_oracle():
    rng = np.random.default_rng(9)
    p = M.init_params(5) + rng.normal(scale=0.05, size=M.N_PARAMS).astype(np.float32)
    X = rng.uniform(0, 2.5, (300, M.N_IN)).astype(np.float32)
    Tt = rng.uniform(0.2, 1.0, 300).astype(np.float32)
    rows = np.array(rng.permutation(300)[:257], np.int32)
    pt, Xt, Tg = (torch.tensor(a, device="cuda") for a in (p, X, Tt))
    y = shp.mlp_forward(pt, Xt).cpu().numpy()
    np.testing.assert_allclose(y, M.forward(p, X), rtol=2e-5, atol=2e-6)
    loss, grad = shp.mlp_loss_grad(pt, Xt, Tg, torch.tensor(rows, device="cuda"))
    L, g = M.loss_and_grad(p, X[rows], Tt[rows])
    assert float(loss.item()) == pytest.approx(L, rel=1e-5)
    g_gpu = grad.cpu().numpy()
    assert np.linalg.norm(g_gpu - g) <= 1e-4 * np.linalg.norm(g)


def test_train_epoch_equals_step_by_step_calls():
    """mlp_train_epoch runs an epoch's minibatches (the last one shorter)
    inside the library: the same parameters, moments and per-minibatch losses
    as mlp_loss_grad then mlp_adam called per minibatch, bit for bit."""
    rng = np.random.default_rng(4)
    X = torch.tensor(rng.uniform(0, 2.5, (3000, M.N_IN)), dtype=torch.float32, device="cuda")
    t = torch.tensor(rng.uniform(0.2, 1.0, 3000), dtype=torch.float32, device="cuda")
    perm = torch.tensor(rng.permutation(3000)[:2900], dtype=torch.int32, device="cuda")
    p0 = cv.init_params(3)
    a = [p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)]
    b = [p0.clone(), torch.zeros_like(p0), torch.zeros_like(p0)]
    losses = shp.mlp_train_epoch(a[0], a[1], a[2], X, t, perm, 512, 5, 3e-3).cpu().numpy()
    ref = []
    for k, s0 in enumerate(range(0, 2900, 512)):
        loss, grad = shp.mlp_loss_grad(b[0], X, t, perm[s0:s0 + 512])
        shp.mlp_adam(b[0], b[1], b[2], grad, 5 + k + 1, 3e-3)
        ref.append(loss.item())
    for u, w in zip(a, b):
        assert torch.equal(u, w)
    np.testing.assert_array_equal(losses, np.array(ref))


def test_adam_step():
    rng = np.random.default_rng(2)
    p = rng.normal(size=100).astype(np.float32)
    g = rng.normal(size=100).astype(np.float32)
    m = rng.normal(scale=0.1, size=100).astype(np.float32)
    v = rng.uniform(0.01, 0.1, size=100).astype(np.float32)
    pt, gt, mt, vt = (torch.tensor(a, device="cuda") for a in (p, g, m, v))
    shp.mlp_adam(pt, mt, vt, gt, step=3, lr=1e-2)
    m1 = 0.9 * m + 0.1 * g
    v1 = 0.999 * v + 0.001 * g * g
    p1 = p - 1e-2 * (m1 / (1 - 0.9 ** 3)) / (np.sqrt(v1 / (1 - 0.999 ** 3)) + 1e-8)
    np.testing.assert_allclose(pt.cpu().numpy(), p1, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(mt.cpu().numpy(), m1, rtol=1e-6, atol=1e-7)


def test_trained_network_reduces_variance():
    """Trained on attributions of 3000 molecules, the network's weights cut
    the union-volume SE on 400 held-out molecules (same samples), and the
    control-variate estimates stay unbiased against the plain ones."""
    train = synth.generate(71, synth.counts_uniform(71, 3000, 18, 60))
    held = synth.generate(72, synth.counts_uniform(72, 400, 18, 60))
    St, Sh = shp.shape_set_load(train), shp.shape_set_load(held)
    feats, targets = cv.attributions_and_features(St, seed=1, M=512)
    net = cv.CrowdingNet(seed=0)
    hist = net.fit(feats, targets, epochs=30, batch=8192, lr=3e-3)
    assert hist[-1] < 0.5 * hist[0]
    om = net.predict(shp.cv_features(Sh))
    v_cv, s_cv, _ = shp.union_volume_cv(Sh, None, om, seed=3, n_samples=8192)
    v_pl, s_pl, _ = shp.union_volume_cv(Sh, None, None, seed=3, n_samples=8192)
    ratio = (s_cv / s_pl).cpu().numpy()
    assert np.median(ratio) < 0.9
    z = ((v_cv - v_pl) / torch.sqrt(s_cv ** 2 + s_pl ** 2)).cpu().numpy()
    assert abs(z.mean()) < 0.2


def test_least_squares_weights_match_oracle():
    """The projection weights of the screen's control variate: GPU (FP32
    sums, conjugate gradients) against the oracle (FP64, Cholesky) on the same
    samples; a list of molecules writes only their atoms."""
    ms = synth.principal_axes(synth.generate(91, [12, 25, 40, 60, 18, 1]))
    S = shp.shape_set_load(ms)
    w = shp.cv_fit_weights(S, seed=4, n_samples=1024, stream_base=7).cpu().numpy()
    ref = O.cv_fit_weights(ms, np.arange(ms.n_mol), seed=4, n=1024, stream_base=7)
    np.testing.assert_allclose(w, ref, rtol=1e-4, atol=2e-4 * np.abs(ref).max())
    pick = np.array([3, 0], np.int32)
    wp = shp.cv_fit_weights(S, seed=5, n_samples=512, idx=pick).cpu().numpy()
    rp = O.cv_fit_weights(ms, pick, seed=5, n=512)
    listed = np.zeros(ms.n_atoms, bool)
    for k in pick:
        listed[ms.offsets[k]:ms.offsets[k + 1]] = True
    np.testing.assert_allclose(wp[listed], rp[listed], rtol=1e-4, atol=2e-4 * np.abs(rp).max())
    assert np.all(wp[~listed] == 0.0)
    with pytest.raises(shp.ShapeError):
        shp.cv_fit_weights(S, seed=1, n_samples=1000)  # not a multiple of 256
