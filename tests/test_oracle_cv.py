"""Pins for the oracle's learned-control-variate pieces: union attributions
(their weighted sum is the union volume), the control-variate volume
estimator (unbiased for any weights, identical to the plain estimator at
zero weights, lower variance at the attributions), the neighbour features,
and the reference MLP's autograd graph."""
import numpy as np
import pytest
import torch

import oracle as O
from oracle import mlp as M
from paper_2607_20766_b300 import synth
from paper_2607_20766_b300.synth import MolSet


@pytest.fixture(scope="module")
def mols():
    return synth.generate(77, [12, 15, 9])


def test_attributions_sum_to_the_union_volume(mols):
    """V = Z E_q[u/m] = sum_i v_i E_{N_i}[u/m] (q is the v-weighted mixture)."""
    om = O.attributions(mols, [0, 1, 2], seed=1, M=8192)
    for i in range(3):
        v = O.mol_tables(mols, i)["v"]
        lo, hi = mols.offsets[i], mols.offsets[i + 1]
        V = O.union_volume_ie(mols, i)
        assert np.dot(om[lo:hi], v) == pytest.approx(V, rel=5e-3)


def test_attribution_of_an_isolated_atom_is_one():
    ms = MolSet(np.array([[0, 0, 0], [40, 0, 0]], np.float32), np.array([1.7, 1.5], np.float32),
                np.array([0, 2], np.int32), np.zeros(2, np.uint8))
    om = O.attributions(ms, [0], seed=3, M=512)
    np.testing.assert_allclose(om, 1.0, atol=1e-12)


def test_control_variate_unbiased_for_any_weights(mols):
    V = O.union_volume_ie(mols, 1)
    rng = np.random.default_rng(0)
    for omega in (np.zeros(mols.n_atoms), rng.uniform(0, 1.2, mols.n_atoms),
                  O.attributions(mols, [0, 1, 2], seed=2, M=2048)):
        idx = np.ones(12, np.int32)
        v, se = O.union_volume_cv(mols, idx, omega, seed=5, n=4096)
        z = (v - V) / se
        assert np.sum(np.abs(z) > 3) <= 1, z


def test_zero_weights_reproduce_the_plain_estimator(mols):
    v0, s0 = O.union_volume_cv(mols, [0, 1, 2], np.zeros(mols.n_atoms), seed=7, n=2000, stream_base=3)
    vp, sp, _, _ = O.union_volume_estimate(mols, [0, 1, 2], seed=7, n=2000, stream_base=3)
    np.testing.assert_allclose(v0, vp, rtol=1e-12)
    np.testing.assert_allclose(s0, sp, rtol=1e-9)


def test_attribution_weights_reduce_variance(mols):
    om = O.attributions(mols, [0, 1, 2], seed=2, M=4096)
    v0, s0 = O.union_volume_cv(mols, [0, 1, 2], np.zeros(mols.n_atoms), seed=9, n=8192)
    v1, s1 = O.union_volume_cv(mols, [0, 1, 2], om, seed=9, n=8192)
    assert np.all(s1 < 0.95 * s0)


def test_features_rigid_invariant_and_sorted(mols):
    f = O.cv_features(mols)
    assert f.shape == (mols.n_atoms, 33)
    d = f[:, 0:32:2]
    assert np.all(np.diff(d[:, :8], axis=1) >= 0)       # the 9-atom molecule pads after 8 neighbours
    np.testing.assert_allclose(f[:, 32], mols.radius / 1.7, rtol=1e-7)
    lo = mols.offsets[2]
    assert np.all(f[lo:, 16:32:2] == 2.5) and np.all(f[lo:, 17:32:2] == 0.0)
    R = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))[0]
    moved = MolSet((mols.xyz.astype(np.float64) @ R.T + 3.0).astype(np.float32), mols.radius, mols.offsets,
                   mols.elem)
    np.testing.assert_allclose(O.cv_features(moved), f, atol=3e-6)
    # nearest neighbour of a bonded atom is at a bond length (1.40 - 1.55 A)
    assert np.all((d[:, 0] * 4 > 1.39) & (d[:, 0] * 4 < 1.56))


def test_reference_mlp_gradients():
    p = M.init_params(3)
    rng = np.random.default_rng(4)
    X = rng.uniform(0, 2.5, (7, M.N_IN))
    T = rng.uniform(0.2, 1.0, 7)
    p64 = M.bf16_round(p).clone().requires_grad_(True)
    Xt, Tt = torch.tensor(X), torch.tensor(T)

    def loss(q):
        W1, b1, W2, b2, w3, b3 = M.unpack(q)
        h1 = torch.nn.functional.gelu(Xt @ W1.T + b1)
        h2 = torch.nn.functional.gelu(h1 @ W2.T + b2)
        return (((h2 @ w3 + b3) - Tt) ** 2).mean()

    assert torch.autograd.gradcheck(loss, (p64,), eps=1e-6, atol=1e-7)
    L, g = M.loss_and_grad(p, X, T)
    assert L == pytest.approx(float(loss(p64)), rel=1e-12)
    # a network with zero hidden weights outputs w3 . gelu(b2) + b3
    q = np.zeros(M.N_PARAMS, np.float32)
    q[-1] = 0.25
    q[-1 - M.N_HID:-1] = 0.5
    q[M.N_HID * M.N_IN + M.N_HID + M.N_HID * M.N_HID:][:M.N_HID] = 1.0  # b2 = 1
    gelu1 = 0.5 * (1 + torch.erf(torch.tensor(1.0, dtype=torch.float64) / np.sqrt(2.0))).item()
    np.testing.assert_allclose(M.forward(q, X), 0.25 + 0.5 * M.N_HID * gelu1, rtol=1e-12)


# ------------------------------------------------ control variate in the screen


def _screen(q, d, seed, n, omega_q=None, omega_d=None, stream_base=0):
    kq, kd = np.arange(q.n_mol), np.arange(d.n_mol)
    sq = np.stack([O.fo_overlap(q, kq, q, kq), np.full(q.n_mol, 1e3)], 1)
    sd = np.stack([O.fo_overlap(d, kd, d, kd), np.full(d.n_mol, 1e3)], 1)
    iq, idd = np.repeat(kq, d.n_mol), np.tile(kd, q.n_mol)
    st = (stream_base + np.arange(len(iq))).astype(np.uint64)
    return O.tanimoto_pairs(q, iq, d, idd, st, sq, sd, seed=seed, n=n, omega_q=omega_q, omega_d=omega_d)


@pytest.fixture(scope="module")
def pair_sets():
    q = synth.principal_axes(synth.generate(31, [12, 9]))
    d = synth.principal_axes(synth.generate(32, [11, 12]))
    return q, d


def test_screen_cv_zero_weights_reproduce_the_plain_estimator(pair_sets):
    q, d = pair_sets
    pl = _screen(q, d, seed=3, n=1000)
    cv = _screen(q, d, seed=3, n=1000, omega_q=np.zeros(q.n_atoms), omega_d=np.zeros(d.n_atoms))
    np.testing.assert_allclose(cv["O"], pl["O"], rtol=1e-12)
    np.testing.assert_allclose(cv["seO"], pl["seO"], rtol=1e-9)


def test_screen_cv_single_atoms_are_exact():
    """One atom per molecule and unit weights: u = g = u~, so every residual is
    zero up to rounding and the union slot is the closed form, i.e. the
    first-order overlap of the two Gaussians."""
    a = MolSet(np.array([[0, 0, 0]], np.float32), np.array([1.7], np.float32), np.array([0, 1], np.int32),
               np.zeros(1, np.uint8))
    b = MolSet(np.array([[1.3, 0.4, -0.2]], np.float32), np.array([1.52], np.float32), np.array([0, 1], np.int32),
               np.zeros(1, np.uint8))
    cv = _screen(a, b, seed=4, n=512, omega_q=np.ones(1), omega_d=np.ones(1))
    fo = O.fo_overlap(a, [0], b, [0])[0]
    assert cv["O"][0, 1] == pytest.approx(fo, rel=1e-12)
    assert cv["seO"][0, 1] < 1e-12 * fo
    pl = _screen(a, b, seed=4, n=512)
    assert abs(pl["O"][0, 1] - fo) < 4 * pl["seO"][0, 1] and pl["seO"][0, 1] > 1e-6 * fo


def test_screen_cv_unbiased_against_inclusion_exclusion(pair_sets):
    """Any weights: the CV union overlap stays within a few SE of the exact
    inclusion-exclusion value (molecules of 9-12 atoms)."""
    q, d = pair_sets
    rng = np.random.default_rng(5)
    exact = np.array([[O.union_overlap_ie(q, i, d, j) for j in range(d.n_mol)] for i in range(q.n_mol)]).reshape(-1)
    for k, (wq, wd) in enumerate([(rng.uniform(0, 1.2, q.n_atoms), rng.uniform(0, 1.2, d.n_atoms)),
                                  (O.attributions(q, [0, 1], seed=6, M=1024),
                                   O.attributions(d, [0, 1], seed=7, M=1024))]):
        for seed in (11, 12, 13):
            cv = _screen(q, d, seed=seed + 10 * k, n=4096, omega_q=wq, omega_d=wd)
            z = (cv["O"][:, 1] - exact) / cv["seO"][:, 1]
            assert np.all(np.abs(z) < 4.5), z


def test_screen_cv_attributions_reduce_variance_on_drug_size_molecules():
    """With the union attributions as weights the residual's variance is lower
    on average for drug-size molecules (20-50 atoms; sparse molecules of ~10
    atoms can see a small increase, which the adaptive screen then pays for)."""
    q = synth.principal_axes(synth.generate(21, [20, 32, 12]))
    d = synth.principal_axes(synth.generate(22, [12, 39, 50, 25]))
    wq = O.attributions(q, np.arange(q.n_mol), seed=3, M=2048)
    wd = O.attributions(d, np.arange(d.n_mol), seed=4, M=2048)
    pl = _screen(q, d, seed=5, n=4096)
    cv = _screen(q, d, seed=5, n=4096, omega_q=wq, omega_d=wd)
    ratio = (cv["seO"][:, 1] / pl["seO"][:, 1]) ** 2
    assert ratio.mean() < 0.85, ratio
    np.testing.assert_array_equal(cv["O"][:, 0], pl["O"][:, 0])  # first-order slot untouched


# ------------------------------------------------ least-squares weights


def _gauss_product_integral(ps, alphas, centres):
    """Integral over R^3 of prod_k p_k exp(-alpha_k |r - c_k|^2) (Gaussian
    product theorem)."""
    A = sum(alphas)
    s = sum(a * c for a, c in zip(alphas, centres))
    q = sum(a * float(c @ c) for a, c in zip(alphas, centres)) - float(s @ s) / A
    return float(np.prod(ps)) * (np.pi / A) ** 1.5 * np.exp(-q)


def test_least_squares_weights_two_atoms_closed_form():
    """Two overlapping atoms: u = g1 + g2 - g1 g2, so every integral of the
    projection has a closed form; the sampled fit matches it."""
    c = np.array([[0.0, 0.0, 0.0], [1.3, 0.4, -0.2]])
    R = np.array([1.7, 1.52])
    ms = MolSet(c.astype(np.float32), R.astype(np.float32), np.array([0, 2], np.int32), np.zeros(2, np.uint8))
    c = ms.xyz.astype(np.float64)
    a = 2.41798793 / ms.radius.astype(np.float64) ** 2
    p = 2.0 * np.sqrt(2.0)

    def I(*ks):  # integral of the product of the listed Gaussians (indices may repeat)
        return _gauss_product_integral([p] * len(ks), [a[k] for k in ks], [c[k] for k in ks])

    G = np.array([[I(0, 0), I(0, 1)], [I(1, 0), I(1, 1)]])
    b = np.array([I(i, 0) + I(i, 1) - I(i, 0, 1) for i in range(2)])  # integral of u g_i
    exact = np.linalg.solve(G, b)
    fits = np.array([O.cv_fit_weights(ms, [0], seed=s, n=1 << 18, ridge=0.0) for s in range(8)])
    se = fits.std(0, ddof=1) / np.sqrt(len(fits))
    assert np.all(np.abs(fits.mean(0) - exact) < 4 * se), (fits.mean(0), exact, se)
    assert np.all(se < 2e-3 * exact)


def test_least_squares_weights_of_isolated_atoms_are_one():
    ms = MolSet(np.array([[0, 0, 0], [30, 0, 0], [0, 30, 0]], np.float32), np.array([1.7, 1.55, 1.52], np.float32),
                np.array([0, 3], np.int32), np.zeros(3, np.uint8))
    np.testing.assert_allclose(O.cv_fit_weights(ms, [0], seed=1, n=1 << 16), 1.0, atol=2e-2)


def test_least_squares_weights_beat_attributions_in_the_screen():
    """The projection weights lower the screen's union variance further than
    the volume attributions do (drug-size molecules)."""
    q = synth.principal_axes(synth.generate(21, [20, 32, 12]))
    d = synth.principal_axes(synth.generate(22, [12, 39, 50, 25]))
    aq = O.attributions(q, np.arange(q.n_mol), seed=3, M=2048)
    ad = O.attributions(d, np.arange(d.n_mol), seed=4, M=2048)
    lq = O.cv_fit_weights(q, np.arange(q.n_mol), seed=5, n=4096)
    ld = O.cv_fit_weights(d, np.arange(d.n_mol), seed=6, n=4096, stream_base=10)
    pl = _screen(q, d, seed=7, n=4096)
    ca = _screen(q, d, seed=7, n=4096, omega_q=aq, omega_d=ad)
    cl = _screen(q, d, seed=7, n=4096, omega_q=lq, omega_d=ld)
    ra = (ca["seO"][:, 1] / pl["seO"][:, 1]) ** 2
    rl = (cl["seO"][:, 1] / pl["seO"][:, 1]) ** 2
    assert rl.mean() < 0.55 and rl.mean() < 0.75 * ra.mean(), (rl, ra)
