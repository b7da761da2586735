"""Pins for the full delta-method SE of the Tanimoto and for the
control-variate self-overlap estimator.

The paper's SE(T) (Sec. confidence-bounded screening) propagates only the
pair overlap's sampling error and treats the self-overlaps O_QQ, O_DD as
exact. When the union self-overlaps are themselves importance-sampled, their
error reaches T too; the oracle's full SE adds
(O / (S - O)^2)^2 (se_QQ^2 + se_DD^2). These tests pin that formula to what
it claims to describe -- the spread of T over independent replicates -- and
pin the self-overlap control variate to the exact inclusion-exclusion value
and to the Gaussian-product closed form."""
import numpy as np
import pytest

import oracle as O
from paper_2607_20766_b300 import synth
from paper_2607_20766_b300.synth import MolSet


def _copies(ms: MolSet, k: int) -> MolSet:
    """k copies of a one-molecule set (each copy gets its own streams)."""
    n = ms.n_atoms
    return MolSet(np.tile(ms.xyz, (k, 1)), np.tile(ms.radius, k), np.arange(k + 1, dtype=np.int32) * n,
                  np.tile(ms.elem, k))


@pytest.fixture(scope="module")
def small_pair():
    # A 8 atoms, B 10 atoms, centroids 0.8 A apart: union T around 0.3-0.5
    return synth.single_pair(n_a=8, n_b=10, seed_a=3, seed_b=4, separation=0.8)


def _replicates(a, b, K, n_self, n_pair):
    qa, db = _copies(a, K), _copies(b, K)
    idx = np.arange(K, dtype=np.int32)
    # fresh self-overlap streams per replicate (tag 2), fresh pair streams (tags 0/1)
    _, _, sq, sq_se = O.union_volume_estimate(qa, idx, seed=101, n=n_self, stream_base=0)
    _, _, sd, sd_se = O.union_volume_estimate(db, idx, seed=101, n=n_self, stream_base=10 * K)
    fo_q = O.fo_overlap(qa, idx, qa, idx)
    fo_d = O.fo_overlap(db, idx, db, idx)
    selfQ, selfD = np.stack([fo_q, sq], 1), np.stack([fo_d, sd], 1)
    seQ = np.stack([np.zeros(K), sq_se], 1)
    seD = np.stack([np.zeros(K), sd_se], 1)
    full = O.tanimoto_pairs(qa, idx, db, idx, idx.astype(np.uint64) + 77, selfQ, selfD, seed=202, n=n_pair,
                            selfQ_se=seQ, selfD_se=seD)
    pair_only = O.tanimoto_pairs(qa, idx, db, idx, idx.astype(np.uint64) + 77, selfQ, selfD, seed=202, n=n_pair)
    return full, pair_only


def test_full_delta_se_matches_the_spread_of_T_over_replicates(small_pair):
    """With noisy self-overlaps (256 samples each) the spread of the union T
    over 400 independent replicates is what the full delta-method SE
    predicts, and several times what the pair-only SE of the paper's formula
    predicts. A wrong derivative (S/(S-O)^2 in place of O/(S-O)^2), a missing
    self term or a missing square would move the ratio far outside the
    chi-square band."""
    a, b = small_pair
    K = 400
    full, pair_only = _replicates(a, b, K, n_self=256, n_pair=4096)
    T = full["T"][:, 1]
    np.testing.assert_array_equal(T, pair_only["T"][:, 1])  # same estimates, only the SE differs
    var_T = T.var(ddof=1)
    r_full = var_T / np.mean(full["seT"][:, 1] ** 2)
    r_pair = var_T / np.mean(pair_only["seT"][:, 1] ** 2)
    # sample variance of 400 near-normal values: relative SD sqrt(2/399) = 7%; +-4 SD band
    assert 0.72 < r_full < 1.30, (r_full, r_pair)
    assert r_pair > 4.0, (r_full, r_pair)
    # first-order slot: closed-form self-overlaps with zero SE -> both SEs agree
    np.testing.assert_allclose(full["seT"][:, 0], pair_only["seT"][:, 0], rtol=1e-12)


def test_full_delta_se_reduces_to_the_paper_formula_for_precise_self_overlaps(small_pair):
    """With self-overlaps from 2^18 samples the self term is negligible: the
    full SE is within 2% of the pair-only SE, and both describe the spread of
    T over replicates."""
    a, b = small_pair
    K = 200
    full, pair_only = _replicates(a, b, K, n_self=1 << 18, n_pair=2048)
    ratio = full["seT"][:, 1] / pair_only["seT"][:, 1]
    assert np.all(ratio >= 1.0) and np.all(ratio < 1.02), ratio.max()
    var_T = full["T"][:, 1].var(ddof=1)
    assert 0.6 < var_T / np.mean(full["seT"][:, 1] ** 2) < 1.45


@pytest.fixture(scope="module")
def mol9():
    return synth.generate(31, [9])


def test_self_overlap_control_variate_unbiased_for_any_weights(mol9):
    """O_AA = sum_ij w_i w_j int g_i g_j + Z E_q[(u^2 - u~^2)/m] against the
    exact union self-overlap (inclusion-exclusion cross series, Eq. incexc),
    and V against the exact union volume, for zero, random and fitted
    weights."""
    S_exact = O.union_overlap_ie(mol9, 0, mol9, 0)
    V_exact = O.union_volume_ie(mol9, 0)
    rng = np.random.default_rng(5)
    fitted = O.cv_fit_weights(mol9, [0], seed=8, n=4096)
    K = 16
    idx = np.zeros(K, np.int32)
    for omega in (np.zeros(mol9.n_atoms), rng.uniform(-0.2, 1.3, mol9.n_atoms), fitted):
        v, vs, so, ss = O.union_self_cv(mol9, idx, omega, seed=12, n=4096)
        for est, se, truth in ((so, ss, S_exact), (v, vs, V_exact)):
            z = (est - truth) / se
            assert np.sum(np.abs(z) > 3) <= 1, z
            assert abs(z.mean()) < 3.5 / np.sqrt(K), z


def test_self_overlap_control_variate_zero_weights_is_the_plain_estimator(mol9):
    idx = np.array([0, 0, 0], np.int32)
    plain = O.union_volume_estimate(mol9, idx, seed=4, n=3000, stream_base=9)
    for omega in (None, np.zeros(mol9.n_atoms)):
        cv = O.union_self_cv(mol9, idx, omega, seed=4, n=3000, stream_base=9)
        for x, y in zip(cv, plain):
            np.testing.assert_allclose(x, y, rtol=1e-12)


def test_self_overlap_control_variate_exact_for_one_atom():
    """One atom with weight 1: u = u~ = g, the residual vanishes and the
    estimate is the closed form, int g^2 = p^2 (pi / (2 alpha))^{3/2}
    (Gaussian product theorem), with zero SE up to rounding; the volume is
    p (pi/alpha)^{3/2}."""
    R, p = 1.7, 2.0 * np.sqrt(2.0)
    ms = MolSet(np.array([[0.3, -1.0, 2.0]], np.float32), np.array([R], np.float32), np.array([0, 1], np.int32),
                np.zeros(1, np.uint8))
    alpha = 2.41798793 / float(np.float32(R)) ** 2
    v, vs, so, ss = O.union_self_cv(ms, [0, 0], np.ones(1), seed=1, n=512)
    np.testing.assert_allclose(so, p * p * (np.pi / (2 * alpha)) ** 1.5, rtol=1e-12)
    np.testing.assert_allclose(v, p * (np.pi / alpha) ** 1.5, rtol=1e-12)
    assert np.all(ss < 1e-12 * so) and np.all(vs < 1e-12 * v)  # rounding of 1 - (1 - g) only

