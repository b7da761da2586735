"""Pins for the oracle's importance-sampling estimators against exact values:
unbiasedness within 3 SE (Eq. expectation, Eq. var, Eq. union-is), the
n^{-1/2} rate, the bounded-weight variance bound for unit heights, the
symmetrised and antithetic variants, and the Tanimoto with its delta-method
SE (Sec. confidence-bounded screening)."""
import numpy as np
import pytest

import oracle as O
from paper_2607_20766_b300 import synth
from paper_2607_20766_b300.synth import MolSet

KAPPA = np.pi * (3 / (4 * np.pi)) ** (2 / 3)


@pytest.fixture(scope="module")
def pair():
    return synth.single_pair()


@pytest.fixture(scope="module")
def exact(pair):
    a, b = pair
    return dict(fo=O.fo_overlap(a, [0], b, [0])[0], ou=O.union_overlap_ie(a, 0, b, 0),
                va=O.union_volume_ie(a, 0), vb=O.union_volume_ie(b, 0), saa=O.union_overlap_ie(a, 0, a, 0))


def _zscores(est, se, truth):
    return (np.asarray(est) - truth) / np.asarray(se)


def test_first_order_and_union_unbiased(pair, exact):
    a, b = pair
    nseed = 24
    est, se = O.overlap_estimate(a, np.zeros(nseed, np.int32), b, np.zeros(nseed, np.int32), seed=17,
                                 n=1 << 14, flags=O.SYMMETRIC)
    for slot, key in ((0, "fo"), (1, "ou")):
        z = _zscores(est[:, slot], se[:, slot], exact[key])
        assert np.sum(np.abs(z) > 3) <= 1, z
        assert abs(z.mean()) < 3.5 / np.sqrt(nseed)
        assert 0.5 < z.std() < 1.6


def test_one_direction_unbiased(pair, exact):
    a, b = pair
    est, se = O.overlap_estimate(a, np.zeros(16, np.int32), b, np.zeros(16, np.int32), seed=5, n=1 << 14,
                                 flags=0)
    for slot, key in ((0, "fo"), (1, "ou")):
        z = _zscores(est[:, slot], se[:, slot], exact[key])
        assert np.sum(np.abs(z) > 3) <= 1, z


def test_volume_and_self_overlap_unbiased(pair, exact):
    a, b = pair
    both = a.concat(b)
    idx = np.array([0] * 12 + [1] * 12, np.int32)
    v, vs, so, ss = O.union_volume_estimate(both, idx, seed=9, n=1 << 14)
    zv = np.concatenate([_zscores(v[:12], vs[:12], exact["va"]), _zscores(v[12:], vs[12:], exact["vb"])])
    zs = _zscores(so[:12], ss[:12], exact["saa"])
    assert np.sum(np.abs(zv) > 3) <= 1, zv
    assert np.sum(np.abs(zs) > 3) <= 1, zs


def test_single_atom_union_weight_is_one():
    """One atom: u = m, w = 1, so V = Z with zero variance."""
    ms = MolSet(np.zeros((1, 3), np.float32), np.array([1.7], np.float32), np.array([0, 1], np.int32),
                np.zeros(1, np.uint8))
    v, vs, so, ss = O.union_volume_estimate(ms, [0], seed=1, n=1000)
    R = float(np.float32(1.7))
    assert v[0] == pytest.approx(4 / 3 * np.pi * R ** 3, rel=1e-8)
    assert vs[0] == pytest.approx(0.0, abs=1e-9)


def test_standard_error_rate(pair):
    """SE proportional to n^{-1/2} (paper Sec. convergence)."""
    a, b = pair
    ns = [1 << k for k in range(9, 16)]
    se_fo, se_u = [], []
    for n in ns:
        est, se = O.overlap_estimate(a, np.zeros(8, np.int32), b, np.zeros(8, np.int32), seed=n, n=n,
                                     flags=O.SYMMETRIC)
        se_fo.append(se[:, 0].mean())
        se_u.append(se[:, 1].mean())
    for s in (se_fo, se_u):
        slope = np.polyfit(np.log(ns), np.log(s), 1)[0]
        assert abs(slope + 0.5) < 0.03


def test_reported_se_matches_spread(pair):
    """The analytic SE (Eq. var) equals the spread of independent estimates."""
    a, b = pair
    est, se = O.overlap_estimate(a, np.zeros(200, np.int32), b, np.zeros(200, np.int32), seed=3, n=2048,
                                 flags=0)
    for slot in (0, 1):
        ratio = est[:, slot].std(ddof=1) / se[:, slot].mean()
        assert 0.85 < ratio < 1.15


def test_unit_height_variance_bound():
    """p <= 1: 0 <= w u_B <= 1, so Var <= Z^2 / (4n) (Sec. union)."""
    a = synth.centre(synth.generate(31, [20]))
    b = synth.centre(synth.generate(32, [25]))
    a.height = np.ones(a.n_atoms, np.float32)
    b.height = np.ones(b.n_atoms, np.float32)
    n = 4096
    est, se = O.overlap_estimate(a, [0], b, [0], seed=2, n=n, flags=0, c_alpha=KAPPA)
    Z = O.mixture_mass(a, c_alpha=KAPPA)[0]
    assert se[0, 1] <= Z / (2 * np.sqrt(n)) * (1 + 1e-12)
    exact = O.grid(a, 0, b, 0, h=0.1, c_alpha=KAPPA)["OU"]
    assert abs(est[0, 1] - exact) < 4 * se[0, 1]


def test_symmetrised_is_average_of_directions(pair):
    a, b = pair
    n, seed = 4096, 77
    s_ab, ne = O.direction_sums(a, 0, b, 0, seed=seed, stream=0, tag=O.TAG_AB, n=n)
    s_ba, _ = O.direction_sums(a, 0, b, 0, seed=seed, stream=0, tag=O.TAG_BA, n=n)
    Za, Zb = O.mixture_mass(a)[0], O.mixture_mass(b)[0]

    def est_se(Z, s):
        mean = s[0] / ne
        var = (s[1] - s[0] * mean) / (ne - 1)
        return Z * mean, Z * np.sqrt(var / ne)

    e1, s1 = est_se(Za, s_ab[2:])
    e2, s2 = est_se(Zb, s_ba[2:])
    est, se = O.overlap_estimate(a, [0], b, [0], seed=seed, n=n, flags=O.SYMMETRIC)
    assert est[0, 1] == pytest.approx(0.5 * (e1 + e2), rel=1e-13)
    assert se[0, 1] == pytest.approx(0.5 * np.hypot(s1, s2), rel=1e-12)


def test_antithetic_unbiased(pair, exact):
    """Antithetic pairs (Sec. IS estimator) stay unbiased. On these molecules
    the reflected sample shares its component and the even part of m_B
    dominates, so the pair is positively correlated: the SE per sample is
    not smaller than without pairing (recorded, not asserted as a gain)."""
    a, b = pair
    k = 16
    est_a, se_a = O.overlap_estimate(a, np.zeros(k, np.int32), b, np.zeros(k, np.int32), seed=41, n=1 << 13,
                                     flags=O.SYMMETRIC | O.ANTITHETIC)
    est_p, se_p = O.overlap_estimate(a, np.zeros(k, np.int32), b, np.zeros(k, np.int32), seed=41, n=1 << 13,
                                     flags=O.SYMMETRIC)
    for slot, key in ((0, "fo"), (1, "ou")):
        z = _zscores(est_a[:, slot], se_a[:, slot], exact[key])
        assert np.sum(np.abs(z) > 3) <= 1, z
    assert 0.7 < se_a[:, 0].mean() / se_p[:, 0].mean() < 1.4


def test_odd_sample_count(pair):
    a, b = pair
    s_odd, ne = O.direction_sums(a, 0, b, 0, seed=1, stream=0, tag=0, n=1001)
    s_even, ne2 = O.direction_sums(a, 0, b, 0, seed=1, stream=0, tag=0, n=1000)
    assert ne == 1001 and ne2 == 1000
    assert s_odd[0] > s_even[0]


def test_tanimoto_identity_and_disjoint(pair):
    """T = O/(O_AA + O_BB - O): a copy of A scores 1 within its SE; a far
    copy scores 0."""
    a, _ = pair
    far = MolSet(a.xyz + np.float32([80, 0, 0]), a.radius, a.offsets, a.elem)
    two = a.concat(far)
    saa = O.union_overlap_ie(a, 0, a, 0)
    foaa = O.fo_overlap(a, [0], a, [0])[0]
    self_ = np.array([[foaa, saa], [foaa, saa]])
    res = O.tanimoto_pairs(two, [0, 0], two, [0, 1], [0, 1], self_, self_, seed=8, n=1 << 14)
    T, seT = res["T"], res["seT"]
    assert np.all(np.abs(T[0] - 1.0) < 3.5 * seT[0])
    assert np.all(np.abs(T[1]) < 1e-12)
    # delta-method SE: S / (S - O)^2 * SE(O)
    S = 2 * self_[0]
    np.testing.assert_allclose(seT[0], S / (S - res["O"][0]) ** 2 * res["seO"][0], rtol=1e-12)
