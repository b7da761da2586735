"""Self-overlaps to a stated precision and the full delta-method SE(T) on
the GPU, against the FP64 oracle on the same streams.

The union self-overlaps O_QQ, O_DD of a Tanimoto are importance-sampled
(Eq. union-is with B = A), so their own error reaches T. The library
estimates them to a requested relative SE (rounds of 256 samples, the stop
decision taken in FP32 from the running sums), optionally with the
weighted-Gaussian control variate, and the screen propagates their SEs into
SE(T) and into the adaptive stop rule. Also the least-squares control-variate
fit's guards: a ridge of 0 on nearly coincident atoms and an id outside the
set."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import synth
from paper_2607_20766_b300.synth import MolSet

from test_gpu_adaptive import assert_close, check_adaptive_against_oracle

pytestmark = pytest.mark.gpu

RTOL = 1e-5


@pytest.fixture(scope="module")
def mols():
    ms = synth.generate(71, [1, 7, 12, 18, 33, 60, 64, 25])
    return ms, shp.shape_set_load(ms)


@pytest.mark.parametrize("n", [1000, 4096])
@pytest.mark.parametrize("with_cv", [False, True])
def test_union_self_estimate_matches_oracle(mols, n, with_cv):
    ms, S = mols
    rng = np.random.default_rng(n + with_cv)
    omega = rng.uniform(-0.1, 1.1, ms.n_atoms).astype(np.float32) if with_cv else None
    idx = np.array([1, 2, 3, 7, 6, 5, 4, 0], np.int32)
    vol, vse, so, sse, nu = shp.union_self_estimate(S, idx, None if omega is None else torch.tensor(omega), seed=8,
                                                    n_samples=n, stream_base=2)
    ref = O.union_self_cv(ms, idx, None if omega is None else omega.astype(np.float64), seed=8, n=n, stream_base=2)
    assert_close(vol.cpu().numpy(), ref[0], what="volume")
    assert_close(so.cpu().numpy(), ref[2], what="self-overlap")
    # the one-atom molecule (id 0) with unit-free weights has a tiny, rounding-level SE: compare the others
    keep = idx != 0
    assert_close(vse.cpu().numpy()[keep], ref[1][keep], rtol=1e-4, what="volume SE")
    assert_close(sse.cpu().numpy()[keep], ref[3][keep], rtol=1e-4, what="self-overlap SE")
    assert np.all(nu.cpu().numpy() == n)
    if not with_cv:  # the plain path is the same estimator as union_volume_estimate
        v2, s2, so2, ss2 = shp.union_volume_estimate(S, idx, seed=8, n_samples=n, stream_base=2)
        assert_close(so.cpu().numpy(), so2.cpu().numpy().astype(np.float64), rtol=2e-6, what="vs union_volume_estimate")


@pytest.mark.parametrize("with_cv", [False, True])
def test_adaptive_self_overlap_stop_rule(mols, with_cv):
    """Rounds of 256 until SE(O_AA)/O_AA <= target: the oracle reproduces the
    estimate at each molecule's n_used and checks the decision (met at
    n_used unless at the cap; not met one round earlier)."""
    ms, S = mols
    target, rnd, cap = 0.004, 256, 1 << 16
    idx = np.arange(1, ms.n_mol, dtype=np.int32)
    omega = O.cv_fit_weights(ms, np.arange(ms.n_mol), seed=5, n=2048).astype(np.float32) if with_cv else None
    om64 = None if omega is None else omega.astype(np.float64)
    _, _, so, sse, nu = shp.union_self_estimate(S, idx, None if omega is None else torch.tensor(omega), seed=3,
                                                n_samples=cap, target_rel_se=target, round=rnd, watch=1)
    so, sse, nu = so.cpu().numpy(), sse.cpu().numpy(), nu.cpu().numpy().astype(np.int64)
    assert np.all(nu % rnd == 0) and np.all(nu >= rnd) and np.all(nu <= cap)
    assert len(np.unique(nu)) >= 3
    for k, m in enumerate(idx):
        ref = O.union_self_cv(ms, [m], om64, seed=3, n=int(nu[k]), stream_base=k)
        assert_close(so[k:k + 1], ref[2], what=f"self-overlap of molecule {m} at n={nu[k]}")
        assert_close(sse[k:k + 1], ref[3], rtol=1e-4, what=f"its SE")
        if nu[k] < cap:
            assert ref[3][0] <= target * abs(ref[2][0]) * (1 + 1e-4)
        if nu[k] > rnd:
            prev = O.union_self_cv(ms, [m], om64, seed=3, n=int(nu[k] - rnd), stream_base=k)
            assert prev[3][0] > target * abs(prev[2][0]) * (1 - 1e-4)


@pytest.fixture(scope="module")
def screen_sets():
    q = synth.principal_axes(synth.generate(23, [22, 40]))
    d = synth.principal_axes(synth.generate(24, synth.counts_heavy(24, 40)))
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    # self-overlaps from 8192 samples: their SE matters against tau
    sq, sq_se, _ = shp.self_overlaps(Sq, seed=6, n_samples=8192, with_se=True)
    sd, sd_se, _ = shp.self_overlaps(Sd, seed=6, n_samples=8192, stream_base=10, with_se=True)
    return q, d, Sq, Sd, sq, sq_se, sd, sd_se


def test_self_overlaps_with_se_match_oracle(screen_sets):
    q, d, Sq, Sd, sq, sq_se, sd, sd_se = screen_sets
    k = np.arange(d.n_mol)
    ref = O.union_volume_estimate(d, k, seed=6, n=8192, stream_base=10)
    assert_close(sd[:, 1].cpu().numpy(), ref[2], what="union self-overlaps")
    assert_close(sd_se[:, 1].cpu().numpy(), ref[3], rtol=1e-4, what="their SEs")
    assert np.all(sd_se[:, 0].cpu().numpy() == 0)
    assert_close(sd[:, 0].cpu().numpy(), O.fo_overlap(d, k, d, k), what="closed-form self-overlaps")


def test_fixed_screen_full_delta_se(screen_sets):
    q, d, Sq, Sd, sq, sq_se, sd, sd_se = screen_sets
    res = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=12, n_fixed=3000, with_overlaps=True, self_se_q=sq_se,
                              self_se_db=sd_se)
    plain = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=12, n_fixed=3000)
    pairs = np.arange(q.n_mol * d.n_mol)
    iq, idd = pairs // d.n_mol, pairs % d.n_mol
    ref = O.tanimoto_pairs(q, iq, d, idd, pairs.astype(np.uint64), sq.cpu().numpy(), sd.cpu().numpy(), seed=12,
                           n=3000, selfQ_se=sq_se.cpu().numpy(), selfD_se=sd_se.cpu().numpy())
    assert_close(res["T"].cpu().numpy(), ref["T"], what="T")
    assert_close(res["seT"].cpu().numpy(), ref["seT"], what="full SE(T)")
    # same T as without the self SEs; the union SE(T) grows, the first-order one does not
    np.testing.assert_array_equal(res["T"].cpu().numpy(), plain["T"].cpu().numpy())
    se_full, se_pair = res["seT"].cpu().numpy(), plain["seT"].cpu().numpy()
    assert np.all(se_full[:, 1] > se_pair[:, 1])
    np.testing.assert_array_equal(se_full[:, 0], se_pair[:, 0])


@pytest.mark.parametrize("with_cv", [False, True])
def test_adaptive_screen_watches_the_full_se(screen_sets, with_cv):
    q, d, Sq, Sd, sq, sq_se, sd, sd_se = screen_sets
    tau, rnd, min_n, cap = 0.01, 256, 512, 16384
    om_q = om_d = None
    kw = {}
    if with_cv:
        om_q = shp.cv_fit_weights(Sq, seed=1, n_samples=1024)
        om_d = shp.cv_fit_weights(Sd, seed=2, n_samples=1024)
        kw = dict(omega_q=om_q, omega_db=om_d)
    res = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=7, tau=tau, round=rnd, min_n=min_n, cap=cap, with_overlaps=True,
                              self_se_q=sq_se, self_se_db=sd_se, stream_base=5, **kw)
    pairs = np.arange(q.n_mol * d.n_mol)
    nu = check_adaptive_against_oracle(
        q, d, res, sq.cpu().numpy(), sd.cpu().numpy(), 7, tau, rnd, min_n, cap, pairs, d.n_mol, stream_base=5,
        omega_q=None if om_q is None else om_q.cpu().numpy().astype(np.float64),
        omega_d=None if om_d is None else om_d.cpu().numpy().astype(np.float64),
        sq_se=sq_se.cpu().numpy(), sd_se=sd_se.cpu().numpy())
    assert len(np.unique(nu)) >= 3
    # every pair that stopped early meets the full SE, not only the pair term
    seT = res["seT"].cpu().numpy()[:, 1]
    assert np.all(seT[nu < cap] <= tau * (1 + 1e-4))


def test_least_squares_fit_ridge_zero_on_nearly_coincident_atoms():
    """Two atoms 0.1 A apart make G nearly singular; with ridge 0 the
    conjugate gradients stop at the last finite iterate instead of writing
    inf/NaN weights."""
    xyz = np.array([[0, 0, 0], [0.1, 0, 0], [1.5, 0, 0], [2.3, 1.2, 0]], np.float32)
    ms = MolSet(xyz, np.array([1.7, 1.7, 1.55, 1.52], np.float32), np.array([0, 4], np.int32),
                np.zeros(4, np.uint8))
    S = shp.shape_set_load(ms)
    om = shp.cv_fit_weights(S, seed=4, n_samples=2048, ridge=0.0)
    assert torch.all(torch.isfinite(om)), om
    # usable as a control variate: the volume estimate with them stays unbiased
    V = O.union_volume_ie(ms, 0)
    vol, se, _ = shp.union_volume_cv(S, np.zeros(8, np.int32), om, seed=6, n_samples=4096)
    z = ((vol.cpu().numpy() - V) / se.cpu().numpy())
    assert np.all(np.isfinite(z)) and np.sum(np.abs(z) > 3) <= 1, z


def test_least_squares_fit_skips_an_id_outside_the_set():
    ms = synth.generate(81, [14, 20, 9])
    S = shp.shape_set_load(ms)
    out = torch.full((ms.n_atoms,), -7.0, dtype=torch.float32, device="cuda")
    shp.cv_fit_weights(S, seed=2, n_samples=1024, idx=[2, 5, 0], out=out)
    om = out.cpu().numpy()
    lo1, hi1 = ms.offsets[1], ms.offsets[2]
    assert np.all(om[lo1:hi1] == -7.0)  # molecule 1 was not listed: untouched
    # the stream is the position in the list: molecule 2 uses stream 0, molecule 0 stream 2
    ref2 = O.cv_fit_weights(ms, [2], seed=2, n=1024, stream_base=0)
    ref0 = O.cv_fit_weights(ms, [0], seed=2, n=1024, stream_base=2)
    for ref, k in ((ref2, 2), (ref0, 0)):
        lo, hi = ms.offsets[k], ms.offsets[k + 1]
        np.testing.assert_allclose(om[lo:hi], ref[lo:hi], rtol=1e-4, atol=2e-4 * np.abs(ref[lo:hi]).max())


def test_full_se_matches_the_spread_of_T_over_replicates():
    """End to end on the GPU: 400 independent replicates of one pair (copies
    of both molecules, so every replicate has its own self-overlap and pair
    streams) with noisy self-overlaps (256 samples): the spread of the union T
    is what the screen's full SE(T) predicts, and several times what the
    paper's pair-only SE predicts."""
    a, b = synth.single_pair(n_a=8, n_b=10, seed_a=3, seed_b=4, separation=0.8)
    K = 400

    def copies(ms):
        n = ms.n_atoms
        return MolSet(np.tile(ms.xyz, (K, 1)), np.tile(ms.radius, K), np.arange(K + 1, dtype=np.int32) * n,
                      np.tile(ms.elem, K))

    Sa, Sb = shp.shape_set_load(copies(a)), shp.shape_set_load(copies(b))
    sa, sa_se, _ = shp.self_overlaps(Sa, seed=101, n_samples=256, with_se=True)
    sb, sb_se, _ = shp.self_overlaps(Sb, seed=101, n_samples=256, stream_base=10 * K, with_se=True)
    k = torch.arange(K, dtype=torch.int32, device="cuda")
    full = shp.tanimoto_screen(Sa, Sb, sa, sb, seed=202, n_fixed=4096, pairs=(k, k), self_se_q=sa_se,
                               self_se_db=sb_se)
    pair_only = shp.tanimoto_screen(Sa, Sb, sa, sb, seed=202, n_fixed=4096, pairs=(k, k))
    T = full["T"][:, 1].cpu().numpy().astype(np.float64)
    np.testing.assert_array_equal(T, pair_only["T"][:, 1].cpu().numpy())
    var_T = T.var(ddof=1)
    r_full = var_T / np.mean(full["seT"][:, 1].cpu().numpy().astype(np.float64) ** 2)
    r_pair = var_T / np.mean(pair_only["seT"][:, 1].cpu().numpy().astype(np.float64) ** 2)
    assert 0.72 < r_full < 1.30, (r_full, r_pair)
    assert r_pair > 4.0, (r_full, r_pair)


def test_edge_cases_of_the_new_entry_points(mols):
    ms, S = mols
    empty = MolSet(np.zeros((0, 3), np.float32), np.zeros(0, np.float32), np.zeros(1, np.int32),
                   np.zeros(0, np.uint8))
    E = shp.shape_set_load(empty)
    out = shp.union_self_estimate(E, None, seed=1, n_samples=256)
    assert all(t.numel() == 0 for t in out)
    with pytest.raises(shp.ShapeError):  # the cap is not a multiple of the round
        shp.union_self_estimate(S, None, seed=1, n_samples=1000, target_rel_se=0.01, round=256)
    with pytest.raises(shp.ShapeError):  # watch is 0 or 1
        shp.union_self_estimate(S, None, seed=1, n_samples=512, watch=2)
    # an out-of-range molecule id gives NaN outputs for that item only
    vol, vse, so, sse, nu = shp.union_self_estimate(S, [0, 99, 2], seed=1, n_samples=512)
    so = so.cpu().numpy()
    assert np.isfinite(so[[0, 2]]).all() and np.isnan(so[1])
    # an empty pair list screens nothing; k = n_db selects every pair
    sq, sq_se, _ = shp.self_overlaps(S, seed=2, n_samples=512, with_se=True)
    none = torch.zeros(0, dtype=torch.int32, device="cuda")
    res = shp.tanimoto_screen(S, S, sq, sq, seed=1, n_fixed=256, pairs=(none, none))
    assert res["T"].shape == (0, 2)
    T_fo = shp.fo_tanimoto_screen(S, S, sq[:, 0], sq[:, 0])
    pq, pd = shp.fo_prefilter_select(S, S, T_fo, ms.n_mol)
    np.testing.assert_array_equal(pd.cpu().numpy(), np.tile(np.arange(ms.n_mol), ms.n_mol))
    # a molecule with itself: first-order Tanimoto 1
    diag = T_fo.view(ms.n_mol, ms.n_mol).diagonal().cpu().numpy()
    np.testing.assert_allclose(diag, 1.0, rtol=2e-5)
    assert shp.fo_tanimoto_screen(S, E, sq[:, 0], torch.zeros(0, dtype=torch.float64)).numel() == 0
