"""Adaptive confidence-bounded screen (Sec. confidence-bounded screening) and
the screen's launch variants, against the FP64 oracle.

The stop decision is an integer (samples used) decided by floating point:
the kernel takes it in FP32 from its running sums. The oracle reproduces
the estimates at the kernel's n_used exactly (same streams: the first n_used
samples of each direction) and checks that the decision is valid -- SE(T)
at n_used is within tolerance of tau or the cap was hit, and SE(T) one round
earlier was above tau or n_used is the minimum.
"""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-5


def assert_close(gpu, ref, rtol=RTOL, what=""):
    gpu = np.asarray(gpu, np.float64)
    e = np.abs(gpu - ref) / np.maximum(np.abs(ref), 1e-300)
    assert np.all(np.isfinite(gpu)), what
    assert e.max() <= rtol, f"{what}: max rel err {e.max():.3e}"


def oracle_self(ms, seed, n, stream_base=0):
    k = np.arange(ms.n_mol)
    fo = O.fo_overlap(ms, k, ms, k)
    so = O.union_volume_estimate(ms, k, seed=seed, n=n, stream_base=stream_base)[2]
    return np.stack([fo, so], 1)


@pytest.fixture(scope="module")
def small_screen():
    q = synth.principal_axes(synth.generate(21, [20, 36, 48]))
    d = synth.principal_axes(synth.generate(22, synth.counts_heavy(22, 50)))
    return q, d, shp.shape_set_load(q), shp.shape_set_load(d), oracle_self(q, 1, 8192), oracle_self(d, 2, 8192)


def check_adaptive_against_oracle(q, d, res, sq, sd, seed, tau, rnd, min_n, cap, pairs, n_db, stream_base=0,
                                  omega_q=None, omega_d=None, sq_se=None, sd_se=None):
    nu = res["n_used"].cpu().numpy().astype(np.int64)[pairs]
    iq, idd = pairs // n_db, pairs % n_db
    assert np.all(nu % rnd == 0) and np.all(nu >= min_n) and np.all(nu <= cap)
    T = res["T"].cpu().numpy()[pairs]
    seT = res["seT"].cpu().numpy()[pairs]
    O_ = res["O"].cpu().numpy()[pairs]
    seO = res["seO"].cpu().numpy()[pairs]
    for n in np.unique(nu):
        sel = nu == n
        ref = O.tanimoto_pairs(q, iq[sel], d, idd[sel], (stream_base + pairs[sel]).astype(np.uint64), sq, sd,
                               seed=seed, n=int(n), omega_q=omega_q, omega_d=omega_d, selfQ_se=sq_se, selfD_se=sd_se)
        assert_close(O_[sel], ref["O"], what=f"O at n={n}")
        assert_close(seO[sel], ref["seO"], what=f"seO at n={n}")
        assert_close(T[sel], ref["T"], what=f"T at n={n}")
        assert_close(seT[sel], ref["seT"], what=f"seT at n={n}")
        # stop rule validity (union slot watched)
        if n < cap:
            assert np.all(ref["seT"][:, 1] <= tau * (1 + 1e-4)), "stopped before SE(T) <= tau"
        if n > min_n:
            prev = O.tanimoto_pairs(q, iq[sel], d, idd[sel], (stream_base + pairs[sel]).astype(np.uint64), sq, sd,
                                    seed=seed, n=int(n - rnd), omega_q=omega_q, omega_d=omega_d, selfQ_se=sq_se,
                                    selfD_se=sd_se)
            assert np.all(prev["seT"][:, 1] > tau * (1 - 1e-4)), "did not stop when SE(T) <= tau"
    return nu


def test_adaptive_parity_and_stop_rule(small_screen):
    q, d, Sq, Sd, sq, sd = small_screen
    tau, rnd, min_n, cap = 0.012, 256, 512, 6144
    res = shp.tanimoto_screen(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=5, tau=tau, round=rnd, min_n=min_n,
                              cap=cap, with_overlaps=True, stream_base=3)
    pairs = np.arange(q.n_mol * d.n_mol)
    nu = check_adaptive_against_oracle(q, d, res, sq, sd, 5, tau, rnd, min_n, cap, pairs, d.n_mol, stream_base=3)
    # the rule must actually adapt on this set: several distinct budgets
    assert len(np.unique(nu)) >= 3


def test_adaptive_first_order_watch(small_screen):
    q, d, Sq, Sd, sq, sd = small_screen
    res = shp.tanimoto_screen(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=9, tau=0.02, round=512, min_n=512,
                              cap=4096, watch=0, with_overlaps=True)
    nu = res["n_used"].cpu().numpy().astype(np.int64)
    pairs = np.arange(len(nu))
    for n in np.unique(nu):
        sel = pairs[nu == n]
        ref = O.tanimoto_pairs(q, sel // d.n_mol, d, sel % d.n_mol, sel.astype(np.uint64), sq, sd, seed=9, n=int(n))
        assert_close(res["T"].cpu().numpy()[sel], ref["T"], what="T")
        if n < 4096:
            assert np.all(ref["seT"][:, 0] <= 0.02 * (1 + 1e-4))


def test_adaptive_rejects_bad_config(small_screen):
    q, d, Sq, Sd, sq, sd = small_screen
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=1, round=100)
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=1, min_n=512, cap=256)
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=1, tau=0.0)


def test_variants_agree(small_screen):
    """Every launch variant draws the same samples; only the summation order
    differs between sample-per-lane widths."""
    q, d, Sq, Sd, sq, sd = small_screen
    tq, td = torch.tensor(sq), torch.tensor(sd)
    nv = shp.screen_variants()
    ref = shp.tanimoto_screen(Sq, Sd, tq, td, seed=4, n_fixed=1000, variant=0, with_overlaps=True)
    for v in range(1, nv):
        r = shp.tanimoto_screen(Sq, Sd, tq, td, seed=4, n_fixed=1000, variant=v, with_overlaps=True)
        assert_close(r["O"].cpu().numpy(), ref["O"].cpu().numpy(), rtol=2e-6, what=f"variant {v}")
    sp4 = [v for v in range(nv) if shp.screen_variant_info(v)["sp"] == 4]
    ada = {v: shp.tanimoto_screen(Sq, Sd, tq, td, seed=4, tau=0.015, min_n=512, cap=4096, variant=v,
                                  with_overlaps=True) for v in sp4}
    for v in sp4[1:]:
        np.testing.assert_array_equal(ada[v]["n_used"].cpu().numpy(), ada[sp4[0]]["n_used"].cpu().numpy())
        assert_close(ada[v]["O"].cpu().numpy(), ada[sp4[0]]["O"].cpu().numpy(), rtol=2e-6,
                     what=f"adaptive variant {v}")
    other = [v for v in range(nv) if v not in sp4]
    assert other, "no variant with another batch width"
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, tq, td, seed=4, tau=0.015, variant=other[0])  # cannot run rounds of 256


def test_tuner_picks_a_valid_variant(small_screen):
    q, d, Sq, Sd, sq, sd = small_screen
    best, times = shp.tanimoto_screen_tune(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=1, n_fixed=2048,
                                           n_sample=64)
    assert 0 <= best < shp.screen_variants()
    assert times[best] > 0 and np.all(times[times > 0] >= times[best])
    best_a, times_a = shp.tanimoto_screen_tune(Sq, Sd, torch.tensor(sq), torch.tensor(sd), seed=1, n_sample=64)
    sp4 = np.array([shp.screen_variant_info(v)["sp"] == 4 for v in range(shp.screen_variants())])
    assert sp4[best_a] and np.all(times_a[~sp4] == -1) and np.all(times_a[sp4] > 0)


def oracle_self_at(ms, ids, n_used, seed, stream_base, target, rnd):
    """The oracle's union self-overlaps and SEs of molecules `ids` at the
    library's sample counts (same streams), and the check of each adaptive
    stop decision: SE/O <= target at n unless capped, > target one round
    earlier unless at the first round."""
    so, se = np.zeros(len(ids)), np.zeros(len(ids))
    for j, (k, n) in enumerate(zip(ids, n_used)):
        _, _, a, b = O.union_volume_estimate(ms, [k], seed=seed, n=int(n), stream_base=stream_base + int(k))
        so[j], se[j] = a[0], b[0]
        assert se[j] <= target * so[j] * (1 + 1e-4)
        if n > rnd:
            _, _, a0, b0 = O.union_volume_estimate(ms, [k], seed=seed, n=int(n - rnd), stream_base=stream_base + int(k))
            assert b0[0] > target * a0[0] * (1 - 1e-4)
    return so, se


def test_adaptive_full_size_sampled():
    """16 queries (20-48 atoms) x 1,000,000 molecules (18-60, heavy-tailed
    toward 40), rounds of 256, full SE(T) <= 0.005 or 65,536 per direction:
    the launch the benchmark times (self-overlaps to relative SE 3.5e-3,
    queries 8.75e-4, their SEs in SE(T) and the stop rule; autotuned
    variant, replayed CUDA graph); 24 sampled pairs and their molecules'
    self-overlaps checked by the oracle."""
    q, d = synth.adaptive_screen()
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    selfq, seq, nq = shp.self_overlaps(Sq, seed=11, n_samples=1 << 24, stream_base=0, target_rel_se=8.75e-4,
                                       round=4096, with_se=True)
    selfd, sed, nd = shp.self_overlaps(Sd, seed=11, n_samples=1 << 22, stream_base=16, target_rel_se=3.5e-3,
                                       round=256, with_se=True)
    kw = dict(self_se_q=seq, self_se_db=sed)
    shp.tanimoto_screen_tune(Sq, Sd, selfq, selfd, seed=77, n_sample=16384, tau=0.005, cap=65536, **kw)
    g = shp.StepGraph(shp.tanimoto_screen, Sq, Sd, selfq, selfd, seed=77, tau=0.005, round=256, min_n=1024,
                      cap=65536, with_overlaps=True, **kw)
    res = g.replay()
    torch.cuda.synchronize()
    nu = res["n_used"].cpu().numpy()
    assert np.all(nu % 256 == 0) and nu.min() >= 1024 and nu.max() <= 65536
    rng = np.random.default_rng(3)
    # 24 pairs of two queries (the oracle's query self-overlaps take ~10^6 samples each)
    pairs = np.sort(np.concatenate([qq * d.n_mol + rng.choice(d.n_mol, 12, replace=False)
                                    for qq in rng.choice(q.n_mol, 2, replace=False)]))
    qs, ds = np.unique(pairs // d.n_mol), np.unique(pairs % d.n_mol)
    sq, sd = np.zeros((q.n_mol, 2)), np.zeros((d.n_mol, 2))
    eq, ed = np.zeros((q.n_mol, 2)), np.zeros((d.n_mol, 2))
    sq[qs, 0] = O.fo_overlap(q, qs, q, qs)
    sd[ds, 0] = O.fo_overlap(d, ds, d, ds)
    sq[qs, 1], eq[qs, 1] = oracle_self_at(q, qs, nq.cpu().numpy()[qs], 11, 0, 8.75e-4, 4096)
    sd[ds, 1], ed[ds, 1] = oracle_self_at(d, ds, nd.cpu().numpy()[ds], 11, 16, 3.5e-3, 256)
    for got, ref, what in ((selfq.cpu().numpy()[qs], sq[qs], "query self-overlaps"),
                           (selfd.cpu().numpy()[ds], sd[ds], "database self-overlaps")):
        assert_close(got, ref, what=what)
    assert_close(sed.cpu().numpy()[ds, 1], ed[ds, 1], rtol=1e-4, what="their SEs")
    check_adaptive_against_oracle(q, d, res, sq, sd, 77, 0.005, 256, 1024, 65536, pairs, d.n_mol, sq_se=eq,
                                  sd_se=ed)


def test_graph_captured_adaptive_step_matches_eager(small_screen):
    """The adaptive step (self-overlaps of both sets + the adaptive screen)
    captured as one CUDA graph: every replay reproduces the eager call bit for
    bit, and the replayed estimates pass the oracle's checks."""
    q, d, Sq, Sd, sq, sd = small_screen

    def step():
        selfq = shp.self_overlaps(Sq, seed=1, n_samples=8192)
        selfd = shp.self_overlaps(Sd, seed=2, n_samples=8192)
        return selfq, selfd, shp.tanimoto_screen(Sq, Sd, selfq, selfd, seed=5, tau=0.012, round=256, min_n=512,
                                                 cap=6144, with_overlaps=True, stream_base=3)

    eager = step()
    g = shp.StepGraph(step)
    for _ in range(2):
        selfq, selfd, res = g.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(selfq.cpu().numpy(), eager[0].cpu().numpy())
        np.testing.assert_array_equal(selfd.cpu().numpy(), eager[1].cpu().numpy())
        for k in ("T", "seT", "O", "seO", "n_used"):
            np.testing.assert_array_equal(res[k].cpu().numpy(), eager[2][k].cpu().numpy())
    pairs = np.arange(q.n_mol * d.n_mol)
    check_adaptive_against_oracle(q, d, res, sq, sd, 5, 0.012, 256, 512, 6144, pairs, d.n_mol, stream_base=3)


def test_control_variate_screen_parity(small_screen):
    """Union slot with the weighted-Gaussian control variate (any weights),
    fixed budget and adaptive, against the oracle on the same streams; every
    variant built with it agrees."""
    q, d, Sq, Sd, sq, sd = small_screen
    rng = np.random.default_rng(8)
    wq = rng.uniform(0.3, 1.1, q.n_atoms).astype(np.float32)
    wd = rng.uniform(0.3, 1.1, d.n_atoms).astype(np.float32)
    tq, td = torch.tensor(sq), torch.tensor(sd)
    gq, gd = torch.tensor(wq), torch.tensor(wd)
    pairs = np.arange(q.n_mol * d.n_mol)
    ref = O.tanimoto_pairs(q, pairs // d.n_mol, d, pairs % d.n_mol, (2 + pairs).astype(np.uint64), sq, sd, seed=6,
                           n=1500, omega_q=wq.astype(np.float64), omega_d=wd.astype(np.float64))
    cv_variants = []
    for v in range(shp.screen_variants()):
        try:
            res = shp.tanimoto_screen(Sq, Sd, tq, td, seed=6, n_fixed=1500, stream_base=2, with_overlaps=True,
                                      omega_q=gq, omega_db=gd, variant=v)
        except shp.ShapeError:
            continue
        cv_variants.append(v)
        for k in ("O", "seO", "T", "seT"):
            assert_close(res[k].cpu().numpy(), ref[k], what=f"{k} (variant {v})")
    assert len(cv_variants) >= 2
    res = shp.tanimoto_screen(Sq, Sd, tq, td, seed=5, tau=0.012, round=256, min_n=512, cap=6144, with_overlaps=True,
                              stream_base=3, omega_q=gq, omega_db=gd)
    check_adaptive_against_oracle(q, d, res, sq, sd, 5, 0.012, 256, 512, 6144, pairs, d.n_mol, stream_base=3,
                                  omega_q=wq.astype(np.float64), omega_d=wd.astype(np.float64))
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, tq, td, seed=5, n_fixed=512, omega_q=gq)  # one weight array only


def test_adaptive_parity_when_centroids_are_apart(small_screen):
    """Database molecules shifted 6 A away from the queries: the adaptive
    kernel stages each direction in its own frame instead of the shared one;
    estimates and stop decisions still match the oracle."""
    q, d, Sq, Sd, sq, sd = small_screen
    from paper_2607_20766_b300.synth import MolSet
    dd = MolSet(d.xyz + np.float32([6.0, 0.0, 0.0]), d.radius, d.offsets, d.elem)
    Sdd = shp.shape_set_load(dd)
    sdd = oracle_self(dd, 2, 8192)
    tau, rnd, min_n, cap = 0.02, 256, 512, 4096
    res = shp.tanimoto_screen(Sq, Sdd, torch.tensor(sq), torch.tensor(sdd), seed=15, tau=tau, round=rnd,
                              min_n=min_n, cap=cap, with_overlaps=True)
    pairs = np.arange(q.n_mol * dd.n_mol)
    check_adaptive_against_oracle(q, dd, res, sq, sdd, 15, tau, rnd, min_n, cap, pairs, dd.n_mol)


def test_graph_captured_control_variate_screen_matches_eager(small_screen):
    """The control-variate screen (fixed and adaptive) replayed from a CUDA
    graph equals the eager call bit for bit."""
    q, d, Sq, Sd, sq, sd = small_screen
    rng = np.random.default_rng(12)
    wq = torch.tensor(rng.uniform(0.4, 1.0, q.n_atoms).astype(np.float32), device="cuda")
    wd = torch.tensor(rng.uniform(0.4, 1.0, d.n_atoms).astype(np.float32), device="cuda")
    tq, td = torch.tensor(sq, device="cuda"), torch.tensor(sd, device="cuda")
    for kw in (dict(n_fixed=1024), dict(tau=0.012, min_n=512, cap=4096)):
        eager = shp.tanimoto_screen(Sq, Sd, tq, td, seed=8, with_overlaps=True, omega_q=wq, omega_db=wd, **kw)
        g = shp.StepGraph(shp.tanimoto_screen, Sq, Sd, tq, td, seed=8, with_overlaps=True, omega_q=wq, omega_db=wd,
                          **kw)
        res = g.replay()
        torch.cuda.synchronize()
        for k in ("T", "seT", "O", "seO", "n_used"):
            np.testing.assert_array_equal(res[k].cpu().numpy(), eager[k].cpu().numpy())


def test_graph_replay_reads_inputs_updated_in_place(small_screen):
    """A captured screen reads its inputs from the addresses seen at capture:
    self-overlaps and control-variate weights updated in place (copy_) are
    picked up by the next replay, which then equals an eager call on the new
    values."""
    q, d, Sq, Sd, sq, sd = small_screen
    tq, td = torch.tensor(sq, device="cuda"), torch.tensor(sd, device="cuda")
    wq = torch.full((q.n_atoms,), 0.5, dtype=torch.float32, device="cuda")
    wd = torch.full((d.n_atoms,), 0.5, dtype=torch.float32, device="cuda")
    g = shp.StepGraph(shp.tanimoto_screen, Sq, Sd, tq, td, seed=9, n_fixed=1024, with_overlaps=True, omega_q=wq,
                      omega_db=wd)
    tq.copy_(tq * 1.01)
    wd.copy_(torch.linspace(0.3, 0.9, d.n_atoms, device="cuda"))
    res = g.replay()
    eager = shp.tanimoto_screen(Sq, Sd, tq, td, seed=9, n_fixed=1024, with_overlaps=True, omega_q=wq, omega_db=wd)
    torch.cuda.synchronize()
    for k in ("T", "seT", "O", "seO"):
        np.testing.assert_array_equal(res[k].cpu().numpy(), eager[k].cpu().numpy())


def test_adaptive_fitted_control_variate_full_size_sampled():
    """The benchmark's control-variate arm at its full size: 16 x 1,000,000
    adaptive screen with least-squares weights fitted from 4096 samples per
    molecule and the full SE(T); 24 sampled pairs recomputed by the oracle
    (same weights, same streams, the library's self-overlaps and SEs) and
    their stop decisions checked."""
    q, d = synth.adaptive_screen()
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    selfq, seq, _ = shp.self_overlaps(Sq, seed=11, n_samples=1 << 24, stream_base=0, target_rel_se=8.75e-4,
                                      round=4096, with_se=True)
    selfd, sed, _ = shp.self_overlaps(Sd, seed=11, n_samples=1 << 22, stream_base=16, target_rel_se=3.5e-3,
                                      round=256, with_se=True)
    wq = shp.cv_fit_weights(Sq, seed=91, n_samples=4096)
    wd = shp.cv_fit_weights(Sd, seed=92, n_samples=4096)
    kw = dict(omega_q=wq, omega_db=wd, self_se_q=seq, self_se_db=sed)
    shp.tanimoto_screen_tune(Sq, Sd, selfq, selfd, seed=77, n_sample=16384, tau=0.005, cap=65536, **kw)
    g = shp.StepGraph(shp.tanimoto_screen, Sq, Sd, selfq, selfd, seed=77, tau=0.005, round=256, min_n=1024,
                      cap=65536, with_overlaps=True, **kw)
    res = g.replay()
    torch.cuda.synchronize()
    nu = res["n_used"].cpu().numpy()
    rng = np.random.default_rng(5)
    pairs = np.sort(rng.choice(len(nu), 24, replace=False))
    sq = np.zeros((q.n_mol, 2))
    sd = np.zeros((d.n_mol, 2))
    qs, ds = np.unique(pairs // d.n_mol), np.unique(pairs % d.n_mol)
    sq[qs] = selfq.cpu().numpy()[qs]  # the screen's T uses the library's self-overlaps and their SEs
    sd[ds] = selfd[torch.as_tensor(ds, device=selfd.device)].cpu().numpy()
    check_adaptive_against_oracle(q, d, res, sq, sd, 77, 0.005, 256, 1024, 65536, pairs, d.n_mol,
                                  omega_q=wq.cpu().numpy().astype(np.float64),
                                  omega_d=wd.cpu().numpy().astype(np.float64), sq_se=seq.cpu().numpy(),
                                  sd_se=sed.cpu().numpy())
