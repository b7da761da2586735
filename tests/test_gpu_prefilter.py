"""The first-order prefilter of the screen (the cheap stage of the paper's
hybrid pipeline, Sec. first-order overlap): the closed-form first-order
Tanimoto of every pair against the FP64 oracle, and the screen of an
explicit pair list, whose pairs get exactly the numbers the full screen
gives them (streams keyed by (query, database) ids)."""
import numpy as np
import pytest
import torch

import oracle as O
import paper_2607_20766_b300 as shp
from paper_2607_20766_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sets():
    q = synth.principal_axes(synth.generate(31, [20, 33, 48]))
    d = synth.principal_axes(synth.generate(32, synth.counts_heavy(32, 300)))
    return q, d, shp.shape_set_load(q), shp.shape_set_load(d)


def test_fo_tanimoto_matches_oracle(sets):
    q, d, Sq, Sd = sets
    kq, kd = np.arange(q.n_mol), np.arange(d.n_mol)
    fq, fd = O.fo_overlap(q, kq, q, kq), O.fo_overlap(d, kd, d, kd)
    T = shp.fo_tanimoto_screen(Sq, Sd, torch.tensor(fq), torch.tensor(fd)).cpu().numpy()
    iq, idd = np.meshgrid(kq, kd, indexing="ij")
    O_ = O.fo_overlap(q, iq.ravel(), d, idd.ravel())
    ref = O_ / (fq[iq.ravel()] + fd[idd.ravel()] - O_)
    np.testing.assert_allclose(T, ref, rtol=2e-5)
    # the library's own closed-form self-overlaps serve as well
    sq, sd = shp.self_overlaps(Sq, seed=1, n_samples=256), shp.self_overlaps(Sd, seed=1, n_samples=256)
    T2 = shp.fo_tanimoto_screen(Sq, Sd, sq[:, 0], sd[:, 0]).cpu().numpy()
    np.testing.assert_allclose(T2, ref, rtol=2e-5)


@pytest.mark.parametrize("adaptive", [False, True])
def test_pair_list_screen_equals_the_full_screen(sets, adaptive):
    q, d, Sq, Sd = sets
    sq, sq_se, _ = shp.self_overlaps(Sq, seed=2, n_samples=4096, with_se=True)
    sd, sd_se, _ = shp.self_overlaps(Sd, seed=2, n_samples=4096, stream_base=5, with_se=True)
    kw = dict(tau=0.01, min_n=512, cap=8192) if adaptive else dict(n_fixed=1024)
    full = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=8, with_overlaps=True, self_se_q=sq_se, self_se_db=sd_se, **kw)
    rng = np.random.default_rng(1)
    pick = rng.choice(q.n_mol * d.n_mol, 200, replace=False)
    # largest database molecules first, as a caller should list them
    pick = pick[np.argsort(-d.counts[pick % d.n_mol], kind="stable")]
    lst = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=8, with_overlaps=True, self_se_q=sq_se, self_se_db=sd_se,
                              pairs=(pick // d.n_mol, pick % d.n_mol), **kw)
    for k in ("T", "seT", "O", "seO", "n_used"):
        np.testing.assert_array_equal(lst[k].cpu().numpy(), full[k].cpu().numpy()[pick], err_msg=k)
    with pytest.raises(shp.ShapeError):
        shp.tanimoto_screen(Sq, Sd, sq, sd, seed=8, n_fixed=256,
                            pairs=(torch.zeros(3, dtype=torch.int32, device="cuda"), None))


@pytest.mark.parametrize("k", [1, 7, 100, 299, 300])
def test_prefilter_selection_is_the_exact_top_k(sets, k):
    """Per query the k largest scores, ties at the k-th by the lowest id,
    each query's pairs in ascending id: against numpy on scores with many
    ties (quantised) and negative values, and on the first-order Tanimoto."""
    q, d, Sq, Sd = sets
    rng = np.random.default_rng(k)
    scores = np.round(rng.normal(0.3, 0.4, (q.n_mol, d.n_mol)), 2).astype(np.float32)
    sq = shp.self_overlaps(Sq, seed=1, n_samples=256)
    sd = shp.self_overlaps(Sd, seed=1, n_samples=256)
    T_fo = shp.fo_tanimoto_screen(Sq, Sd, sq[:, 0], sd[:, 0]).cpu().numpy().reshape(q.n_mol, d.n_mol)
    for S in (scores, T_fo):
        pq, pd = shp.fo_prefilter_select(Sq, Sd, torch.tensor(S.reshape(-1)), k)
        pq, pd = pq.cpu().numpy().reshape(q.n_mol, k), pd.cpu().numpy().reshape(q.n_mol, k)
        for i in range(q.n_mol):
            order = np.lexsort((np.arange(d.n_mol), -S[i].astype(np.float64)))[:k]  # value desc, id asc
            np.testing.assert_array_equal(pq[i], i)
            np.testing.assert_array_equal(pd[i], np.sort(order))


def test_prefilter_selection_rejects_bad_k(sets):
    q, d, Sq, Sd = sets
    T = torch.zeros(q.n_mol * d.n_mol, dtype=torch.float32, device="cuda")
    for k in (0, d.n_mol + 1):
        with pytest.raises(shp.ShapeError):
            shp.fo_prefilter_select(Sq, Sd, T, k)


def test_prefilter_full_size_sampled():
    """The benchmark's prefilter launch: 16 queries (20-48 atoms) x 1,000,000
    molecules (18-60, heavy-tailed toward 40). The first-order Tanimoto of
    512 sampled pairs against the oracle's closed form, and the best 10% per
    query (fo_prefilter_select) against a full sort of the same scores:
    exactly the k largest, ties at the k-th by the lowest id."""
    q, d = synth.adaptive_screen()
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    kq, kd = np.arange(q.n_mol), np.arange(d.n_mol)
    fq = O.fo_overlap(q, kq, q, kq)
    rng = np.random.default_rng(17)
    fd_gpu = shp.self_overlaps(Sd, seed=1, n_samples=256)[:, 0].contiguous()
    T = shp.fo_tanimoto_screen(Sq, Sd, torch.tensor(fq, device="cuda"), fd_gpu)
    pick = rng.choice(q.n_mol * d.n_mol, 512, replace=False)
    iq, idd = pick // d.n_mol, pick % d.n_mol
    O_ = O.fo_overlap(q, iq, d, idd)
    fd = O.fo_overlap(d, idd, d, idd)
    ref = O_ / (fq[iq] + fd - O_)
    np.testing.assert_allclose(T.cpu().numpy()[pick], ref, rtol=2e-5)
    k = d.n_mol // 10
    pq, pd = shp.fo_prefilter_select(Sq, Sd, T, k)
    S = T.view(q.n_mol, d.n_mol)
    # value descending, id ascending: a stable sort of the ids by -T
    order = torch.sort(-S, dim=1, stable=True).indices[:, :k]
    want = torch.sort(order.to(torch.int32), dim=1).values
    assert torch.equal(pq.view(q.n_mol, k), torch.arange(q.n_mol, dtype=torch.int32, device="cuda")[:, None]
                       .expand(q.n_mol, k))
    assert torch.equal(pd.view(q.n_mol, k), want)


def test_kept_molecules_get_the_whole_sets_values(sets):
    """prefilter_db_ids marks the kept database molecules; as an idx list with
    id-keyed streams the per-molecule estimators then give every kept
    molecule exactly the values of the call over the whole set (self-overlaps
    fixed and to a relative SE, least-squares weights), and skip the rest."""
    q, d, Sq, Sd = sets
    rng = np.random.default_rng(5)
    pd = torch.tensor(rng.choice(d.n_mol, 120), dtype=torch.int32, device="cuda")
    ids = shp.prefilter_db_ids(Sd, pd)
    keep = np.zeros(d.n_mol, bool)
    keep[pd.cpu().numpy()] = True
    want = np.where(keep, np.arange(d.n_mol), -1)
    np.testing.assert_array_equal(ids.cpu().numpy(), want)
    full = shp.self_overlaps(Sd, seed=3, n_samples=2048, stream_base=7)
    sub = shp.self_overlaps(Sd, seed=3, n_samples=2048, stream_base=7, idx=ids)
    np.testing.assert_array_equal(sub.cpu().numpy()[keep], full.cpu().numpy()[keep])
    assert np.all(np.isnan(sub.cpu().numpy()[~keep, 1]))
    fs, fse, fn = shp.self_overlaps(Sd, seed=3, n_samples=1 << 16, stream_base=7, target_rel_se=1e-2, with_se=True)
    ss, sse, sn = shp.self_overlaps(Sd, seed=3, n_samples=1 << 16, stream_base=7, target_rel_se=1e-2, with_se=True,
                                    idx=ids)
    for a, b in ((ss, fs), (sse, fse), (sn, fn)):
        np.testing.assert_array_equal(a.cpu().numpy()[keep], b.cpu().numpy()[keep])
    wf = shp.cv_fit_weights(Sd, seed=4, n_samples=1024)
    ws = shp.cv_fit_weights(Sd, seed=4, n_samples=1024, idx=ids, id_streams=True)
    atom_keep = np.repeat(keep, np.diff(d.offsets))
    np.testing.assert_array_equal(ws.cpu().numpy()[atom_keep], wf.cpu().numpy()[atom_keep])
    assert np.all(ws.cpu().numpy()[~atom_keep] == 0)
    # id-keyed streams apply to per-molecule calls only
    with pytest.raises(shp.ShapeError):
        shp.overlap_estimate(Sq, [0], Sd, [0], seed=1, n_samples=256, flags=shp.ID_STREAMS)


def test_hybrid_screen_keeps_the_full_screens_numbers(sets):
    """pipeline.hybrid_screen (first-order prefilter, union stage on the kept
    molecules only) against the unfiltered pipeline with the same seeds:
    every kept pair has the full screen's T, SE(T) and sample count bit for
    bit, the kept molecules' self-overlaps are the full call's, and each
    query keeps exactly its k best first-order pairs."""
    from paper_2607_20766_b300 import pipeline
    q, d, Sq, Sd = sets
    kw = dict(tau=0.01, cap=8192, min_n=512, round=256, self_rel_se=1e-2, fit_samples=1024)
    res = pipeline.hybrid_screen(Sq, Sd, 0.1, **kw)
    k = int(0.1 * d.n_mol)
    assert res["pairs_q"].numel() == q.n_mol * k
    sq, sq_se, _ = shp.self_overlaps(Sq, seed=11, n_samples=1 << 24, stream_base=0, target_rel_se=2.5e-3, round=4096,
                                     with_se=True)
    sd, sd_se, _ = shp.self_overlaps(Sd, seed=11, n_samples=1 << 22, stream_base=16, target_rel_se=1e-2, round=256,
                                     with_se=True)
    wq = shp.cv_fit_weights(Sq, seed=91, n_samples=1024)
    wd = shp.cv_fit_weights(Sd, seed=92, n_samples=1024)
    full = shp.tanimoto_screen(Sq, Sd, sq, sd, seed=77, tau=0.01, round=256, min_n=512, cap=8192, omega_q=wq,
                               omega_db=wd, self_se_q=sq_se, self_se_db=sd_se)
    flat = (res["pairs_q"].long() * d.n_mol + res["pairs_db"].long()).cpu().numpy()
    for key in ("T", "seT", "n_used"):
        np.testing.assert_array_equal(res[key].cpu().numpy(), full[key].cpu().numpy()[flat], err_msg=key)
    kept = res["ids"].cpu().numpy() >= 0
    np.testing.assert_array_equal(res["self_db"].cpu().numpy()[kept], sd.cpu().numpy()[kept])
    T_fo = res["T_fo"].view(q.n_mol, d.n_mol)
    kth = torch.sort(T_fo, dim=1, descending=True).values[:, k - 1]
    got = T_fo.gather(1, res["pairs_db"].view(q.n_mol, k).long())
    assert torch.all(got >= kth[:, None])


def test_fo_tanimoto_query_groups():
    """37 queries: two full groups of 16 per block and a ragged third, odd and
    even atom counts (the packed pairs' padding) from 1 to 64 atoms on both
    sides, against the oracle."""
    qc = np.concatenate([[1, 64, 63, 2], synth.counts_uniform(61, 33, 7, 48)]).astype(np.int32)
    dc = np.concatenate([synth.counts_heavy(62, 200), [1, 64, 2, 63]]).astype(np.int32)
    q = synth.principal_axes(synth.generate(61, qc))
    d = synth.principal_axes(synth.generate(62, dc))
    Sq, Sd = shp.shape_set_load(q), shp.shape_set_load(d)
    kq, kd = np.arange(q.n_mol), np.arange(d.n_mol)
    fq, fd = O.fo_overlap(q, kq, q, kq), O.fo_overlap(d, kd, d, kd)
    T = shp.fo_tanimoto_screen(Sq, Sd, torch.tensor(fq), torch.tensor(fd)).cpu().numpy()
    iq, idd = np.meshgrid(kq, kd, indexing="ij")
    O_ = O.fo_overlap(q, iq.ravel(), d, idd.ravel())
    np.testing.assert_allclose(T, O_ / (fq[iq.ravel()] + fd[idd.ravel()] - O_), rtol=2e-5)
    assert np.any(q.counts % 2 == 1) and np.any(q.counts % 2 == 0)
