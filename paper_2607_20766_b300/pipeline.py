"""The paper's hybrid screening pipeline as one call (Sec. hybrid pipeline):
the closed-form first-order Tanimoto ranks every (query, database) pair, each
query keeps its best fraction, and only the kept pairs go through the
union-Tanimoto estimator, with the union stage's per-molecule work (the
self-overlaps to a stated precision and the control-variate weights)
restricted to the database molecules some query keeps.

Every step is a library call (kernels in ``libshape.so``); this module only
sequences them. The random streams are keyed by molecule and pair ids
(``id_streams`` for the kept molecules), so every kept pair gets exactly the
numbers the unfiltered screen with the same seeds gives it."""
from __future__ import annotations

import torch

from . import _binding as B


# Relative SE of the kept database molecules' union self-overlaps. Each kept
# molecule serves few pairs (1.6-4.4 at 5-25% kept of 16 queries), so a
# looser self-overlap costs fewer samples than the longer pair runs it
# causes under the full delta-method SE(T) (16 x 1M, tau 0.005: 5.5e-3 took
# the 5% / 10% / 25% pipelines from 0.48 / 0.78 / 1.41 s at 3.5e-3 to
# 0.40 / 0.67 / 1.30 s; 7e-3 was slower again).
DEFAULT_SELF_REL_SE = 5.5e-3


def hybrid_screen(Q: B.ShapeSet, D: B.ShapeSet, keep: float, tau: float = 0.005, cap: int = 65536,
                  min_n: int = 1024, round: int = 256, self_rel_se: float = DEFAULT_SELF_REL_SE,
                  fit_samples: int = 4096,
                  control_variate: bool = True, seed: int = 77, self_seed: int = 11, self_base_q: int = 0,
                  self_base_db: int = 16, fit_seed_q: int = 91, fit_seed_db: int = 92, stream=None) -> dict:
    """Screen every query of Q against D through the first-order prefilter.

    keep: fraction of D each query keeps (at least one molecule). The kept
    pairs are screened adaptively (union SE(T) <= tau, full delta-method SE
    with the self-overlaps' own errors; rounds of `round`, min_n to cap per
    direction), with the least-squares control variate when
    control_variate. Self-overlaps: database molecules to relative SE
    self_rel_se, queries to a quarter of it (on a side stream), caps 2^22 and
    2^24 samples. Returns a dict with pairs_q, pairs_db (int32 [n_q * k], per
    query ascending database id), T, seT ([n_q * k, 2]), n_used, the
    first-order scores T_fo ([n_q * n_db]), the kept-molecule idx list ids
    ([n_db], -1 where no query keeps the molecule), and self_q, self_db with
    their SEs (NaN rows for molecules not kept)."""
    if not 0.0 < keep <= 1.0:
        raise ValueError("keep must be in (0, 1]")
    main = stream if stream is not None else torch.cuda.current_stream()
    dev = Q.device
    k = max(1, int(keep * D.n_mol))
    iq = torch.arange(Q.n_mol, dtype=torch.int32, device=dev)
    idb = torch.arange(D.n_mol, dtype=torch.int32, device=dev)
    side = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(main):
        fo_q = B.fo_overlap(Q, iq, Q, iq)
        fo_d = B.fo_overlap(D, idb, D, idb)
        T_fo = B.fo_tanimoto_screen(Q, D, fo_q, fo_d)
        pq, pd = B.fo_prefilter_select(Q, D, T_fo, k)
        ids = B.prefilter_db_ids(D, pd)
        side.wait_stream(main)
        with torch.cuda.stream(side):
            sq, sq_se, _ = B.self_overlaps(Q, seed=self_seed, n_samples=1 << 24, stream_base=self_base_q,
                                           target_rel_se=self_rel_se / 4, round=4096, with_se=True)
            wq = B.cv_fit_weights(Q, seed=fit_seed_q, n_samples=fit_samples) if control_variate else None
        sd, sd_se, _ = B.self_overlaps(D, seed=self_seed, n_samples=1 << 22, stream_base=self_base_db,
                                       target_rel_se=self_rel_se, round=round, with_se=True, idx=ids)
        wd = (B.cv_fit_weights(D, seed=fit_seed_db, n_samples=fit_samples, idx=ids, id_streams=True)
              if control_variate else None)
        main.wait_stream(side)
        for t in (sq, sq_se, wq):
            if t is not None:
                t.record_stream(main)
        res = B.tanimoto_screen(Q, D, sq, sd, seed=seed, tau=tau, round=round, min_n=min_n, cap=cap,
                                omega_q=wq, omega_db=wd, pairs=(pq, pd), self_se_q=sq_se, self_se_db=sd_se)
    res.update(pairs_q=pq, pairs_db=pd, T_fo=T_fo, ids=ids, self_q=sq, self_db=sd, self_se_q=sq_se,
               self_se_db=sd_se)
    return res
