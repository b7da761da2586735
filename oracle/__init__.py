"""FP64 CPU oracle for the importance-sampling shape-overlap estimator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package. It
shares no code with the CUDA library (its C source ``oracle.c`` is written
independently from the paper's equations and the written stream/sampler
conventions listed at the top of that file).

Pins (``tests/test_oracle_*.py``): Philox words against an independent
Philox4x32-10 (Triton's CPU interpreter), alias-table mass invariants and
pick frequencies, sampler moments, the first-order closed form (Eq. fo),
hard-sphere single-atom volumes (Eq. occ with lambda = 1 and its p = 2 sqrt 2
counterpart), full inclusion-exclusion (Eq. incexc) against grid quadrature,
and the IS estimators within 3 SE of those exact values.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

SYMMETRIC = 1
ANTITHETIC = 2
TAG_AB, TAG_BA, TAG_SELF = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile liboracle.so (gcc, -O2, OpenMP, strict IEEE double)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Set(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("radius", ctypes.c_void_p), ("height", ctypes.c_void_p),
                ("offsets", ctypes.c_void_p), ("n_mol", ctypes.c_int32), ("c_alpha", ctypes.c_double)]


_P = ctypes.c_void_p
_SIGS = {
    "orc_philox4x32_10": [_P, _P, _P],
    "orc_normal_pair": [ctypes.c_uint32, ctypes.c_uint32, _P],
    "orc_alias_build": [ctypes.c_int, _P, _P, _P, _P],
    "orc_mol_tables": [_P, ctypes.c_int32, _P, _P, _P, _P, _P],
    "orc_draw": [_P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                 ctypes.c_int64, ctypes.c_int, _P, _P],
    "orc_occupancy": [_P, ctypes.c_int32, _P, ctypes.c_int64, _P, _P, _P],
    "orc_direction_sums": [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_uint64,
                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _P, _P],
    "orc_overlap_estimate": [_P, _P, _P, _P, ctypes.c_int64, _P, ctypes.c_uint64, ctypes.c_uint64,
                             ctypes.c_uint32, ctypes.c_uint32, _P, _P, ctypes.c_int],
    "orc_union_volume_estimate": [_P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                                  ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P, _P, ctypes.c_int],
    "orc_fo_overlap": [_P, _P, _P, _P, ctypes.c_int64, _P, _P, ctypes.c_int],
    "orc_mixture_mass": [_P, _P, ctypes.c_int64, _P],
    "orc_union_volume_ie": [_P, ctypes.c_int32, _P],
    "orc_union_overlap_ie": [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, ctypes.c_int],
    "orc_grid": [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_double, ctypes.c_double, _P,
                 ctypes.c_int],
    "orc_tanimoto_pairs": [_P, _P, _P, _P, _P, ctypes.c_int64, _P, _P, _P, _P, ctypes.c_uint64,
                           ctypes.c_uint32, ctypes.c_uint32, _P, _P, _P, _P, _P, _P, ctypes.c_int],
    "orc_crn_points": [_P, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _P],
    "orc_pose_objective": [ctypes.c_double, _P, ctypes.c_uint32, _P, ctypes.c_int32, _P, ctypes.c_int, _P],
    "orc_pose_grad_fd": [ctypes.c_double, _P, ctypes.c_uint32, _P, ctypes.c_int32, _P, ctypes.c_int,
                         ctypes.c_double, _P, _P],
    "orc_fo_pose_grad": [_P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P],
    "orc_attributions": [_P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, ctypes.c_int],
    "orc_cv_fit_weights": [_P, _P, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                           _P, ctypes.c_int],
    "orc_union_volume_cv": [_P, _P, ctypes.c_int64, _P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P,
                            ctypes.c_int],
    "orc_cv_features": [_P, _P],
    "orc_union_self_cv": [_P, _P, ctypes.c_int64, _P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P, _P,
                          _P, ctypes.c_int],
}


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int if name != "orc_philox4x32_10" else None
        L.orc_normal_pair.restype = None
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"{what} failed with status {rc}")


class OSet:
    """Keeps host arrays of a molecule set alive for the C oracle."""

    def __init__(self, ms, c_alpha: float = 2.41798793):
        self.xyz = np.ascontiguousarray(ms.xyz, dtype=np.float32)
        self.radius = np.ascontiguousarray(ms.radius, dtype=np.float32)
        self.height = None if ms.height is None else np.ascontiguousarray(ms.height, dtype=np.float32)
        self.offsets = np.ascontiguousarray(ms.offsets, dtype=np.int32)
        self.s = _Set(self.xyz.ctypes.data, self.radius.ctypes.data, _ptr(self.height),
                      self.offsets.ctypes.data, len(self.offsets) - 1, c_alpha)

    @property
    def ref(self):
        return ctypes.byref(self.s)

    @property
    def n_mol(self):
        return len(self.offsets) - 1


def _oset(ms, c_alpha=2.41798793):
    return ms if isinstance(ms, OSet) else OSet(ms, c_alpha)


# ---------------------------------------------------------------- primitives

def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def normal_pair(a: int, b: int) -> np.ndarray:
    out = np.empty(2, dtype=np.float64)
    lib().orc_normal_pair(a, b, out.ctypes.data)
    return out


def alias_build(v):
    v = np.ascontiguousarray(v, dtype=np.float64)
    n = len(v)
    thr = np.empty(n, np.uint32)
    al = np.empty(n, np.uint8)
    mass = np.empty(n, np.uint64)
    _check(lib().orc_alias_build(n, v.ctypes.data, thr.ctypes.data, al.ctypes.data, mass.ctypes.data),
           "alias_build")
    return thr, al, mass


def mol_tables(ms, idx, c_alpha=2.41798793):
    s = _oset(ms, c_alpha)
    n = int(s.offsets[idx + 1] - s.offsets[idx])
    alpha, v = np.empty(n), np.empty(n)
    Z = ctypes.c_double()
    thr, al = np.empty(n, np.uint32), np.empty(n, np.uint8)
    _check(lib().orc_mol_tables(s.ref, idx, alpha.ctypes.data, v.ctypes.data, ctypes.addressof(Z),
                                thr.ctypes.data, al.ctypes.data), "mol_tables")
    return dict(alpha=alpha, v=v, Z=Z.value, thr=thr, alias=al)


def draw(ms, idx, seed, stream, tag, n, antithetic=False, c_alpha=2.41798793):
    s = _oset(ms, c_alpha)
    r = np.empty((n, 3))
    comp = np.empty(n, np.int32)
    _check(lib().orc_draw(s.ref, idx, seed, stream, tag, n, int(antithetic), r.ctypes.data,
                          comp.ctypes.data), "draw")
    return r, comp


def occupancy(ms, idx, r, pose=None, c_alpha=2.41798793):
    s = _oset(ms, c_alpha)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = len(r)
    m, u = np.empty(n), np.empty(n)
    p = None if pose is None else np.ascontiguousarray(pose, dtype=np.float32)
    _check(lib().orc_occupancy(s.ref, idx, _ptr(p), n, r.ctypes.data, m.ctypes.data, u.ctypes.data),
           "occupancy")
    return m, u


def direction_sums(A, ia, B, ib, seed, stream, tag, n, flags=0, poseB=None, c_alpha=2.41798793):
    sa, sb = _oset(A, c_alpha), _oset(B, c_alpha)
    sums = np.empty(4)
    ne = ctypes.c_double()
    p = None if poseB is None else np.ascontiguousarray(poseB, dtype=np.float32)
    _check(lib().orc_direction_sums(sa.ref, ia, sb.ref, ib, _ptr(p), seed, stream, tag, n, flags,
                                    sums.ctypes.data, ctypes.addressof(ne)), "direction_sums")
    return sums, ne.value


# ---------------------------------------------------------------- estimators

def overlap_estimate(A, ia, B, ib, seed, n, flags=SYMMETRIC, stream_base=0, poses=None,
                     n_threads=0, c_alpha=2.41798793):
    """est[n_pairs, 2], se[n_pairs, 2]: slot 0 first order, slot 1 union."""
    sa, sb = _oset(A, c_alpha), _oset(B, c_alpha)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    npairs = len(ia)
    est, se = np.empty((npairs, 2)), np.empty((npairs, 2))
    p = None if poses is None else np.ascontiguousarray(poses, dtype=np.float32)
    _check(lib().orc_overlap_estimate(sa.ref, ia.ctypes.data, sb.ref, ib.ctypes.data, npairs, _ptr(p),
                                      seed, stream_base, n, flags, est.ctypes.data, se.ctypes.data,
                                      n_threads), "overlap_estimate")
    return est, se


def union_volume_estimate(S, idx, seed, n, flags=0, stream_base=0, n_threads=0, c_alpha=2.41798793):
    """(vol, vol_se, self_overlap, self_se), each [len(idx)]."""
    s = _oset(S, c_alpha)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    k = len(idx)
    v, vs, so, ss = np.empty(k), np.empty(k), np.empty(k), np.empty(k)
    _check(lib().orc_union_volume_estimate(s.ref, idx.ctypes.data, k, seed, stream_base, n, flags,
                                           v.ctypes.data, vs.ctypes.data, so.ctypes.data,
                                           ss.ctypes.data, n_threads), "union_volume_estimate")
    return v, vs, so, ss


def fo_overlap(A, ia, B, ib, poses=None, n_threads=0, c_alpha=2.41798793):
    sa, sb = _oset(A, c_alpha), _oset(B, c_alpha)
    ia = np.ascontiguousarray(ia, dtype=np.int32)
    ib = np.ascontiguousarray(ib, dtype=np.int32)
    out = np.empty(len(ia))
    p = None if poses is None else np.ascontiguousarray(poses, dtype=np.float32)
    _check(lib().orc_fo_overlap(sa.ref, ia.ctypes.data, sb.ref, ib.ctypes.data, len(ia), _ptr(p),
                                out.ctypes.data, n_threads), "fo_overlap")
    return out


def mixture_mass(S, idx=None, c_alpha=2.41798793):
    s = _oset(S, c_alpha)
    if idx is None:
        idx = np.arange(s.n_mol)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    Z = np.empty(len(idx))
    _check(lib().orc_mixture_mass(s.ref, idx.ctypes.data, len(idx), Z.ctypes.data), "mixture_mass")
    return Z


def union_volume_ie(S, idx=0, c_alpha=2.41798793) -> float:
    s = _oset(S, c_alpha)
    V = ctypes.c_double()
    _check(lib().orc_union_volume_ie(s.ref, idx, ctypes.addressof(V)), "union_volume_ie")
    return V.value


def union_overlap_ie(A, ia, B, ib, poseB=None, n_threads=0, c_alpha=2.41798793) -> float:
    sa, sb = _oset(A, c_alpha), _oset(B, c_alpha)
    O = ctypes.c_double()
    p = None if poseB is None else np.ascontiguousarray(poseB, dtype=np.float32)
    _check(lib().orc_union_overlap_ie(sa.ref, ia, sb.ref, ib, _ptr(p), ctypes.addressof(O), n_threads),
           "union_overlap_ie")
    return O.value


def grid(A, ia, B=None, ib=0, h=0.1, pad=6.5, poseB=None, n_threads=0, c_alpha=2.41798793):
    """dict(VA, VB, OU, OFO, ZA, SA) from midpoint quadrature (spacing h)."""
    sa = _oset(A, c_alpha)
    sb = None if B is None else _oset(B, c_alpha)
    out = np.empty(6)
    p = None if poseB is None else np.ascontiguousarray(poseB, dtype=np.float32)
    _check(lib().orc_grid(sa.ref, ia, None if sb is None else sb.ref, ib, _ptr(p), h, pad,
                          out.ctypes.data, n_threads), "grid")
    return dict(VA=out[0], VB=out[1], OU=out[2], OFO=out[3], ZA=out[4], SA=out[5])


def tanimoto_pairs(Q, iq, D, idd, stream_ids, selfQ, selfD, seed, n, flags=0, n_threads=0,
                   c_alpha=2.41798793, omega_q=None, omega_d=None, selfQ_se=None, selfD_se=None):
    """Fixed-budget symmetric screen of explicit pairs. Returns dict of
    [n_pairs, 2] arrays O, seO, T, seT (slot 0 first order, slot 1 union).
    omega_q/omega_d (per set atom): control-variate weights of the union slot.
    selfQ_se/selfD_se (like selfQ/selfD): standard errors of the
    self-overlaps; seT is then the full delta-method SE of T."""
    sq, sd = _oset(Q, c_alpha), _oset(D, c_alpha)
    if (omega_q is None) != (omega_d is None):
        raise ValueError("give both omega_q and omega_d or neither")
    if (selfQ_se is None) != (selfD_se is None):
        raise ValueError("give both selfQ_se and selfD_se or neither")
    eq = None if selfQ_se is None else np.ascontiguousarray(selfQ_se, dtype=np.float64)
    ed = None if selfD_se is None else np.ascontiguousarray(selfD_se, dtype=np.float64)
    wq = None if omega_q is None else np.ascontiguousarray(omega_q, dtype=np.float64)
    wd = None if omega_d is None else np.ascontiguousarray(omega_d, dtype=np.float64)
    iq = np.ascontiguousarray(iq, dtype=np.int32)
    idd = np.ascontiguousarray(idd, dtype=np.int32)
    st = np.ascontiguousarray(stream_ids, dtype=np.uint64)
    selfQ = np.ascontiguousarray(selfQ, dtype=np.float64)
    selfD = np.ascontiguousarray(selfD, dtype=np.float64)
    k = len(iq)
    O, sO, T, sT = (np.empty((k, 2)) for _ in range(4))
    _check(lib().orc_tanimoto_pairs(sq.ref, iq.ctypes.data, sd.ref, idd.ctypes.data, st.ctypes.data, k,
                                    selfQ.ctypes.data, selfD.ctypes.data, _ptr(eq), _ptr(ed), seed, n, flags,
                                    _ptr(wq), _ptr(wd),
                                    O.ctypes.data, sO.ctypes.data, T.ctypes.data, sT.ctypes.data, n_threads),
           "tanimoto_pairs")
    return dict(O=O, seO=sO, T=T, seT=sT)


# ---------------------------------------------------------------- alignment

TAG_CRN = 3
OBJ_FO, OBJ_UNION = 0, 1


def crn_points(Q, iq, seed, stream, n, c_alpha=2.41798793, antithetic=False):
    """[n, 4] float64: CRN points drawn from Q[iq] (tag 3) and their union
    weights u/m; antithetic: each odd point reflects the even one about its
    component centre."""
    s = _oset(Q, c_alpha)
    pts = np.empty((n, 4))
    _check(lib().orc_crn_points(s.ref, iq, seed, stream, n, int(antithetic), pts.ctypes.data), "crn_points")
    return pts


def pose_objective(ZQ, points, B, ib, pose, objective=OBJ_UNION, c_alpha=2.41798793):
    sb = _oset(B, c_alpha)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    p = np.ascontiguousarray(pose, dtype=np.float32)
    F = ctypes.c_double()
    _check(lib().orc_pose_objective(ZQ, pts.ctypes.data, len(pts), sb.ref, ib, p.ctypes.data, objective,
                                    ctypes.addressof(F)), "pose_objective")
    return F.value


def pose_grad_fd(ZQ, points, B, ib, pose, objective=OBJ_UNION, h=1e-3, c_alpha=2.41798793):
    """(F, dF/dpose[7]) with central differences of step h in the raw pose."""
    sb = _oset(B, c_alpha)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    p = np.ascontiguousarray(pose, dtype=np.float64)
    F = ctypes.c_double()
    g = np.empty(7)
    _check(lib().orc_pose_grad_fd(ZQ, pts.ctypes.data, len(pts), sb.ref, ib, p.ctypes.data, objective, h,
                                  ctypes.addressof(F), g.ctypes.data), "pose_grad_fd")
    return F.value, g


def fo_pose_grad(A, ia, B, ib, pose, c_alpha=2.41798793):
    """(O_fo, dO_fo/dpose[7]): closed form (Eq. fo) and its analytic gradient."""
    sa, sb = _oset(A, c_alpha), _oset(B, c_alpha)
    p = np.ascontiguousarray(pose, dtype=np.float64)
    F = ctypes.c_double()
    g = np.empty(7)
    _check(lib().orc_fo_pose_grad(sa.ref, ia, sb.ref, ib, p.ctypes.data, ctypes.addressof(F), g.ctypes.data),
           "fo_pose_grad")
    return F.value, g


# ---------------------------------------------------------------- control variate

TAG_ATTR = 5


def attributions(S, idx, seed, M, stream_base=0, n_threads=0, c_alpha=2.41798793):
    """Union attributions omega*_i = E_{N(c_i, 1/(2 alpha_i))}[u/m], M samples per
    atom; concatenated over idx (atom order)."""
    s = _oset(S, c_alpha)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n_at = int(sum(s.offsets[i + 1] - s.offsets[i] for i in idx))
    out = np.empty(n_at)
    _check(lib().orc_attributions(s.ref, idx.ctypes.data, len(idx), seed, stream_base, M, out.ctypes.data, n_threads),
           "attributions")
    return out


def union_volume_cv(S, idx, omega, seed, n, stream_base=0, n_threads=0, c_alpha=2.41798793):
    """(vol, vol_se) with the weighted-Gaussian control variate; omega per set atom."""
    s = _oset(S, c_alpha)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    om = np.ascontiguousarray(omega, dtype=np.float64)
    v, vs = np.empty(len(idx)), np.empty(len(idx))
    _check(lib().orc_union_volume_cv(s.ref, idx.ctypes.data, len(idx), om.ctypes.data, seed, stream_base, n,
                                     v.ctypes.data, vs.ctypes.data, n_threads), "union_volume_cv")
    return v, vs


def union_self_cv(S, idx, omega, seed, n, stream_base=0, n_threads=0, c_alpha=2.41798793):
    """(vol, vol_se, self_ov, self_se), each [len(idx)]: union volumes and
    union self-overlaps with the weighted-Gaussian control variate omega (per
    set atom; None = the plain estimators), n samples per molecule (tag 2)."""
    s = _oset(S, c_alpha)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    om = None if omega is None else np.ascontiguousarray(omega, dtype=np.float64)
    k = len(idx)
    v, vs, so, ss = (np.empty(k) for _ in range(4))
    _check(lib().orc_union_self_cv(s.ref, idx.ctypes.data, k, _ptr(om), seed, stream_base, n, v.ctypes.data,
                                   vs.ctypes.data, so.ctypes.data, ss.ctypes.data, n_threads), "union_self_cv")
    return v, vs, so, ss


def cv_fit_weights(S, idx, seed, n, stream_base=0, ridge=1e-6, n_threads=0, c_alpha=2.41798793):
    """[n_atoms] float64: least-squares control-variate weights of the listed
    molecules (other atoms 0): the projection of u onto the molecule's own
    Gaussians, with b estimated from n samples (tag 6)."""
    s = _oset(S, c_alpha)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    om = np.zeros(int(s.offsets[-1]))
    _check(lib().orc_cv_fit_weights(s.ref, idx.ctypes.data, len(idx), seed, stream_base, n, ridge, om.ctypes.data,
                                    n_threads), "cv_fit_weights")
    return om


def cv_features(S, c_alpha=2.41798793):
    """[n_atoms, 33] float64: 16-nearest-neighbour (d/4, R/1.7) pairs and own R/1.7."""
    s = _oset(S, c_alpha)
    out = np.empty((int(s.offsets[-1]), 33))
    _check(lib().orc_cv_features(s.ref, out.ctypes.data), "cv_features")
    return out
