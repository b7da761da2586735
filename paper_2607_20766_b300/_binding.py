"""ctypes binding of libshape.so (argument marshalling only).

Every computation runs in the library's CUDA kernels; torch provides device
memory and the current stream. There is no CPU fallback: without the built
library or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes
import functools
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libshape.so")

SHP_OK = 0
SYMMETRIC = 1
ANTITHETIC = 2
ID_STREAMS = 4  # idx lists: molecule idx[k] draws from stream stream_base + idx[k]
TAG_AB, TAG_BA, TAG_SELF = 0, 1, 2
MAX_ATOMS = 64

# Every entry point declared in include/shape.h.
EXPORTS = ("shp_last_error", "shp_version", "shp_fail_next_allocations", "shape_set_load", "shape_set_free", "shape_set_free_async", "shape_set_info",
           "shape_set_tables", "overlap_estimate", "union_volume_estimate", "fo_overlap",
           "tanimoto_screen", "shp_screen_variants", "shp_screen_variant_info", "tanimoto_screen_tune", "align_crn_points",
           "overlap_pose_grad", "align_rigid", "shape_set_frames", "union_attributions", "union_volume_cv",
           "cv_features", "mlp_forward", "mlp_loss_grad", "mlp_adam", "mlp_loss_grad_noalloc", "cv_fit_weights",
           "union_self_estimate", "shp_eval_probe", "fo_tanimoto_screen",
           "fo_prefilter_select", "prefilter_db_ids", "mlp_train_epoch")
MLP_IN, MLP_HIDDEN, MLP_PARAMS = 33, 64, 6401
OBJ_FO, OBJ_UNION, OBJ_FO_CLOSED = 0, 1, 2

_P = ctypes.c_void_p


class ShpMC(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("stream_base", ctypes.c_uint64), ("n_samples", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]


class ShpScreen(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("stream_base", ctypes.c_uint64), ("n_fixed", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("tau", ctypes.c_float), ("round", ctypes.c_uint32),
                ("min_n", ctypes.c_uint32), ("cap", ctypes.c_uint32), ("watch", ctypes.c_uint32),
                ("variant", ctypes.c_int32), ("omega_q", ctypes.c_void_p), ("omega_db", ctypes.c_void_p),
                ("self_se_q", ctypes.c_void_p), ("self_se_db", ctypes.c_void_p), ("stream_stride", ctypes.c_uint64),
                ("pairs_q", ctypes.c_void_p), ("pairs_db", ctypes.c_void_p), ("n_pairs", ctypes.c_int64)]


class ShpAlign(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_uint64), ("stream", ctypes.c_uint64), ("starts", ctypes.c_uint32),
                ("steps", ctypes.c_uint32), ("n_crn", ctypes.c_uint32), ("objective", ctypes.c_uint32),
                ("lr", ctypes.c_float), ("lr_t", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("n_score", ctypes.c_uint32),
                ("crn_flags", ctypes.c_uint32)]


_lib = None


def load_library():
    """Load libshape.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2607_20766_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    L.shp_last_error.restype = ctypes.c_char_p
    L.shp_last_error.argtypes = []
    L.shp_version.restype = ctypes.c_int
    sig = {
        "shape_set_load": [_P, _P, _P, ctypes.c_double, _P, ctypes.c_int32, _P, _P],
        "shp_fail_next_allocations": [ctypes.c_int32],
        "shape_set_free": [_P],
        "shape_set_free_async": [_P, _P],
        "shape_set_info": [_P, _P, _P, _P],
        "shape_set_tables": [_P, _P, _P, _P],
        "overlap_estimate": [_P, _P, _P, _P, ctypes.c_int64, _P, _P, _P, _P, _P],
        "union_volume_estimate": [_P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P],
        "fo_overlap": [_P, _P, _P, _P, ctypes.c_int64, _P, _P, _P],
        "tanimoto_screen": [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P],
        "shp_screen_variants": [],
        "shp_screen_variant_info": [ctypes.c_int32, _P],
        "tanimoto_screen_tune": [_P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int64, _P, _P, _P],
        "align_crn_points": [_P, ctypes.c_int32, _P, _P, _P],
        "overlap_pose_grad": [_P, ctypes.c_int32, _P, ctypes.c_uint32, _P, _P, ctypes.c_int64, _P, ctypes.c_uint32,
                              _P, _P, _P],
        "align_rigid": [_P, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P, _P, _P, _P, _P, _P, _P],
        "shape_set_frames": [_P, _P],
        "union_attributions": [_P, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32, _P, _P],
        "union_volume_cv": [_P, _P, ctypes.c_int64, _P, _P, ctypes.c_float, ctypes.c_uint32, _P, _P, _P, _P],
        "cv_features": [_P, _P, _P],
        "fo_tanimoto_screen": [_P, _P, _P, _P, _P, _P],
        "fo_prefilter_select": [_P, _P, _P, ctypes.c_int64, _P, _P, _P],
        "prefilter_db_ids": [_P, _P, ctypes.c_int64, _P, _P],
        "shp_eval_probe": [_P, ctypes.c_int32, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, _P,
                           _P, _P],
        "union_self_estimate": [_P, _P, ctypes.c_int64, _P, _P, ctypes.c_float, ctypes.c_uint32, ctypes.c_uint32, _P,
                                _P, _P, _P, _P, _P],
        "cv_fit_weights": [_P, _P, ctypes.c_int64, _P, ctypes.c_float, _P, _P],
        "mlp_forward": [_P, _P, _P, ctypes.c_int64, _P, _P],
        "mlp_loss_grad": [_P, _P, _P, _P, ctypes.c_int64, _P, _P, _P],
        "mlp_loss_grad_noalloc": [_P, _P, _P, _P, ctypes.c_int64, _P, _P, _P],
        "mlp_adam": [_P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                     ctypes.c_float, _P],
        "mlp_train_epoch": [_P, _P, _P, _P, _P, _P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, ctypes.c_float, _P, _P],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    _lib = L
    return L


class ShapeError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libshape status {status}: {msg}")
        self.status = status


def _check(rc: int):
    if rc != SHP_OK:
        raise ShapeError(rc, load_library().shp_last_error().decode())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dptr(t):
    return None if t is None else t.data_ptr()


def _on_stream(fn):
    """Run a wrapper with its `stream` argument (a torch.cuda.Stream) as the
    current stream, so that the device temporaries it creates (index and
    argument tensors made contiguous, outputs) are allocated on, and ordered
    with, the stream the library call is queued on. A raw cudaStream_t
    handle (an int) is passed through unchanged."""
    @functools.wraps(fn)
    def wrapped(*args, stream=None, **kwargs):
        if isinstance(stream, torch.cuda.Stream):
            with torch.cuda.stream(stream):
                return fn(*args, stream=stream, **kwargs)
        return fn(*args, stream=stream, **kwargs)
    return wrapped


def _device_i32(x, device) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        t = x.to(device=device, dtype=torch.int32)
    else:
        t = torch.as_tensor(np.asarray(x, dtype=np.int32), device=device)
    return t.contiguous()


class ShapeSet:
    """A molecule set resident in device memory (opaque shp_set handle)."""

    def __init__(self, handle: int, n_mol: int, n_atoms: int, counts: np.ndarray, device: torch.device):
        self.handle = ctypes.c_void_p(handle)
        self.n_mol = n_mol
        self.n_atoms = n_atoms
        self.counts = counts
        self.device = device

    def tables(self):
        """Host copies: (Z [n_mol] float64, thr [n_atoms] uint32, alias [n_atoms] uint8)."""
        Z = np.empty(self.n_mol, np.float64)
        thr = np.empty(self.n_atoms, np.uint32)
        al = np.empty(self.n_atoms, np.uint8)
        _check(load_library().shape_set_tables(self.handle, Z.ctypes.data, thr.ctypes.data, al.ctypes.data))
        return Z, thr, al

    def frames(self):
        """Host copy of the principal frames, [n_mol, 12] float32 (centroid, axes row-major)."""
        out = np.empty((self.n_mol, 12), np.float32)
        _check(load_library().shape_set_frames(self.handle, out.ctypes.data))
        return out

    def free(self, stream=None):
        """Release the device memory: synchronously, or in stream order on
        `stream` (no other stream may still use the set)."""
        if self.handle is not None and self.handle.value:
            if stream is None:
                load_library().shape_set_free(self.handle)
            else:
                load_library().shape_set_free_async(self.handle, _stream(stream))
        self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def shape_set_load(ms, c_alpha: float = 2.41798793, stream=None, device=None) -> ShapeSet:
    """Upload a MolSet (host arrays) to the current CUDA device, in order on
    `stream` (default: the current stream); returns once the host arrays
    have been consumed."""
    if not torch.cuda.is_available():
        raise RuntimeError("shape_set_load needs a CUDA device")
    L = load_library()
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    xyz = np.ascontiguousarray(ms.xyz, dtype=np.float32)
    rad = np.ascontiguousarray(ms.radius, dtype=np.float32)
    hgt = None if ms.height is None else np.ascontiguousarray(ms.height, dtype=np.float32)
    off = np.ascontiguousarray(ms.offsets, dtype=np.int32)
    h = ctypes.c_void_p()
    with torch.cuda.device(device):
        _check(L.shape_set_load(xyz.ctypes.data, rad.ctypes.data, None if hgt is None else hgt.ctypes.data,
                                c_alpha, off.ctypes.data, len(off) - 1, _stream(stream), ctypes.byref(h)))
    return ShapeSet(h.value, len(off) - 1, int(off[-1]), np.diff(off).astype(np.int32), device)


@_on_stream
def overlap_estimate(A: ShapeSet, ia, B: ShapeSet, ib, seed: int, n_samples: int, flags: int = SYMMETRIC,
                     stream_base: int = 0, pose=None, stream=None, out=None):
    """(est, se): [n_pairs, 2] float64 device tensors; slot 0 first order, slot 1 union."""
    dev = A.device
    ia = _device_i32(ia, dev)
    ib = _device_i32(ib, dev)
    n = ia.numel()
    if ib.numel() != n:
        raise ValueError("ia and ib differ in length")
    if pose is not None:
        pose = torch.as_tensor(pose, dtype=torch.float32, device=dev).contiguous()
        if pose.shape != (n, 7):
            raise ValueError("pose must be [n_pairs, 7]")
    est, se = out if out is not None else (torch.empty((n, 2), dtype=torch.float64, device=dev),
                                           torch.empty((n, 2), dtype=torch.float64, device=dev))
    mc = ShpMC(seed, stream_base, n_samples, flags)
    _check(load_library().overlap_estimate(A.handle, _dptr(ia), B.handle, _dptr(ib), n, _dptr(pose),
                                           ctypes.byref(mc), _dptr(est), _dptr(se), _stream(stream)))
    return est, se


@_on_stream
def union_volume_estimate(S: ShapeSet, idx=None, seed: int = 0, n_samples: int = 4096, flags: int = 0,
                          stream_base: int = 0, stream=None, out=None):
    """(vol, vol_se, self_overlap, self_se): [n] float64 device tensors."""
    dev = S.device
    if idx is not None:
        idx = _device_i32(idx, dev)
        n = idx.numel()
    else:
        n = S.n_mol
    outs = out if out is not None else tuple(torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4))
    mc = ShpMC(seed, stream_base, n_samples, flags)
    _check(load_library().union_volume_estimate(S.handle, _dptr(idx), n, ctypes.byref(mc), *(_dptr(t) for t in outs),
                                                _stream(stream)))
    return outs


@_on_stream
def fo_overlap(A: ShapeSet, ia, B: ShapeSet, ib, pose=None, stream=None, out=None):
    """Closed-form first-order overlaps, [n_pairs] float64 device tensor."""
    dev = A.device
    ia = _device_i32(ia, dev)
    ib = _device_i32(ib, dev)
    n = ia.numel()
    if pose is not None:
        pose = torch.as_tensor(pose, dtype=torch.float32, device=dev).contiguous()
    res = out if out is not None else torch.empty(n, dtype=torch.float64, device=dev)
    _check(load_library().fo_overlap(A.handle, _dptr(ia), B.handle, _dptr(ib), n, _dptr(pose), _dptr(res),
                                     _stream(stream)))
    return res


def screen_config(seed: int, n_fixed: int = 0, tau: float = 0.005, round: int = 256, min_n: int = 1024,
                  cap: int = 65536, watch: int = 1, flags: int = 0, stream_base: int = 0,
                  variant: int = -1, omega_q: torch.Tensor | None = None,
                  omega_db: torch.Tensor | None = None, self_se_q: torch.Tensor | None = None,
                  self_se_db: torch.Tensor | None = None, stream_stride: int = 0,
                  pairs_q: torch.Tensor | None = None, pairs_db: torch.Tensor | None = None) -> ShpScreen:
    """A shp_screen: fixed budget when n_fixed > 0, else adaptive (tau, round, min_n, cap, watch);
    omega_q/omega_db (float32 device, per set atom): control variate of the union slot;
    self_se_q/self_se_db (float64 device, [n, 2]): SEs of the self-overlaps (full delta-method SE(T));
    pair (q, d) uses Philox stream stream_base + q * stream_stride + d (stride 0 = n_db)."""
    n_list = 0 if pairs_q is None else pairs_q.numel()
    return ShpScreen(seed, stream_base, n_fixed, flags, tau, round, min_n, cap, watch, variant,
                     _dptr(omega_q), _dptr(omega_db), _dptr(self_se_q), _dptr(self_se_db), stream_stride,
                     _dptr(pairs_q), _dptr(pairs_db), n_list)


def _self_se(t, S: "ShapeSet"):
    if t is None:
        return None
    return t.to(device=S.device, dtype=torch.float64).contiguous()


def _weights(omega, S: "ShapeSet"):
    if omega is None:
        return None
    return omega.to(device=S.device, dtype=torch.float32).contiguous()


@_on_stream
def tanimoto_screen(Q: ShapeSet, D: ShapeSet, self_q: torch.Tensor, self_db: torch.Tensor, seed: int,
                    n_fixed: int = 0, flags: int = 0, stream_base: int = 0, stream=None, with_overlaps: bool = False,
                    out=None, tau: float = 0.005, round: int = 256, min_n: int = 1024, cap: int = 65536,
                    watch: int = 1, variant: int = -1, omega_q: torch.Tensor | None = None,
                    omega_db: torch.Tensor | None = None, self_se_q: torch.Tensor | None = None,
                    self_se_db: torch.Tensor | None = None, stream_stride: int = 0, pairs=None):
    """Screen every query against every database molecule (fixed budget when
    n_fixed > 0, else adaptive). Returns dict T, seT ([n_q * n_db, 2]
    float32), n_used ([n_q * n_db] int32 view of uint32) and, with
    with_overlaps, O, seO ([n_q * n_db, 2] float64). omega_q, omega_db
    (per-atom weights of each set) turn on the union slot's control
    variate; self_se_q, self_se_db (SEs of self_q, self_db) make seT, and
    the adaptive stop rule, the full delta-method SE. Pair (q, d) draws from
    stream stream_base + q * stream_stride + d (stream_stride 0 = n_db): a
    database shard [start, end) of n_global molecules passes start and
    n_global to reproduce the whole screen's numbers. pairs = (q ids, d
    ids) screens only those pairs (outputs indexed by list position, the
    same numbers the full screen gives them)."""
    dev = Q.device
    pq = pd = None
    if pairs is not None:
        if pairs[0] is None or pairs[1] is None:
            raise ShapeError(-1, "tanimoto_screen: a pair list needs both query and database ids")
        pq, pd = _device_i32(pairs[0], dev), _device_i32(pairs[1], dev)
        if pq.numel() != pd.numel():
            raise ValueError("pair lists differ in length")
    npairs = Q.n_mol * D.n_mol if pq is None else pq.numel()
    if out is None:
        out = dict(T=torch.empty((npairs, 2), dtype=torch.float32, device=dev),
                   seT=torch.empty((npairs, 2), dtype=torch.float32, device=dev),
                   n_used=torch.empty(npairs, dtype=torch.int32, device=dev))
        if with_overlaps:
            out["O"] = torch.empty((npairs, 2), dtype=torch.float64, device=dev)
            out["seO"] = torch.empty((npairs, 2), dtype=torch.float64, device=dev)
    if pq is not None and npairs == 0:
        return out  # an empty list: nothing to screen (the C call reads NULL arrays as "no list")
    omega_q, omega_db = _weights(omega_q, Q), _weights(omega_db, D)
    self_se_q, self_se_db = _self_se(self_se_q, Q), _self_se(self_se_db, D)
    cfg = screen_config(seed, n_fixed, tau, round, min_n, cap, watch, flags, stream_base, variant, omega_q, omega_db,
                        self_se_q, self_se_db, stream_stride, pq, pd)
    self_q = self_q.to(device=dev, dtype=torch.float64).contiguous()
    self_db = self_db.to(device=dev, dtype=torch.float64).contiguous()
    _check(load_library().tanimoto_screen(Q.handle, D.handle, ctypes.byref(cfg), _dptr(self_q), _dptr(self_db),
                                          _dptr(out["T"]), _dptr(out["seT"]), _dptr(out.get("O")),
                                          _dptr(out.get("seO")), _dptr(out.get("n_used")), _stream(stream)))
    return out


@_on_stream
def fo_tanimoto_screen(Q: ShapeSet, D: ShapeSet, fo_self_q: torch.Tensor, fo_self_db: torch.Tensor, stream=None,
                       out: torch.Tensor | None = None) -> torch.Tensor:
    """Closed-form first-order Tanimoto of every pair, [n_q * n_db] float32
    (pair q * n_db + d); fo_self_*: the closed-form self-overlaps [n]."""
    dev = Q.device
    T = out if out is not None else torch.empty(Q.n_mol * D.n_mol, dtype=torch.float32, device=dev)
    sq = fo_self_q.to(device=dev, dtype=torch.float64).contiguous()
    sd = fo_self_db.to(device=dev, dtype=torch.float64).contiguous()
    _check(load_library().fo_tanimoto_screen(Q.handle, D.handle, _dptr(sq), _dptr(sd), _dptr(T), _stream(stream)))
    return T


@_on_stream
def fo_prefilter_select(Q: ShapeSet, D: ShapeSet, T: torch.Tensor, k: int, stream=None):
    """(pairs_q, pairs_db) int32 device tensors [n_q * k]: for every query the
    k database molecules with the largest scores T ([n_q * n_db] float32),
    ties at the k-th score by lowest id, each query's pairs in ascending id."""
    dev = Q.device
    T = T.to(device=dev, dtype=torch.float32).contiguous()
    pq = torch.empty(Q.n_mol * k, dtype=torch.int32, device=dev)
    pd = torch.empty(Q.n_mol * k, dtype=torch.int32, device=dev)
    _check(load_library().fo_prefilter_select(Q.handle, D.handle, _dptr(T), k, _dptr(pq), _dptr(pd), _stream(stream)))
    return pq, pd


@_on_stream
def prefilter_db_ids(D: ShapeSet, pairs_db: torch.Tensor, stream=None) -> torch.Tensor:
    """[n_db] int32 device tensor: d for every database molecule d listed in
    pairs_db, -1 for the rest; as idx (with id_streams) it restricts the
    per-molecule estimators to the kept molecules, results at position d."""
    pd = _device_i32(pairs_db, D.device)
    ids = torch.empty(D.n_mol, dtype=torch.int32, device=D.device)
    _check(load_library().prefilter_db_ids(D.handle, _dptr(pd), pd.numel(), _dptr(ids), _stream(stream)))
    return ids


def fail_next_allocations(count: int) -> None:
    """Test hook: the next `count` device allocations of library calls fail
    as out of memory (0 clears)."""
    _check(load_library().shp_fail_next_allocations(count))


@_on_stream
def eval_probe(Q: ShapeSet, iq: int, D: ShapeSet, id_: int, variant: int = -1, draw: bool = False,
               batches: int = 256, stream=None) -> int:
    """Roofline calibration: the screen variant's per-sample work on the pair
    (Q[iq], D[id_]) with or without the random draw (see shp_eval_probe);
    returns the sample x atom evaluations of the call (time it with events)."""
    sink = torch.zeros(1, dtype=torch.float64, device=Q.device)
    ev = ctypes.c_int64()
    _check(load_library().shp_eval_probe(Q.handle, iq, D.handle, id_, variant, int(draw), batches, _dptr(sink),
                                         ctypes.byref(ev), _stream(stream)))
    return ev.value


def screen_variants() -> int:
    return load_library().shp_screen_variants()


def screen_variant_info(v: int) -> dict:
    """Launch shape of screen variant v: sample pairs per lane (sp), loop
    form, warps per CTA and CTAs per SM."""
    info = (ctypes.c_int32 * 4)()
    _check(load_library().shp_screen_variant_info(v, info))
    return dict(sp=info[0], form=info[1], warps=info[2], ctas=info[3])


@_on_stream
def tanimoto_screen_tune(Q: ShapeSet, D: ShapeSet, self_q: torch.Tensor, self_db: torch.Tensor, seed: int,
                         n_fixed: int = 0, n_sample: int = 4096, stream=None, tau: float = 0.005, round: int = 256,
                         min_n: int = 1024, cap: int = 65536, watch: int = 1, omega_q: torch.Tensor | None = None,
                         omega_db: torch.Tensor | None = None, self_se_q: torch.Tensor | None = None,
                         self_se_db: torch.Tensor | None = None):
    """Autotune the screen's launch variant on n_sample pairs (with the
    control variate when omega_q/omega_db are given); returns (best variant,
    per-variant milliseconds, -1 where not valid)."""
    dev = Q.device
    npairs = Q.n_mol * D.n_mol
    T = torch.empty((npairs, 2), dtype=torch.float32, device=dev)
    seT = torch.empty((npairs, 2), dtype=torch.float32, device=dev)
    nu = torch.empty(npairs, dtype=torch.int32, device=dev)
    omega_q, omega_db = _weights(omega_q, Q), _weights(omega_db, D)
    self_se_q, self_se_db = _self_se(self_se_q, Q), _self_se(self_se_db, D)
    cfg = screen_config(seed, n_fixed, tau, round, min_n, cap, watch, omega_q=omega_q, omega_db=omega_db,
                        self_se_q=self_se_q, self_se_db=self_se_db)
    nv = screen_variants()
    times = np.empty(nv, np.float32)
    best = ctypes.c_int32(-1)
    self_q = self_q.to(device=dev, dtype=torch.float64).contiguous()
    self_db = self_db.to(device=dev, dtype=torch.float64).contiguous()
    _check(load_library().tanimoto_screen_tune(Q.handle, D.handle, ctypes.byref(cfg), _dptr(self_q), _dptr(self_db),
                                               _dptr(T), _dptr(seT), _dptr(nu), n_sample, times.ctypes.data,
                                               ctypes.byref(best), _stream(stream)))
    return best.value, times


@_on_stream
def self_overlaps(S: ShapeSet, seed: int, n_samples: int, stream_base: int = 0, stream=None,
                  target_rel_se: float = 0.0, round: int = 256, omega=None, with_se: bool = False, idx=None):
    """[n, 2] float64 device tensor (n = n_mol, or the length of idx): slot 0
    closed-form first-order self-overlap, slot 1 union self-overlap estimate
    (n_samples draws, or rounds of `round` up to the cap n_samples until its
    relative SE is <= target_rel_se; omega: control-variate weights per set
    atom). With with_se, returns (self, se, n_used): se [n, 2] (slot 0 zero,
    the closed form is exact) and the samples per molecule. With idx, only
    the listed molecules, each on its own id's stream (stream_base + id), so
    they get exactly the values of the call over the whole set."""
    dev = S.device
    by_id = idx is not None
    idx = torch.arange(S.n_mol, dtype=torch.int32, device=dev) if idx is None else _device_i32(idx, dev)
    n = idx.numel()
    out = torch.empty((n, 2), dtype=torch.float64, device=dev)
    fo = fo_overlap(S, idx, S, idx, stream=stream)
    if target_rel_se <= 0 and omega is None and not with_se:
        vol, vse, so, sse = union_volume_estimate(S, idx, seed=seed, n_samples=n_samples, stream_base=stream_base,
                                                  stream=stream, flags=ID_STREAMS if by_id else 0)
        nu = None
    else:
        _, _, so, sse, nu = union_self_estimate(S, idx if by_id else None, omega=omega, seed=seed,
                                                n_samples=n_samples, target_rel_se=target_rel_se, round=round,
                                                watch=1, stream_base=stream_base, stream=stream, id_streams=by_id)
    out[:, 0] = fo
    out[:, 1] = so
    if not with_se:
        return out
    se = torch.zeros((n, 2), dtype=torch.float64, device=dev)
    se[:, 1] = sse
    return out, se, nu


# ---------------------------------------------------------------- alignment

@_on_stream
def align_crn_points(Q: ShapeSet, iq: int, seed: int, n: int, stream_base: int = 0, stream=None,
                     antithetic: bool = False):
    """[n, 4] float32 device tensor: CRN points of Q[iq] and their union
    weights (antithetic: in pairs reflected about their component centre)."""
    pts = torch.empty((n, 4), dtype=torch.float32, device=Q.device)
    mc = ShpMC(seed, stream_base, n, ANTITHETIC if antithetic else 0)
    _check(load_library().align_crn_points(Q.handle, iq, ctypes.byref(mc), _dptr(pts), _stream(stream)))
    return pts


@_on_stream
def overlap_pose_grad(Q: ShapeSet, iq: int, points: torch.Tensor, B: ShapeSet, ib, pose, objective: int = OBJ_UNION,
                      stream=None):
    """(value [n] float64, grad [n, 7] float32): CRN overlap of B[ib[k]] posed by
    pose[k] and its gradient with respect to the raw pose."""
    dev = Q.device
    ib = _device_i32(ib, dev)
    n = ib.numel()
    pose = torch.as_tensor(pose, dtype=torch.float32, device=dev).contiguous()
    if pose.shape != (n, 7):
        raise ValueError("pose must be [n, 7]")
    points = None if points is None else points.contiguous()  # unused by OBJ_FO_CLOSED
    value = torch.empty(n, dtype=torch.float64, device=dev)
    grad = torch.empty((n, 7), dtype=torch.float32, device=dev)
    n_points = 0 if points is None else points.shape[0]
    _check(load_library().overlap_pose_grad(Q.handle, iq, _dptr(points), n_points, B.handle, _dptr(ib), n,
                                            _dptr(pose), objective, _dptr(value), _dptr(grad), _stream(stream)))
    return value, grad


class PoseOverlap(torch.autograd.Function):
    """Differentiable CRN overlap (Eq. grad): forward and adjoint come from
    one fused kernel launch; backward scales the saved pose gradient."""

    @staticmethod
    def forward(ctx, pose, Q, iq, points, B, ib, objective):
        value, grad = overlap_pose_grad(Q, iq, points, B, ib, pose.detach(), objective)
        ctx.save_for_backward(grad)
        return value.to(pose.dtype)

    @staticmethod
    def backward(ctx, g_out):
        (grad,) = ctx.saved_tensors
        return (g_out[:, None] * grad).to(g_out.dtype), None, None, None, None, None, None


def pose_overlap(pose, Q: ShapeSet, iq: int, points: torch.Tensor, B: ShapeSet, ib, objective: int = OBJ_UNION):
    """Autograd-enabled CRN overlap of B[ib[k]] under pose[k] ([n, 7])."""
    return PoseOverlap.apply(pose, Q, iq, points, B, ib, objective)


@_on_stream
def align_rigid(Q: ShapeSet, iq: int, B: ShapeSet, ib, self_q: torch.Tensor, self_db: torch.Tensor, seed: int = 0,
                starts: int = 8, steps: int = 100, n_crn: int = 1024, objective: int = OBJ_UNION, lr: float = 0.02,
                lr_t: float = 0.05, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, n_score: int = 4096,
                stream_base: int = 0, with_starts: bool = False, stream=None, antithetic: bool = True):
    """Multi-start Adam alignment of B[ib[k]] onto Q[iq]. Returns dict pose
    ([n, 7]), T ([n]) and, with with_starts, T_starts ([n, starts]) and
    pose_starts ([n, starts, 7], every start's final raw pose). antithetic
    (the default): the CRN points in antithetic pairs, each odd point the
    reflection of the even one about its component centre (same n_crn), whose
    union objective peaks at the exact superposition of a rigid copy; False:
    independent points (SHP_ANTITHETIC off in shp_align.crn_flags)."""
    dev = Q.device
    ib = _device_i32(ib, dev)
    n = ib.numel()
    cfg = ShpAlign(seed, stream_base, starts, steps, n_crn, objective, lr, lr_t, beta1, beta2, eps, n_score,
                   ANTITHETIC if antithetic else 0)
    out = dict(pose=torch.empty((n, 7), dtype=torch.float32, device=dev),
               T=torch.empty(n, dtype=torch.float32, device=dev))
    if with_starts:
        out["T_starts"] = torch.empty((n, starts), dtype=torch.float32, device=dev)
        out["pose_starts"] = torch.empty((n, starts, 7), dtype=torch.float32, device=dev)
    self_q = self_q.to(device=dev, dtype=torch.float64).contiguous()
    self_db = self_db.to(device=dev, dtype=torch.float64).contiguous()
    _check(load_library().align_rigid(Q.handle, iq, B.handle, _dptr(ib), n, ctypes.byref(cfg), _dptr(self_q),
                                      _dptr(self_db), _dptr(out["pose"]), _dptr(out["T"]), _dptr(out.get("T_starts")),
                                      _dptr(out.get("pose_starts")), _stream(stream)))
    return out


# ---------------------------------------------------------------- control variate

@_on_stream
def union_attributions(S: ShapeSet, seed: int, M: int = 512, stream_base: int = 0, stream=None):
    """[n_atoms] float32 device tensor: om*_i = E_{N(c_i, 1/(2 alpha_i))}[u/m]."""
    out = torch.empty(S.n_atoms, dtype=torch.float32, device=S.device)
    _check(load_library().union_attributions(S.handle, seed, stream_base, M, _dptr(out), _stream(stream)))
    return out


@_on_stream
def union_volume_cv(S: ShapeSet, idx=None, omega=None, seed: int = 0, n_samples: int = 4096,
                    target_rel_se: float = 0.0, round: int = 256, stream_base: int = 0, stream=None,
                    id_streams: bool = False):
    """(vol, vol_se, n_used): union volumes with the control variate omega
    (per set atom; None = plain), fixed n_samples or adaptive to a relative SE.
    id_streams: molecule idx[k] uses stream stream_base + idx[k]."""
    dev = S.device
    if idx is not None:
        idx = _device_i32(idx, dev)
        n = idx.numel()
    else:
        n = S.n_mol
    if omega is not None:
        omega = torch.as_tensor(omega, dtype=torch.float32, device=dev).contiguous()
    vol = torch.empty(n, dtype=torch.float64, device=dev)
    se = torch.empty(n, dtype=torch.float64, device=dev)
    nu = torch.empty(n, dtype=torch.int32, device=dev)
    mc = ShpMC(seed, stream_base, n_samples, ID_STREAMS if id_streams else 0)
    _check(load_library().union_volume_cv(S.handle, _dptr(idx), n, ctypes.byref(mc), _dptr(omega), target_rel_se,
                                          round, _dptr(vol), _dptr(se), _dptr(nu), _stream(stream)))
    return vol, se, nu


@_on_stream
def union_self_estimate(S: ShapeSet, idx=None, omega=None, seed: int = 0, n_samples: int = 4096,
                        target_rel_se: float = 0.0, round: int = 256, watch: int = 1, stream_base: int = 0,
                        stream=None, id_streams: bool = False):
    """(vol, vol_se, self_ov, self_se, n_used): union volumes and union
    self-overlaps, plain or with the control variate omega, fixed n_samples
    or rounds until the watched estimate (0 volume, 1 self-overlap) reaches
    target_rel_se (n_samples is then the cap). id_streams: molecule idx[k]
    uses stream stream_base + idx[k], so a subset gets the whole set's values."""
    dev = S.device
    if idx is not None:
        idx = _device_i32(idx, dev)
        n = idx.numel()
    else:
        n = S.n_mol
    if omega is not None:
        omega = torch.as_tensor(omega, dtype=torch.float32, device=dev).contiguous()
    outs = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(4)]
    nu = torch.empty(n, dtype=torch.int32, device=dev)
    mc = ShpMC(seed, stream_base, n_samples, ID_STREAMS if id_streams else 0)
    _check(load_library().union_self_estimate(S.handle, _dptr(idx), n, ctypes.byref(mc), _dptr(omega), target_rel_se,
                                              round, watch, *(_dptr(t) for t in outs), _dptr(nu), _stream(stream)))
    return (*outs, nu)


@_on_stream
def cv_fit_weights(S: ShapeSet, seed: int, n_samples: int = 1024, stream_base: int = 0, ridge: float = 1e-6,
                   idx=None, out: torch.Tensor | None = None, stream=None, id_streams: bool = False) -> torch.Tensor:
    """[n_atoms] float32 device tensor: least-squares control-variate weights
    (the projection of u onto each molecule's Gaussians, the right-hand side
    from n_samples of its own samples) for the listed molecules (all if idx
    is None). id_streams: molecule idx[k] uses stream stream_base + idx[k]."""
    dev = S.device
    omega = out if out is not None else torch.zeros(S.n_atoms, dtype=torch.float32, device=dev)
    if idx is None:
        n, ip = S.n_mol, None
    else:
        ip = _device_i32(idx, dev)
        n = ip.numel()
    mc = ShpMC(seed, stream_base, n_samples, ID_STREAMS if id_streams else 0)
    _check(load_library().cv_fit_weights(S.handle, _dptr(ip), n, ctypes.byref(mc), ridge, _dptr(omega),
                                         _stream(stream)))
    return omega


@_on_stream
def cv_features(S: ShapeSet, stream=None):
    """[n_atoms, 33] float32 device tensor of per-atom neighbour features."""
    out = torch.empty((S.n_atoms, MLP_IN), dtype=torch.float32, device=S.device)
    _check(load_library().cv_features(S.handle, _dptr(out), _stream(stream)))
    return out


@_on_stream
def mlp_forward(params: torch.Tensor, x: torch.Tensor, rows=None, stream=None):
    n = x.shape[0] if rows is None else rows.numel()
    y = torch.empty(n, dtype=torch.float32, device=x.device)
    _check(load_library().mlp_forward(_dptr(params), _dptr(x), _dptr(rows), n, _dptr(y), _stream(stream)))
    return y


@_on_stream
def mlp_loss_grad(params: torch.Tensor, x: torch.Tensor, target: torch.Tensor, rows=None, stream=None, out=None):
    """(loss [1] float64, grad [6401] float32) device tensors."""
    n = x.shape[0] if rows is None else rows.numel()
    grad, loss = out if out is not None else (torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device),
                                              torch.empty(1, dtype=torch.float64, device=x.device))
    _check(load_library().mlp_loss_grad(_dptr(params), _dptr(x), _dptr(target), _dptr(rows), n, _dptr(grad),
                                        _dptr(loss), _stream(stream)))
    return loss, grad


@_on_stream
def mlp_adam(params, m, v, grad, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8, stream=None):
    _check(load_library().mlp_adam(_dptr(params), _dptr(m), _dptr(v), _dptr(grad), params.numel(), step, lr, beta1,
                                   beta2, eps, _stream(stream)))


@_on_stream
def mlp_train_epoch(params, m, v, x, target, perm, batch: int, step0: int, lr: float, beta1: float = 0.9,
                    beta2: float = 0.999, eps: float = 1e-8, stream=None) -> torch.Tensor:
    """One epoch of minibatches over perm (mlp_loss_grad then mlp_adam per
    minibatch, steps step0 + 1 ...), the loop inside the library; returns
    each minibatch's mean squared error ([ceil(n / batch)] float64 device)."""
    perm = _device_i32(perm, params.device)
    n = perm.numel()
    losses = torch.empty((n + batch - 1) // batch, dtype=torch.float64, device=params.device)
    _check(load_library().mlp_train_epoch(_dptr(params), _dptr(m), _dptr(v), _dptr(x), _dptr(target), _dptr(perm), n,
                                          batch, step0, lr, beta1, beta2, eps, _dptr(losses), _stream(stream)))
    return losses
