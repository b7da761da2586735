"""Seeded synthetic molecule sets (inputs for both the CUDA path and the oracle).

Holds no shape-overlap arithmetic: it only builds atom centres, elements and
radii (a random tree walk, see ``molgen.cpp``) and the principal-axis
pre-alignment used by the screening workloads. Stand-in for the paper's
drug-like molecules and screening libraries (Sec. "Results and Discussion"),
which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libmolgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libmolgen.so in-tree (g++, OpenMP)."""
    src = os.path.join(_HERE, "molgen.cpp")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.molgen_counts.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_void_p]
        lib.molgen_generate.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass
class MolSet:
    """A batch of molecules in flat (SoA-by-atom) host arrays."""
    xyz: np.ndarray          # float32 [n_atoms, 3], Angstrom
    radius: np.ndarray       # float32 [n_atoms], Angstrom
    offsets: np.ndarray      # int32 [n_mol + 1]
    elem: np.ndarray         # uint8 [n_atoms]: 0 C, 1 N, 2 O, 3 S
    height: np.ndarray | None = None  # float32 [n_atoms] or None (library default 2*sqrt(2))

    @property
    def n_mol(self) -> int:
        return len(self.offsets) - 1

    @property
    def n_atoms(self) -> int:
        return int(self.offsets[-1])

    @property
    def counts(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int32)

    def mol(self, i: int) -> np.ndarray:
        return self.xyz[self.offsets[i]:self.offsets[i + 1]]

    def subset(self, idx) -> "MolSet":
        idx = np.asarray(idx, dtype=np.int64)
        cnt = self.counts[idx]
        off = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(cnt, out=off[1:])
        sel = np.concatenate([np.arange(self.offsets[i], self.offsets[i + 1]) for i in idx]) \
            if len(idx) else np.zeros(0, dtype=np.int64)
        return MolSet(self.xyz[sel].copy(), self.radius[sel].copy(), off.astype(np.int32),
                      self.elem[sel].copy(), None if self.height is None else self.height[sel].copy())

    def concat(self, other: "MolSet") -> "MolSet":
        off = np.concatenate([self.offsets, other.offsets[1:] + self.offsets[-1]]).astype(np.int32)
        h = None
        if self.height is not None or other.height is not None:
            dh = np.float32(2.0 * np.sqrt(2.0))
            h1 = self.height if self.height is not None else np.full(self.n_atoms, dh, np.float32)
            h2 = other.height if other.height is not None else np.full(other.n_atoms, dh, np.float32)
            h = np.concatenate([h1, h2])
        return MolSet(np.concatenate([self.xyz, other.xyz]), np.concatenate([self.radius, other.radius]),
                      off, np.concatenate([self.elem, other.elem]), h)


def counts_uniform(seed: int, n: int, lo: int, hi: int) -> np.ndarray:
    out = np.empty(n, dtype=np.int32)
    if _load().molgen_counts(seed, n, 0, lo, hi, out.ctypes.data) != 0:
        raise ValueError("bad count arguments")
    return out


def counts_heavy(seed: int, n: int, lo: int = 18, hi: int = 60) -> np.ndarray:
    """round(40 + 6 t_3) clipped to [lo, hi]: heavy-tailed toward 40 atoms."""
    out = np.empty(n, dtype=np.int32)
    if _load().molgen_counts(seed, n, 1, lo, hi, out.ctypes.data) != 0:
        raise ValueError("bad count arguments")
    return out


def generate(seed: int, counts, first: int = 0) -> MolSet:
    """Molecules first .. first+len(counts)-1 of stream ``seed`` (random tree walks)."""
    counts = np.asarray(counts, dtype=np.int64)
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    n_atoms = int(off[-1])
    xyz = np.empty((n_atoms, 3), dtype=np.float32)
    rad = np.empty(n_atoms, dtype=np.float32)
    el = np.empty(n_atoms, dtype=np.uint8)
    rc = _load().molgen_generate(seed, first, len(counts), off.ctypes.data, xyz.ctypes.data,
                                 rad.ctypes.data, el.ctypes.data)
    if rc != 0:
        raise RuntimeError("molecule generation failed")
    return MolSet(xyz, rad, off.astype(np.int32), el)


def principal_axes(ms: MolSet) -> MolSet:
    """Pre-align every molecule at its principal axes.

    Weights are the atomic hard-sphere volumes (proportional to R^3). The
    frame is centred at the weighted centroid, axes sorted by decreasing
    second moment, the first two axes oriented so the weighted third moment
    of the projection is non-negative, and the third axis completes a proper
    (right-handed) rotation.
    """
    n = ms.n_mol
    cnt = ms.counts.astype(np.int64)
    mol_of = np.repeat(np.arange(n), cnt)
    w = ms.radius.astype(np.float64) ** 3
    x = ms.xyz.astype(np.float64)
    wsum = np.bincount(mol_of, weights=w, minlength=n)
    cen = np.stack([np.bincount(mol_of, weights=w * x[:, k], minlength=n) for k in range(3)], 1)
    cen /= wsum[:, None]
    d = x - cen[mol_of]
    cov = np.zeros((n, 3, 3))
    for a in range(3):
        for b in range(3):
            cov[:, a, b] = np.bincount(mol_of, weights=w * d[:, a] * d[:, b], minlength=n)
    evals, evecs = np.linalg.eigh(cov)          # ascending
    evecs = evecs[:, :, ::-1]                   # descending second moment
    proj = np.einsum("ia,iab->ib", d, evecs[mol_of])
    for k in range(2):
        skew = np.bincount(mol_of, weights=w * proj[:, k] ** 3, minlength=n)
        sgn = np.where(skew < 0, -1.0, 1.0)
        evecs[:, :, k] *= sgn[:, None]
    evecs[:, :, 2] = np.cross(evecs[:, :, 0], evecs[:, :, 1])
    proj = np.einsum("ia,iab->ib", d, evecs[mol_of])
    return MolSet(proj.astype(np.float32), ms.radius.copy(), ms.offsets.copy(), ms.elem.copy(),
                  None if ms.height is None else ms.height.copy())


def centre(ms: MolSet) -> MolSet:
    """Translate each molecule so its (unweighted) atom centroid is at the origin."""
    cnt = ms.counts.astype(np.int64)
    mol_of = np.repeat(np.arange(ms.n_mol), cnt)
    x = ms.xyz.astype(np.float64)
    cen = np.stack([np.bincount(mol_of, weights=x[:, k], minlength=ms.n_mol) for k in range(3)], 1)
    cen /= cnt[:, None]
    return MolSet((x - cen[mol_of]).astype(np.float32), ms.radius.copy(), ms.offsets.copy(),
                  ms.elem.copy(), None if ms.height is None else ms.height.copy())


def single_pair(n_a: int = 12, n_b: int = 15, seed_a: int = 0, seed_b: int = 1,
                separation: float = 1.0) -> tuple[MolSet, MolSet]:
    """One pair of small molecules: A (n_a atoms) and B (n_b atoms), each from
    its own seed, both centred, B's centroid shifted ``separation`` A along x."""
    a = centre(generate(seed_a, [n_a]))
    b = centre(generate(seed_b, [n_b]))
    b.xyz[:, 0] += np.float32(separation)
    return a, b


def fixed_screen(n_db: int = 100_000, n_query_atoms: int = 32, seed: int = 2026,
                 lo: int = 18, hi: int = 60) -> tuple[MolSet, MolSet]:
    """1 query of n_query_atoms atoms x n_db database molecules (counts uniform
    in [lo, hi]), all pre-aligned at their principal axes."""
    q = principal_axes(generate(seed, [n_query_atoms]))
    db = principal_axes(generate(seed + 1, counts_uniform(seed + 1, n_db, lo, hi)))
    return q, db


def adaptive_screen(n_q: int = 16, n_db: int = 1_000_000, seed: int = 4242) -> tuple[MolSet, MolSet]:
    """n_q queries (20-48 atoms, uniform) x n_db database molecules (18-60
    atoms, heavy-tailed toward 40), pre-aligned at principal axes."""
    q = principal_axes(generate(seed, counts_uniform(seed, n_q, 20, 48)))
    db = principal_axes(generate(seed + 1, counts_heavy(seed + 1, n_db)))
    return q, db
