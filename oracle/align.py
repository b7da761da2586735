"""FP64 restatement of the multi-start rigid alignment (Sec. differentiable
alignment and the hybrid pipeline): principal frames, start poses, Adam
ascent on the pose with a cosine step-size decay, best start by the union
Tanimoto.

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` to check the CUDA
optimiser's trajectories; never by the product package. It shares no code
with the library: the frames come from numpy's symmetric eigensolver, the
gradients from central differences of the oracle's FP64 CRN objective (or
the oracle's analytic first-order gradient for the closed-form objective),
the random start rotations from the oracle's own Philox4x32-10.

Conventions the paper leaves open, stated here and implemented separately
in the library:
  - principal frame: centroid weighted by the Gaussian volumes v_i =
    p_i (pi / alpha_i)^{3/2}; axes = eigenvectors of the v-weighted second
    moment matrix by decreasing eigenvalue; the first two axes point so that
    the v-weighted third moment of the projection is >= 0; the third axis is
    their cross product (a proper rotation E with the axes as columns);
  - starts s = 0..3: R = E_Q M_s E_B^T with M_s = diag(sx, sy, sx sy),
    (sx, sy) = (1, 1), (1, -1), (-1, 1), (-1, -1); starts s >= 4: M_s a
    uniform random rotation (Shoemake's method) from the Philox words of
    counter (s, pair lo, pair hi, 4) under the alignment seed, uniforms
    (word >> 8) 2^-24, unit quaternion (sqrt(u1) cos 2 pi u3,
    sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2, sqrt(u1) sin 2 pi u3);
    translation t = c_Q - R c_B (centroids matched);
  - pose = raw quaternion (w, x, y, z) and translation; the objective
    normalises the quaternion; after every step the raw quaternion is
    renormalised;
  - Adam ascent, bias-corrected, step t = 1..T:
      m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
      pose += d_t lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
    d_t = (1 + cos(pi (t - 1) / T)) / 2, lr for the quaternion and lr_t for
    the translation.
"""
from __future__ import annotations

import numpy as np

from . import _oset, crn_points, fo_pose_grad, lib, mixture_mass, mol_tables, philox

OBJ_FO, OBJ_UNION, OBJ_FO_CLOSED = 0, 1, 2
TAG_START = 4


def _mol(ms, idx, c_alpha=2.41798793):
    s = _oset(ms, c_alpha)
    lo, hi = int(s.offsets[idx]), int(s.offsets[idx + 1])
    x = s.xyz[lo:hi].astype(np.float64)
    v = mol_tables(ms, idx, c_alpha)["v"]
    return x, v


def principal_frame(ms, idx, c_alpha=2.41798793):
    """(centroid [3], E [3, 3] with the axes as columns, det +1)."""
    x, v = _mol(ms, idx, c_alpha)
    c = (v[:, None] * x).sum(0) / v.sum()
    d = x - c
    C = (v[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0)
    ev, V = np.linalg.eigh(C)
    order = np.argsort(-ev, kind="stable")
    E = np.empty((3, 3))
    for a in range(2):
        ax = V[:, order[a]]
        if (v * (d @ ax) ** 3).sum() < 0:
            ax = -ax
        E[:, a] = ax
    E[:, 2] = np.cross(E[:, 0], E[:, 1])
    return c, E


def quat_to_rot(q):
    q = np.asarray(q, np.float64)
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def rot_to_quat(R):
    """Unit quaternion (w, x, y, z) of a rotation matrix (Shepperd's
    method: the branch of the largest of trace, R00, R11, R22)."""
    R = np.asarray(R, np.float64)
    tr = np.trace(R)
    if tr > 0:
        s = 2.0 * np.sqrt(tr + 1.0)
        return np.array([0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s])
    if R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = 2.0 * np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2])
        return np.array([(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s])
    if R[1, 1] > R[2, 2]:
        s = 2.0 * np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2])
        return np.array([(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s])
    s = 2.0 * np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1])
    return np.array([(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s])


def random_rotation(seed: int, pair: int, s: int):
    """Shoemake's uniform random rotation from the Philox words of counter
    (s, pair lo, pair hi, 4) under key (seed lo, seed hi)."""
    w = philox([s, pair & 0xFFFFFFFF, (pair >> 32) & 0xFFFFFFFF, TAG_START],
               [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF])
    u1, u2, u3 = ((int(w[k]) >> 8) * 2.0 ** -24 for k in range(3))
    r1, r2 = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.array([r2 * np.cos(2 * np.pi * u3), r1 * np.sin(2 * np.pi * u2), r1 * np.cos(2 * np.pi * u2),
                  r2 * np.sin(2 * np.pi * u3)])
    return quat_to_rot(q)


_SIGNS = ((1.0, 1.0), (1.0, -1.0), (-1.0, 1.0), (-1.0, -1.0))


def start_pose(frame_q, frame_b, s: int, seed: int = 0, pair: int = 0):
    """Raw pose [7] of start s for the pair (Q, B) from their principal frames."""
    cq, Eq = frame_q
    cb, Eb = frame_b
    if s < 4:
        sx, sy = _SIGNS[s]
        M = np.diag([sx, sy, sx * sy])
    else:
        M = random_rotation(seed, pair, s)
    R = Eq @ M @ Eb.T
    return np.concatenate([rot_to_quat(R), cq - R @ cb])


def objective_grad(Q, iq, B, ib, pose, objective, points=None, ZQ=None, h=1e-5):
    """(F, dF/d raw pose [7]) in FP64: central differences of the CRN
    objective (Eq. grad's estimator), or the analytic gradient of the closed
    form (Eq. fo)."""
    if objective == OBJ_FO_CLOSED:
        return fo_pose_grad(Q, iq, B, ib, pose)
    sb = _oset(B)
    pts = np.ascontiguousarray(points, dtype=np.float64)
    p = np.ascontiguousarray(pose, dtype=np.float64)
    import ctypes
    F = ctypes.c_double()
    g = np.empty(7)
    rc = lib().orc_pose_grad_fd(ZQ, pts.ctypes.data, len(pts), sb.ref, ib, p.ctypes.data, objective, h,
                                ctypes.addressof(F), g.ctypes.data)
    if rc != 0:
        raise ValueError(f"pose_grad_fd failed with status {rc}")
    return F.value, g


def adam(Q, iq, B, ib, pose0, steps, objective=OBJ_UNION, points=None, lr=0.02, lr_t=0.05, beta1=0.9,
         beta2=0.999, eps=1e-8, total=None):
    """Adam ascent of the objective from pose0 for `steps` steps of a run of
    `total` steps (the cosine decay's length; default steps). Returns the
    raw pose after each step, [steps + 1, 7] (row 0 = pose0)."""
    total = steps if total is None else total
    ZQ = float(mixture_mass(Q, [iq])[0]) if objective != OBJ_FO_CLOSED else None
    pose = np.asarray(pose0, np.float64).copy()
    m = np.zeros(7)
    v = np.zeros(7)
    traj = [pose.copy()]
    lrs = np.array([lr] * 4 + [lr_t] * 3)
    for t in range(1, steps + 1):
        _, g = objective_grad(Q, iq, B, ib, pose, objective, points, ZQ)
        m = beta1 * m + (1 - beta1) * g
        v = beta2 * v + (1 - beta2) * g * g
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        decay = 0.5 * (1 + np.cos(np.pi * (t - 1) / total))
        pose = pose + decay * lrs * mh / (np.sqrt(vh) + eps)
        pose[:4] /= np.linalg.norm(pose[:4])
        traj.append(pose.copy())
    return np.array(traj)


def crn(Q, iq, seed, stream, n, antithetic=False):
    """The CRN points of the alignment (tag 3) with their union weights."""
    return crn_points(Q, iq, seed=seed, stream=stream, n=n, antithetic=antithetic)
