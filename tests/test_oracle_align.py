"""Pins for the oracle's alignment pieces (Sec. differentiable alignment,
Eq. pose, Eq. grad): the analytic first-order gradient against finite
differences of the closed form, the CRN objectives against the exact
overlaps at a pose, and invariances of the pose gradient."""
import numpy as np
import pytest

import oracle as O
from paper_2607_20766_b300 import synth

POSE = np.array([0.9, 0.1, -0.2, 0.3, 0.4, -0.3, 0.2])


@pytest.fixture(scope="module")
def pair():
    return synth.single_pair()


def test_analytic_fo_gradient_matches_finite_differences(pair):
    a, b = pair
    F, g = O.fo_pose_grad(a, 0, b, 0, POSE)
    h = 1e-5
    fd = np.empty(7)
    for d in range(7):
        pp, pm = POSE.copy(), POSE.copy()
        pp[d] += h
        pm[d] -= h
        fd[d] = (O.fo_pose_grad(a, 0, b, 0, pp)[0] - O.fo_pose_grad(a, 0, b, 0, pm)[0]) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * np.abs(g).max())
    assert F == pytest.approx(O.fo_overlap(a, [0], b, [0], poses=POSE.astype(np.float32)[None])[0], rel=1e-6)


def test_quaternion_scale_invariance(pair):
    a, b = pair
    _, g = O.fo_pose_grad(a, 0, b, 0, POSE)
    assert abs(np.dot(g[:4], POSE[:4])) < 1e-9 * np.abs(g).max()
    _, g2 = O.fo_pose_grad(a, 0, b, 0, np.concatenate([3 * POSE[:4], POSE[4:]]))
    np.testing.assert_allclose(g2[:4], g[:4] / 3, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(g2[4:], g[4:], rtol=1e-9)


def test_identical_copy_is_stationary(pair):
    a, _ = pair
    F, g = O.fo_pose_grad(a, 0, a, 0, np.array([1.0, 0, 0, 0, 0, 0, 0]))
    assert np.abs(g).max() < 1e-9 * F


def test_crn_objectives_estimate_the_exact_overlaps(pair):
    a, b = pair
    ZQ = O.mixture_mass(a)[0]
    pts = O.crn_points(a, 0, seed=3, stream=0, n=1 << 16)
    fo = O.pose_objective(ZQ, pts, b, 0, POSE, objective=O.OBJ_FO)
    un = O.pose_objective(ZQ, pts, b, 0, POSE, objective=O.OBJ_UNION)
    fo_exact = O.fo_overlap(a, [0], b, [0], poses=POSE.astype(np.float32)[None])[0]
    un_exact = O.union_overlap_ie(a, 0, b, 0, poseB=POSE.astype(np.float32))
    assert fo == pytest.approx(fo_exact, rel=0.015)
    assert un == pytest.approx(un_exact, rel=0.015)
    # the union weights are those of the query at the points
    m, u = O.occupancy(a, 0, pts[:100, :3])
    np.testing.assert_allclose(pts[:100, 3], u / m, rtol=1e-14)


def test_antithetic_crn_points(pair):
    """Antithetic CRN points: each odd point is the reflection of the even one
    about an atom centre of the query (the even point's component), the even
    points are those of the plain layout, and the objectives still estimate
    the exact overlaps."""
    a, b = pair
    plain = O.crn_points(a, 0, seed=3, stream=0, n=2000)
    anti = O.crn_points(a, 0, seed=3, stream=0, n=2000, antithetic=True)
    np.testing.assert_array_equal(anti[0::2], plain[0::2])
    mid = 0.5 * (anti[0::2, :3] + anti[1::2, :3])
    d = np.linalg.norm(mid[:, None, :] - a.xyz[None, :, :].astype(np.float64), axis=2).min(1)
    assert d.max() < 1e-12
    assert not np.allclose(anti[1::2], plain[1::2])
    ZQ = O.mixture_mass(a)[0]
    pts = O.crn_points(a, 0, seed=4, stream=0, n=1 << 16, antithetic=True)
    un = O.pose_objective(ZQ, pts, b, 0, POSE, objective=O.OBJ_UNION)
    un_exact = O.union_overlap_ie(a, 0, b, 0, poseB=POSE.astype(np.float32))
    assert un == pytest.approx(un_exact, rel=0.015)


def test_crn_first_order_gradient_estimates_the_analytic_one(pair):
    a, b = pair
    ZQ = O.mixture_mass(a)[0]
    pts = O.crn_points(a, 0, seed=5, stream=1, n=1 << 15)
    _, g_is = O.pose_grad_fd(ZQ, pts, b, 0, POSE, objective=O.OBJ_FO, h=1e-4)
    _, g_an = O.fo_pose_grad(a, 0, b, 0, POSE)
    assert np.linalg.norm(g_is - g_an) < 0.05 * np.linalg.norm(g_an)


def test_fd_gradient_converges_in_h(pair):
    """Central differences of the (smooth) CRN objective: h = 1e-3 agrees
    with h = 1e-4 to O(h^2)."""
    a, b = pair
    ZQ = O.mixture_mass(a)[0]
    pts = O.crn_points(a, 0, seed=5, stream=2, n=2048)
    _, g3 = O.pose_grad_fd(ZQ, pts, b, 0, POSE, objective=O.OBJ_UNION, h=1e-3)
    _, g4 = O.pose_grad_fd(ZQ, pts, b, 0, POSE, objective=O.OBJ_UNION, h=1e-4)
    # truncation error of the h = 1e-3 step is ~1e-5 of the gradient norm
    assert np.linalg.norm(g3 - g4) < 1e-4 * np.linalg.norm(g4)


# ---------------------------------------------------------------- multi-start Adam (oracle/align.py)

from scipy.spatial.transform import Rotation  # noqa: E402

from oracle import align as OA  # noqa: E402
from paper_2607_20766_b300.synth import MolSet  # noqa: E402


def _moved(ms, R, t):
    return MolSet((ms.xyz.astype(np.float64) @ R.T + t).astype(np.float32), ms.radius.copy(), ms.offsets.copy(),
                  ms.elem.copy())


def _rmsd(a, b, pose):
    R = OA.quat_to_rot(pose[:4])
    moved = b.xyz.astype(np.float64) @ R.T + pose[4:]
    return float(np.sqrt(((moved - a.xyz.astype(np.float64)) ** 2).sum(1).mean()))


@pytest.fixture(scope="module")
def copy_pair():
    a = synth.centre(synth.generate(60, [22]))
    R = Rotation.random(random_state=3).as_matrix()
    t = np.array([2.0, -1.0, 0.5])
    return a, _moved(a, R, t), R, t


def test_principal_frame_is_equivariant(copy_pair):
    a, b, R, t = copy_pair
    ca, Ea = OA.principal_frame(a, 0)
    cb, Eb = OA.principal_frame(b, 0)
    np.testing.assert_allclose(Ea.T @ Ea, np.eye(3), atol=1e-12)
    assert np.linalg.det(Ea) == pytest.approx(1.0, abs=1e-12)
    np.testing.assert_allclose(cb, R @ ca + t, atol=2e-6)      # float32 coordinates
    np.testing.assert_allclose(Eb, R @ Ea, atol=2e-5)


def test_identity_start_superposes_a_rigid_copy(copy_pair):
    """Start 0 maps B's principal frame onto A's: for B a rigid copy of A it is
    the exact superposition (R^T, -R^T t)."""
    a, b, R, t = copy_pair
    p0 = OA.start_pose(OA.principal_frame(a, 0), OA.principal_frame(b, 0), 0)
    np.testing.assert_allclose(OA.quat_to_rot(p0[:4]), R.T, atol=2e-5)
    np.testing.assert_allclose(p0[4:], -R.T @ t, atol=1e-4)
    assert _rmsd(a, b, p0) < 1e-4
    # the other three sign patterns are proper rotations by pi about the frame axes
    for s in (1, 2, 3):
        ps = OA.start_pose(OA.principal_frame(a, 0), OA.principal_frame(b, 0), s)
        D = OA.quat_to_rot(ps[:4]) @ OA.quat_to_rot(p0[:4]).T
        assert np.trace(D) == pytest.approx(-1.0, abs=1e-6)  # rotation angle pi


def test_random_starts_are_uniform_rotations():
    """Shoemake's method gives Haar-uniform rotations: E[R] = 0 and
    E[q q^T] = I/4 for the unit quaternion."""
    Rs = np.array([OA.random_rotation(seed=5, pair=p, s=4 + k) for p in range(500) for k in range(4)])
    np.testing.assert_allclose(Rs.mean(0), 0.0, atol=0.06)  # sd of a mean of 2000 entries ~ 0.013
    qs = np.array([OA.rot_to_quat(R) for R in Rs])
    np.testing.assert_allclose(np.einsum("ni,nj->ij", qs, qs) / len(qs), np.eye(4) / 4, atol=0.03)
    for R in Rs[:50]:
        np.testing.assert_allclose(OA.quat_to_rot(OA.rot_to_quat(R)), R, atol=1e-12)


def test_first_adam_step_moves_each_parameter_by_the_step_size(pair):
    a, b = pair
    pose0 = np.array([0.95, 0.2, -0.1, 0.2, 0.3, -0.2, 0.1])
    pose0[:4] /= np.linalg.norm(pose0[:4])
    traj = OA.adam(a, 0, b, 0, pose0, steps=1, objective=OA.OBJ_FO_CLOSED, lr=1e-3, lr_t=2e-3)
    _, g = O.fo_pose_grad(a, 0, b, 0, pose0)
    raw = pose0 + np.array([1e-3] * 4 + [2e-3] * 3) * np.sign(g)
    np.testing.assert_allclose(traj[1][4:], raw[4:], atol=1e-9)
    np.testing.assert_allclose(traj[1][:4], raw[:4] / np.linalg.norm(raw[:4]), atol=1e-9)


def test_adam_recovers_a_displaced_copy_on_the_closed_form(copy_pair):
    """From the exact superposition moved by 15 degrees and 0.6 A, 100 steps on
    the closed-form first-order overlap return to it (the overlap of a
    molecule with a rigid copy of itself is largest at the superposition)."""
    a, b, R, t = copy_pair
    p_true = OA.start_pose(OA.principal_frame(a, 0), OA.principal_frame(b, 0), 0)
    kick = Rotation.from_rotvec(np.radians(15) * np.array([0.6, 0.0, 0.8])).as_matrix()
    Rs = kick @ OA.quat_to_rot(p_true[:4])
    pose0 = np.concatenate([OA.rot_to_quat(Rs), p_true[4:] + np.array([0.6, 0.0, 0.0])])
    assert _rmsd(a, b, pose0) > 0.5
    traj = OA.adam(a, 0, b, 0, pose0, steps=100, objective=OA.OBJ_FO_CLOSED)
    assert _rmsd(a, b, traj[-1]) < 0.02


def test_finite_difference_gradient_matches_the_analytic_first_order_gradient(pair):
    """The CRN first-order objective with many points is an unbiased estimate
    of the closed form; its FD gradient (the oracle optimiser's gradient)
    agrees with the analytic one within sampling error."""
    a, b = pair
    ZQ = float(O.mixture_mass(a, [0])[0])
    g = np.array([OA.objective_grad(a, 0, b, 0, POSE, OA.OBJ_FO, OA.crn(a, 0, seed=2 + k, stream=0, n=1 << 16), ZQ)[1]
                  for k in range(8)])
    _, g_an = O.fo_pose_grad(a, 0, b, 0, POSE)
    z = (g.mean(0) - g_an) / (g.std(0, ddof=1) / np.sqrt(len(g)))
    assert np.all(np.abs(z) < 4.5), z
