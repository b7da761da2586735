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
