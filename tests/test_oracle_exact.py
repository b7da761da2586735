"""Pins for the oracle's exact targets: the first-order closed form (Eq. fo),
the inclusion-exclusion union series (Eq. incexc) and midpoint grid
quadrature of Eq. union-overlap, checked against each other, against
textbook closed forms and against the paper's hard-sphere normalisation
(Eq. occ: a single occupancy integrates to the sphere volume)."""
import json
import os

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import oracle as O
from paper_2607_20766_b300 import synth
from paper_2607_20766_b300.synth import MolSet

KAPPA = np.pi * (3 / (4 * np.pi)) ** (2 / 3)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def one_atom(R, p=None, xyz=(0.0, 0.0, 0.0)):
    return MolSet(np.array([xyz], np.float32), np.array([R], np.float32), np.array([0, 1], np.int32),
                  np.zeros(1, np.uint8), None if p is None else np.array([p], np.float32))


def test_kappa_constant_matches_alpha_convention():
    """alpha = 2.41798793 / R^2 with height 2 sqrt 2 is lambda = 1/2 of Eq. occ."""
    assert abs(2 * KAPPA - 2.41798793) < 1e-8


@pytest.mark.parametrize("R", [1.52, 1.55, 1.70, 1.80])
def test_single_atom_volume_is_sphere(R):
    R = float(np.float32(R))  # radii are stored as float32
    sphere = 4.0 / 3.0 * np.pi * R ** 3
    # height 2 sqrt 2, alpha = 2 kappa / R^2
    V = O.union_volume_ie(one_atom(R), 0)
    assert V == pytest.approx(sphere, rel=1e-8)
    # unit height, alpha = kappa / R^2 (Eq. occ with lambda = 1)
    V1 = O.union_volume_ie(one_atom(R, p=1.0), 0, c_alpha=KAPPA)
    assert V1 == pytest.approx(sphere, rel=1e-12)
    g = O.grid(one_atom(R), 0, h=0.1)
    assert g["VA"] == pytest.approx(sphere, rel=1e-8)
    assert g["ZA"] == pytest.approx(sphere, rel=1e-8)


def test_two_atom_union_is_textbook():
    """V = v1 + v2 - integral g1 g2, the product of two Gaussians being a
    Gaussian (Gaussian product theorem)."""
    ms = MolSet(np.array([[0, 0, 0], [1.3, 0.4, -0.2]], np.float32), np.array([1.7, 1.52], np.float32),
                np.array([0, 2], np.int32), np.zeros(2, np.uint8))
    p = 2 * np.sqrt(2)
    a = 2.41798793 / ms.radius.astype(np.float64) ** 2
    d2 = float(np.sum(ms.xyz[1].astype(np.float64) ** 2))
    v = p * (np.pi / a) ** 1.5
    cross = p * p * (np.pi / a.sum()) ** 1.5 * np.exp(-a[0] * a[1] / a.sum() * d2)
    assert O.union_volume_ie(ms, 0) == pytest.approx(v.sum() - cross, rel=1e-13)
    assert O.fo_overlap(ms, [0], ms, [0])[0] == pytest.approx(
        sum(p * p * (np.pi / (a[i] + a[j])) ** 1.5 * np.exp(-a[i] * a[j] / (a[i] + a[j]) * (d2 if i != j else 0))
            for i in range(2) for j in range(2)), rel=1e-13)


@pytest.fixture(scope="module")
def pair():
    return synth.single_pair()


@pytest.fixture(scope="module")
def grid_ab(pair):
    a, b = pair
    return O.grid(a, 0, b, 0, h=0.1, pad=6.5)


def test_inclusion_exclusion_matches_grid(pair, grid_ab):
    a, b = pair
    assert O.union_volume_ie(a, 0) == pytest.approx(grid_ab["VA"], rel=1e-10)
    assert O.union_volume_ie(b, 0) == pytest.approx(grid_ab["VB"], rel=1e-10)
    assert O.union_overlap_ie(a, 0, b, 0) == pytest.approx(grid_ab["OU"], rel=1e-10)
    assert O.union_overlap_ie(a, 0, a, 0) == pytest.approx(grid_ab["SA"], rel=1e-10)


def test_first_order_closed_form_matches_grid(pair, grid_ab):
    a, b = pair
    assert O.fo_overlap(a, [0], b, [0])[0] == pytest.approx(grid_ab["OFO"], rel=1e-10)
    assert O.mixture_mass(a)[0] == pytest.approx(grid_ab["ZA"], rel=1e-10)


def test_grid_is_converged(pair):
    a, b = pair
    g1 = O.grid(a, 0, b, 0, h=0.1, pad=6.5)
    g2 = O.grid(a, 0, b, 0, h=0.05, pad=7.0)
    for k in ("VA", "VB", "OU", "OFO"):
        assert g1[k] == pytest.approx(g2[k], rel=1e-11)


def test_union_identities(pair):
    """u_{A or B} = u_A + u_B - u_A u_B, so V(A+B) = V_A + V_B - O_AB; and
    the first-order model over-counts: O_FO > O_union (paper Sec. FO)."""
    a, b = pair
    both = a.concat(b)
    merged = MolSet(both.xyz, both.radius, np.array([0, both.n_atoms], np.int32), both.elem)
    VAB = O.grid(merged, 0, h=0.1)["VA"]
    VA, VB = O.union_volume_ie(a, 0), O.union_volume_ie(b, 0)
    OU = O.union_overlap_ie(a, 0, b, 0)
    assert VAB == pytest.approx(VA + VB - OU, rel=1e-10)
    assert O.fo_overlap(a, [0], b, [0])[0] > OU
    assert O.union_overlap_ie(a, 0, b, 0) == pytest.approx(O.union_overlap_ie(b, 0, a, 0), rel=1e-12)


def test_far_apart_molecules_are_additive(pair):
    a, b = pair
    far = MolSet(b.xyz + np.float32([60, 0, 0]), b.radius, b.offsets, b.elem)
    assert O.union_overlap_ie(a, 0, far, 0) < 1e-12
    assert O.fo_overlap(a, [0], far, [0])[0] < 1e-12


def test_pose_is_a_proper_rotation_plus_translation(pair):
    a, b = pair
    q = np.array([0.3, -0.5, 0.7, 0.2])
    q /= np.linalg.norm(q)
    t = np.array([0.4, -1.1, 0.25])
    pose = np.concatenate([q, t]).astype(np.float32)
    rot = Rotation.from_quat([pose[1], pose[2], pose[3], pose[0]])  # scipy is scalar-last
    moved = MolSet((rot.apply(b.xyz.astype(np.float64)) + pose[4:].astype(np.float64)).astype(np.float32),
                   b.radius, b.offsets, b.elem)
    fo_pose = O.fo_overlap(a, [0], b, [0], poses=pose[None])[0]
    fo_moved = O.fo_overlap(a, [0], moved, [0])[0]
    assert fo_pose == pytest.approx(fo_moved, rel=1e-6)
    ou_pose = O.union_overlap_ie(a, 0, b, 0, poseB=pose)
    assert ou_pose == pytest.approx(O.union_overlap_ie(a, 0, moved, 0), rel=1e-6)
    # unnormalised quaternion is normalised inside
    pose2 = pose.copy()
    pose2[:4] *= 3.0
    assert O.fo_overlap(a, [0], b, [0], poses=pose2[None])[0] == pytest.approx(fo_pose, rel=1e-6)


def test_occupancy_bounds_for_unit_heights():
    """For p <= 1: 0 <= u <= m, so the union weight w = u/m lies in [0, 1]
    (paper Sec. union, bounded reweighting)."""
    ms = synth.generate(8, [30])
    ms.height = np.full(ms.n_atoms, 1.0, np.float32)
    rng = np.random.default_rng(0)
    r = rng.normal(scale=3.0, size=(5000, 3))
    m, u = O.occupancy(ms, 0, r, c_alpha=KAPPA)
    # 1 - prod(1 - g) carries an absolute rounding error of ~1e-16
    assert np.all(u >= -1e-15) and np.all(u <= m * (1 + 1e-12) + 1e-15)
    sel = m > 1e-6
    w = u[sel] / m[sel]
    assert np.all((w >= 0) & (w <= 1 + 1e-9))


def test_occupancy_single_point_values():
    """At an atom centre far from others, m = u = p exactly."""
    ms = one_atom(1.7, xyz=(1.0, 2.0, 3.0))
    m, u = O.occupancy(ms, 0, np.array([[1.0, 2.0, 3.0], [1.0, 2.0, 4.0]]))
    assert m[0] == pytest.approx(2 * np.sqrt(2), rel=1e-15)
    assert u[0] == pytest.approx(2 * np.sqrt(2), rel=1e-15)
    assert m[1] == pytest.approx(2 * np.sqrt(2) * np.exp(-2.41798793 / float(np.float32(1.7)) ** 2), rel=1e-14)


def test_first_order_over_count_is_paper_scale():
    """Context check (not an exact pin): the paper reports first order
    over-counting the union by 3.2-3.6x for drug-like molecules (Sec.
    accuracy). Synthetic tree walks of drug-like size land in that region."""
    ms = synth.generate(21, [12, 14, 16])
    ratios = [O.fo_overlap(ms, [i], ms, [i])[0] / O.union_overlap_ie(ms, i, ms, i) for i in range(3)]
    assert all(2.5 < r < 4.5 for r in ratios)


def test_golden_single_pair_exact(pair):
    """Regression against values written by tests/golden/make_golden.py."""
    with open(os.path.join(GOLDEN, "single_pair_exact.json")) as f:
        g = json.load(f)
    a, b = pair
    assert O.union_volume_ie(a, 0) == pytest.approx(g["V_A"], rel=1e-12)
    assert O.union_volume_ie(b, 0) == pytest.approx(g["V_B"], rel=1e-12)
    assert O.union_overlap_ie(a, 0, b, 0) == pytest.approx(g["O_union_AB"], rel=1e-12)
    assert O.fo_overlap(a, [0], b, [0])[0] == pytest.approx(g["O_fo_AB"], rel=1e-12)
