"""Pins of the oracle's quaternion algebra (Appendix A.2, A.4).

The oracle's product and rotation are checked against hand-worked values
(tests/golden), against Lemma MW, against scipy's rotation routines and
against the closed-form distance identities of Appendix A.4.
"""
import os

import numpy as np
import pytest

import oracle
from oracle import matrix_form as mf

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(x) for x in line.split()])
    return np.array(rows)


def test_unit_products_golden():
    """Hamilton's table, worked out from the product rule of Appendix A.2."""
    for r in _rows("quaternion_units.txt"):
        a, b, ab = r[:4], r[4:8], r[8:12]
        np.testing.assert_array_equal(oracle.qmul(a, b), ab)


def test_rotation_golden():
    """R(q) v for q = [cos(theta/2), sin(theta/2) n], values worked by hand."""
    for r in _rows("rotations.txt"):
        n = r[:3] / np.linalg.norm(r[:3])
        th = np.deg2rad(r[3])
        q = np.concatenate([[np.cos(th / 2)], np.sin(th / 2) * n])
        np.testing.assert_allclose(oracle.qrotate(q, r[4:7]), r[7:10], atol=1e-15)


def test_lemma_mw():
    """Lemma MW: ab = M(a) b = W(b) a; M(a*) = M(a)^T; W(a*) = W(a)^T;
    M(a)^T M(a) = W(a)^T W(a) = |a|^2 I."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        ab = oracle.qmul(a, b)
        np.testing.assert_allclose(mf.M(a) @ b, ab, rtol=0, atol=1e-14)
        np.testing.assert_allclose(mf.W(b) @ a, ab, rtol=0, atol=1e-14)
        ac = a * np.array([1, -1, -1, -1])
        np.testing.assert_array_equal(mf.M(ac), mf.M(a).T)
        np.testing.assert_array_equal(mf.W(ac), mf.W(a).T)
        n2 = a @ a
        np.testing.assert_allclose(mf.M(a).T @ mf.M(a), n2 * np.eye(4), atol=1e-13)
        np.testing.assert_allclose(mf.W(a).T @ mf.W(a), n2 * np.eye(4), atol=1e-13)
        # D a = a^*, used to write p^* as D p in Appendix B
        np.testing.assert_array_equal(mf.D @ a, ac)


def test_product_associative_and_norm_multiplicative():
    rng = np.random.default_rng(1)
    for _ in range(100):
        a, b, c = rng.standard_normal((3, 4))
        np.testing.assert_allclose(oracle.qmul(oracle.qmul(a, b), c), oracle.qmul(a, oracle.qmul(b, c)),
                                   atol=1e-13)
        np.testing.assert_allclose(np.linalg.norm(oracle.qmul(a, b)),
                                   np.linalg.norm(a) * np.linalg.norm(b), rtol=1e-14)


def _rotmat(q):
    return np.stack([oracle.qrotate(q, e) for e in np.eye(3)], axis=1)


def test_rotation_matrix_properties_and_scipy():
    """R(q) is orthonormal with det +1 and equals scipy's matrix of q
    (scipy stores quaternions scalar last)."""
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(2)
    for _ in range(100):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        R = _rotmat(q)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-14
        ref = Rot.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-14)


def test_axis_angle_formula():
    """R = cos(th) I + (1 - cos(th)) n n^T + sin(th) n^  (Appendix A.2)."""
    rng = np.random.default_rng(3)
    for _ in range(100):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        th = rng.uniform(-np.pi, np.pi)
        q = np.concatenate([[np.cos(th / 2)], np.sin(th / 2) * n])
        hat = np.array([[0, -n[2], n[1]], [n[2], 0, -n[0]], [-n[1], n[0], 0]])
        R = np.cos(th) * np.eye(3) + (1 - np.cos(th)) * np.outer(n, n) + np.sin(th) * hat
        np.testing.assert_allclose(_rotmat(q), R, atol=1e-14)


def test_distance_identities():
    """Appendix A.4: |R1 - R2|_F = 2 sqrt(2) sin(theta/2) and
    |q1 - q2| = 2 sin(theta/4) for the closer sign, theta the geodesic angle."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        q1, q2 = rng.standard_normal((2, 4))
        q1 /= np.linalg.norm(q1)
        q2 /= np.linalg.norm(q2)
        R1, R2 = _rotmat(q1), _rotmat(q2)
        th = np.arccos(np.clip((np.trace(R1.T @ R2) - 1) / 2, -1, 1))
        assert abs(np.linalg.norm(R1 - R2) - 2 * np.sqrt(2) * np.sin(th / 2)) < 1e-12
        dq = min(np.linalg.norm(q1 - q2), np.linalg.norm(q1 + q2))
        assert abs(dq - 2 * np.sin(th / 4)) < 1e-7  # arccos loses precision near 0
