"""Pins of the oracle's projective algebra against closed-form algebra and library
routines (SVD null spaces, numpy inverses, scipy rotations) -- never against the
oracle itself.  Eq. numbers refer to arXiv 1806.02637."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

import synth
from oracle import oracle as orc

RNG = np.random.default_rng(20240611)


def _null(A):
    """Right null vector of A (library SVD)."""
    return np.linalg.svd(A)[2][-1]


def _rand_P(rng):
    """A random camera P = K [R | -R C] with det M > 0."""
    R = Rotation.random(random_state=int(rng.integers(1 << 30))).as_matrix()
    C = rng.normal(0, 500, 3)
    K = np.array([[rng.uniform(800, 3000), rng.normal(0, 5), rng.uniform(100, 600)],
                  [0, rng.uniform(800, 3000), rng.uniform(100, 600)], [0, 0, 1]])
    return K @ np.hstack([R, (-R @ C)[:, None]]), C


@pytest.mark.parametrize("trial", range(20))
def test_meet_dual_incidence(trial):
    """Eq. (4)/(5) with the sign reading: x = L_K p lies on a, b and p."""
    a, b, p = RNG.standard_normal((3, 4))
    x = orc.dual(orc.meet(a, b), corrected=True) @ p
    scale = np.linalg.norm(x) * max(np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(p))
    assert abs(a @ x) <= 1e-13 * scale
    assert abs(b @ x) <= 1e-13 * scale
    assert abs(p @ x) <= 1e-13 * scale
    # x is the (unique) common point of the three planes: library null vector
    n = _null(np.stack([a, b, p]))
    assert np.linalg.norm(np.cross(x[:3] * n[3] - n[:3] * x[3], [1, 0, 0])) <= 1e-10 * scale
    assert abs(abs(x @ n) / np.linalg.norm(x) - 1.0) <= 1e-12


def test_printed_sign_fails_incidence():
    """Eq. (5) exactly as printed does not annihilate the planes of the meet; this
    is why the oracle takes the sign reading (p enters with the opposite sign)."""
    a, b = RNG.standard_normal((2, 4))
    K = orc.dual(orc.meet(a, b), corrected=False)
    assert np.linalg.norm(K @ a) > 1e-3 * np.linalg.norm(a) ** 2 * np.linalg.norm(b)
    Kc = orc.dual(orc.meet(a, b), corrected=True)
    assert np.linalg.norm(Kc @ a) <= 1e-13 * np.linalg.norm(a) ** 2 * np.linalg.norm(b)
    assert np.linalg.norm(Kc @ b) <= 1e-13 * np.linalg.norm(b) ** 2 * np.linalg.norm(a)
    assert np.allclose(Kc, -Kc.T)


def test_meet_components():
    """Eq. (4) for axis-aligned planes: z = 0 meet y = 0 is the x axis."""
    L = orc.meet([0, 0, 1, 0], [0, 1, 0, 0])
    # p = az bw - aw bz = 0, q = ay bw - aw by = 0, r = ay bz - az by = -1, s = t = u = 0
    assert np.allclose(L, [0, 0, -1, 0, 0, 0])
    # the dual matrix maps the plane x = 1 (1,0,0,-1) to the point (1, 0, 0, 1)
    x = orc.dual(L) @ np.array([1.0, 0, 0, -1])
    assert np.allclose(x / x[3], [1, 0, 0, 1])


@pytest.mark.parametrize("trial", range(10))
def test_source_is_null_vector(trial):
    """Source from the rows of P (meet construction): P X = 0, equal to the SVD null vector."""
    P, C = _rand_P(RNG)
    X = orc.source(P)
    assert np.linalg.norm(P @ X) <= 1e-9 * np.linalg.norm(P) * np.linalg.norm(X)
    assert np.allclose(X[:3] / X[3], C, rtol=0, atol=1e-8 * (1 + np.abs(C).max()))
    n = _null(P)
    assert abs(abs(X @ n) / np.linalg.norm(X) - 1) < 1e-12


def test_trajectory_sources():
    cfg = synth.CONFIGS["c2"]
    P = synth.trajectory(cfg)
    th = synth.view_angles(cfg)
    for i in (0, 100, 495):
        v = orc.view_setup(P[i])
        assert np.allclose(v["C"], cfg.sid * np.array([np.cos(th[i]), np.sin(th[i]), 0]), atol=1e-9)
        assert np.allclose(v["up"], [0, 0, -1], atol=1e-12)


@pytest.mark.parametrize("trial", range(20))
def test_line_inf_equals_cofactor_and_pinv(trial):
    """Eq. (13)/(14) give l = cof(M) n = det(M) P^{+T} E for any plane E through the
    source (the paper's claim that both algorithms give the same lines)."""
    P, C = _rand_P(RNG)
    n = RNG.standard_normal(3)
    E = np.append(n, -n @ C)
    l_inf = orc.line_inf(P, E)
    M = P[:, :3]
    cof = np.linalg.det(M) * np.linalg.inv(M).T          # library inverse, independent
    assert np.allclose(l_inf, cof @ n, rtol=1e-10, atol=1e-10 * np.abs(cof @ n).max())
    l_lib = np.linalg.pinv(P).T @ E                       # library (SVD) pseudo-inverse
    assert np.allclose(l_inf, np.linalg.det(M) * l_lib, rtol=1e-9, atol=1e-9 * np.abs(l_inf).max())
    # the literal normal-equation form P^T (P P^T)^{-1} is only as accurate as
    # cond(P P^T) allows (about 1e12 for raw camera matrices)
    l_pinv = orc.line_pinv(P, E)
    tol = 50 * np.finfo(float).eps * np.linalg.cond(P @ P.T)
    assert np.linalg.norm(l_pinv - l_lib) <= tol * np.linalg.norm(l_lib)
    # the line back-projects to E: P^T l is proportional to E
    bp = P.T @ l_inf
    assert np.linalg.norm(np.cross(bp[:3], E[:3])) <= 1e-9 * np.linalg.norm(bp[:3]) * np.linalg.norm(E[:3])


def test_line_transform_rule():
    """Eq. (12): the dual matrix of the transformed line is T L_K T^T, where the line
    is the meet of the planes transformed by Eq. (9)."""
    a, b = RNG.standard_normal((2, 4))
    T = np.eye(4)
    T[:3, :3] = Rotation.random(random_state=3).as_matrix() * 1.7
    T[:3, 3] = RNG.normal(0, 10, 3)
    Ti = np.linalg.inv(T).T
    K1 = orc.dual(orc.meet(Ti @ a, Ti @ b))
    K2 = T @ orc.dual(orc.meet(a, b)) @ T.T
    ratio = K1[np.abs(K2) > 1e-6] / K2[np.abs(K2) > 1e-6]
    assert np.allclose(ratio, ratio[0], rtol=1e-9)


def test_apply_motion_matches_library_rotation():
    """P' = P T(theta) with R = Rz Ry Rx (scipy intrinsic ZYX)."""
    P, _ = _rand_P(RNG)
    th = np.array([0.01, -0.02, 0.03, 1.0, -2.0, 3.0])
    R = Rotation.from_euler("ZYX", th[2::-1]).as_matrix()
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = th[3:]
    assert np.allclose(orc.apply_motion(P, th), P @ T, rtol=1e-12, atol=1e-9)


def test_view_setup_normalisation():
    P, C = _rand_P(RNG)
    for sigma in (-3.0, 0.5, 1e3):
        v = orc.view_setup(sigma * P)
        assert np.isclose(np.linalg.norm(v["P"][2, :3]), 1.0)
        assert np.linalg.det(v["P"][:, :3]) > 0
        assert np.allclose(v["C"], C, atol=1e-8 * (1 + np.abs(C).max()))
