"""Pins of the rigid-body primal constraints (Section 4: the near-null space
of elasticity, the rigid motions, taken into the BDDC primal space): the
constraint rows of a class span exactly the rigid motions restricted to it
(closed forms for a straight edge and a planar face, an SVD rank check
against the six modes written about the origin for jittered classes), BDDC
theory in the symmetric case (M^-1 symmetric, spectrum >= 1, and the largest
eigenvalue cannot grow when constraints are added), and the BDDC-GMRES
solve against a direct solve."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC, Classification, class_rotations
from oracle.krylov import gmres
from workloads import lv_problem, slab_problem


def _rank(M, rtol=1e-9):
    s = np.linalg.svd(np.atleast_2d(M), compute_uv=False)
    return int(np.sum(s > rtol * s[0])) if s.size and s[0] > 0 else 0


def _rigid_modes(X):
    """The six rigid motions at nodes X, written about the origin: three
    translations and u(x) = omega x x for omega = e_x, e_y, e_z."""
    m = len(X)
    cols = []
    for c in range(3):
        t = np.zeros((m, 3))
        t[:, c] = 1.0
        cols.append(t.reshape(-1))
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    zero = np.zeros(m)
    cols.append(np.stack([zero, -z, y], axis=1).reshape(-1))   # e_x cross x
    cols.append(np.stack([z, zero, -x], axis=1).reshape(-1))   # e_y cross x
    cols.append(np.stack([-y, x, zero], axis=1).reshape(-1))   # e_z cross x
    return np.column_stack(cols)


def _class_rows(X):
    m = len(X)
    avg = np.zeros((3, 3 * m))
    for c in range(3):
        avg[c, c::3] = 1.0 / m
    return np.vstack([avg, class_rotations(X)])


def test_straight_edge_closed_form():
    # nodes at x = 0, 1, 2 on the x-axis: the rotations about y and z move
    # the nodes by -(x - 1) e_z and (x - 1) e_y; the rotation about x moves
    # nothing and is dropped
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    R = class_rotations(X)
    assert R.shape == (2, 9)
    want = np.zeros((2, 9))
    want[0, 2::3] = [1.0, 0.0, -1.0]
    want[1, 1::3] = [-1.0, 0.0, 1.0]
    want /= np.sqrt(2.0)
    # same row space (the basis inside it is free)
    assert np.allclose(R @ R.T, np.eye(2), atol=1e-14)
    assert np.allclose(want @ R.T @ R, want, atol=1e-14)


def test_planar_face_has_three_rotations():
    # unit square in the plane z = 0: in-plane rotation plus two tilts
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1, 0], [1.0, 1, 0]])
    R = class_rotations(X)
    assert R.shape == (3, 12)
    # the in-plane rotation about the centroid (0.5, 0.5) is in the span
    y = X - 0.5 * np.array([1.0, 1.0, 0.0])
    spin = np.stack([-y[:, 1], y[:, 0], np.zeros(4)], axis=1).reshape(-1)
    assert np.linalg.norm(spin - R.T @ (R @ spin)) <= 1e-14 * np.linalg.norm(spin)
    # a tilt about the x-axis through the centroid: u_z = y - 1/2
    tilt = np.stack([np.zeros(4), np.zeros(4), y[:, 1]], axis=1).reshape(-1)
    assert np.linalg.norm(tilt - R.T @ (R @ tilt)) <= 1e-14 * np.linalg.norm(tilt)


def test_single_node_has_no_rotation():
    assert class_rotations(np.array([[0.3, 0.2, 0.1]])).shape == (0, 3)


@pytest.mark.parametrize("kind", ["slab_jitter", "lv"])
def test_rows_span_the_restricted_rigid_modes(kind):
    if kind == "slab_jitter":
        prob = slab_problem(6, 6, 4, parts=(2, 2, 2), jitter=0.2)
    else:
        prob = lv_problem(nt=3, ntheta=12, nu=6, n_parts=6)
    fe = FEProblem(prob)
    cl = Classification(fe, prob["elem_part"], prob["n_parts"])
    assert cl.edges and cl.faces
    for cls in cl.edges + cl.faces:
        X = fe.coords[cls]
        C = _class_rows(X)
        B = _rigid_modes(X)
        rc, rb, rboth = _rank(C), _rank(B), _rank(np.hstack([C.T, B]))
        assert rc == C.shape[0]            # independent rows
        assert rc == rb == rboth           # same span as the rigid modes
        # rotations are orthonormal and orthogonal to the averages
        R = C[3:]
        if len(X) == 1:
            assert R.shape[0] == 0
            continue
        assert np.allclose(R @ R.T, np.eye(R.shape[0]), atol=1e-12)
        assert np.abs(C[:3] @ R.T).max() <= 1e-12


def _setup(prob):
    fe = FEProblem(prob)
    K, (Ke, Kf) = fe.tangent(np.zeros(fe.n_free), 1.0)
    return fe, K, Ke, Kf


def _spectrum(fe, K, pc):
    n = fe.n_free
    Minv = np.column_stack([pc.apply(e) for e in np.eye(n)])
    ev = np.linalg.eigvals(Minv @ K.toarray())
    return Minv, ev


@pytest.mark.parametrize("base", ["VE", "EF"])
def test_symmetric_case_with_rotations(base):
    # p = 0, gamma = 0, d = 0: SPD tangent.  Adding constraints shrinks the
    # constrained space, so lambda_max cannot grow, and lambda_min >= 1 holds
    # for every primal space whose constraints are the same on all subdomains
    # sharing a class.
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), jitter=0.15, pressure=0.0, gamma=0.0)
    fe, K, Ke, Kf = _setup(prob)
    pc0 = BDDC(fe, Ke, Kf, base)
    pc1 = BDDC(fe, Ke, Kf, base + "R")
    assert pc1.n_pi > pc0.n_pi
    M1, ev1 = _spectrum(fe, K, pc1)
    _, ev0 = _spectrum(fe, K, pc0)
    assert np.abs(M1 - M1.T).max() <= 1e-10 * np.abs(M1).max()
    assert np.abs(ev1.imag).max() <= 1e-8 * np.abs(ev1).max()
    assert ev1.real.min() >= 1.0 - 1e-9
    assert ev1.real.max() <= ev0.real.max() * (1.0 + 1e-9)


def test_rotations_on_the_ventricle_solve_matches_direct():
    prob = lv_problem(nt=3, ntheta=12, nu=6, n_parts=6, pressure=2.0e3, gamma=1.5e4)
    fe = FEProblem(prob)
    d = 1e-4 * np.random.default_rng(3).standard_normal(fe.n_free)
    K, (Ke, Kf) = fe.tangent(d, 1.0)
    r = np.random.default_rng(4).standard_normal(fe.n_free)
    x_ref = spla.spsolve(K.tocsc(), r)
    its = {}
    for primal in ("EF", "EFR"):
        pc = BDDC(fe, Ke, Kf, primal)
        x, its[primal], _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-12)
        assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    assert its["EFR"] <= its["EF"]


def test_rotations_refused_for_multilevel():
    prob = slab_problem(4, 4, 2, parts=(2, 2, 1), pressure=0.0, gamma=0.0)
    fe, K, Ke, Kf = _setup(prob)
    with pytest.raises(ValueError):
        BDDC(fe, Ke, Kf, "VER", level2=dict(part=np.zeros(4, dtype=int), n_parts=1))
