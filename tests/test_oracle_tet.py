"""Pins of the oracle's tetrahedral elements (P1, P2) and of the ventricle
workload: quadrature exactness against the closed-form monomial integrals,
nodal interpolation, the patch test, the pressure resultant on the
endocardium (p times the area of the base opening, by the divergence
theorem), the fibre frame and the tangent against finite differences."""
from math import factorial

import numpy as np
import pytest

from oracle import elements as el
from oracle import material as mat
from oracle.assembly import FEProblem
from oracle.bddc import outer_boundary_nodes
from workloads import lv_problem
from workloads.lv import ring_sizes


def _tet_monomial(a, b, c):
    # int over the unit tetrahedron of x^a y^b z^c = a! b! c! / (a+b+c+3)!
    return factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 3)


@pytest.mark.parametrize("k", [1, 2])
def test_tet_rules_integrate_monomials(k):
    P, W = el.tet_volume_rule(k)
    for a in range(k + 1):
        for b in range(k + 1 - a):
            for c in range(k + 1 - a - b):
                got = np.sum(W * P[:, 0] ** a * P[:, 1] ** b * P[:, 2] ** c)
                assert np.isclose(got, _tet_monomial(a, b, c), rtol=1e-14, atol=0)
    st, w = el.tri_rule(k)
    for a in range(k + 1):
        for b in range(k + 1 - a):
            got = np.sum(w * st[:, 0] ** a * st[:, 1] ** b)
            want = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert np.isclose(got, want, rtol=1e-14, atol=0)


@pytest.mark.parametrize("k", [1, 2])
def test_tet_shape_functions(k):
    nodes = el.tet_nodes(k)
    N, dN = el.tet_shape(k, nodes)
    assert np.allclose(N, np.eye(nodes.shape[0]), atol=1e-14)
    x = np.random.default_rng(0).dirichlet(np.ones(4), 9)[:, 1:]
    N, dN = el.tet_shape(k, x)
    assert np.allclose(N.sum(1), 1.0)
    assert np.allclose(dN.sum(1), 0.0, atol=1e-13)
    assert np.allclose(N @ nodes, x)                      # linear reproduction
    if k == 2:                                            # quadratic reproduction
        assert np.allclose(N @ (nodes[:, 0] * nodes[:, 2]), x[:, 0] * x[:, 2])
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (el.tet_shape(k, x + e)[0] - el.tet_shape(k, x - e)[0]) / (2 * h)
        assert np.allclose(dN[:, :, j], fd, atol=1e-8)


@pytest.mark.parametrize("k", [1, 2])
def test_tet_face_rules(k):
    for f in range(4):
        pts, w, es, et = el.tet_face_rule(k, f)
        L = np.column_stack([1.0 - pts.sum(1), pts])
        assert np.allclose(L[:, f], 0.0)                  # on the face opposite f
        nrm = np.cross(es, et)
        cen = np.delete(el.TET_VERTS, f, axis=0).mean(0)
        assert nrm @ (cen - el.TET_VERTS[f]) > 0          # outward
        fn = el.tet_face_nodes(k, f)
        N, _ = el.tet_shape(k, pts)
        other = [a for a in range(N.shape[1]) if a not in fn]
        assert np.allclose(N[:, other], 0.0, atol=1e-14)  # only face nodes live there
        assert np.isclose(w.sum(), 0.5)


def test_nodal_fiber_frame():
    rng = np.random.default_rng(1)
    f = rng.standard_normal((20, 3))
    n = rng.standard_normal((20, 3))
    R = mat.nodal_fiber_frame(f, n)
    assert np.allclose(np.einsum("qji,qjk->qik", R, R), np.eye(3), atol=1e-13)
    assert np.allclose(np.linalg.det(R), 1.0)
    assert np.allclose(R[:, :, 0], f / np.linalg.norm(f, axis=1)[:, None])
    # reduces to the slab frame for f in the x-y plane and n = e_z
    a = rng.uniform(-1, 1, 7)
    fs = np.column_stack([np.cos(a), np.sin(a), 0 * a])
    Rn = mat.nodal_fiber_frame(fs, np.tile([0.0, 0.0, 1.0], (7, 1)))
    Rs = mat.slab_helix_frame(a, 0.0, 1.0, 0.0, 1.0)
    assert np.allclose(Rn, Rs, atol=1e-14)


def _small_lv(k, **kw):
    base = dict(nt=3, ntheta=10, nu=5, order=k, n_parts=1)
    base.update(kw)
    return lv_problem(**base)


def test_lv_mesh_is_valid():
    for k in (1, 2):
        prob = _small_lv(k, jitter=0.15)
        X, E = prob["coords"], prob["elems"]
        v = X[E[:, :4]]
        vol = np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]),
                        v[:, 3] - v[:, 0])
        assert vol.min() > 0
        # every interior face is shared by exactly two elements
        faces = {}
        for f in range(4):
            cn = [a for a in range(4) if a != f]
            for key in map(tuple, np.sort(E[:, cn], axis=1)):
                faces[key] = faces.get(key, 0) + 1
        assert max(faces.values()) == 2
        assert np.all(np.abs(X[prob["dirichlet_nodes"], 2]) < 1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_tet_patch_test(k):
    prob = _small_lv(k, jitter=0.15)
    prob["dirichlet_nodes"] = np.zeros(0, dtype=np.int32)
    prob["pressure_faces"] = np.zeros((0, 2), dtype=np.int32)
    nn = prob["coords"].shape[0]
    prob["fibers"] = {"kind": "nodal", "f": np.tile([0.6, 0.8, 0.0], (nn, 1)),
                      "n": np.tile([0.0, 0.3, 1.0], (nn, 1))}
    fe = FEProblem(prob)
    F0 = np.array([[1.05, 0.03, -0.02], [0.01, 0.97, 0.04], [-0.03, 0.02, 1.02]])
    u = fe.coords @ (F0 - np.eye(3)).T
    r = fe.residual(u.reshape(-1), 1.0).reshape(-1, 3)
    interior = ~outer_boundary_nodes(fe)
    assert interior.sum() > 10
    scale = np.abs(r).max()
    assert np.abs(r[interior]).max() <= 1e-11 * scale
    assert np.abs(r.sum(0)).max() <= 1e-11 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_lv_pressure_resultant(k):
    # At d = 0 with gamma = 0 the residual is the endocardial load.  The
    # endocardium and the base opening enclose the cavity, so the integral
    # of the outward tissue normal over the endocardium equals the area of
    # the (polygonal) opening times e_z.
    p, nth, nu, a = 1.7e3, 16, 5, 0.025
    prob = _small_lv(k, gamma=0.0, pressure=p, ntheta=nth, nu=nu, a_endo=a)
    prob["dirichlet_nodes"] = np.zeros(0, dtype=np.int32)
    fe = FEProblem(prob)
    r = fe.residual(np.zeros(fe.n_free), 1.0).reshape(-1, 3)
    nb = ring_sizes(nth, nu)[-1]                          # nodes on the base ring
    area = 0.5 * nb * a * a * np.sin(2 * np.pi / nb)
    assert np.allclose(r.sum(0), [0.0, 0.0, p * area], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("k", [1, 2])
def test_tet_tangent_matches_residual_differences(k):
    prob = _small_lv(k, pressure=2.0e3, gamma=3.0e4)
    fe = FEProblem(prob)
    rng = np.random.default_rng(3)
    Xs = fe.coords[fe.free_nodes]
    d = (1.5e-3 * np.sin(40 * Xs) + 2e-5 * rng.standard_normal(Xs.shape)).reshape(-1)
    K, _ = fe.tangent(d, 0.8)
    for _ in range(3):
        v = rng.standard_normal(fe.n_free)
        eps = 1e-6 * np.linalg.norm(d) / np.linalg.norm(v)
        fd = (fe.residual(d + eps * v, 0.8) - fe.residual(d - eps * v, 0.8)) / (2 * eps)
        kv = K @ v
        assert np.linalg.norm(kv - fd) <= 1e-7 * np.linalg.norm(kv)
