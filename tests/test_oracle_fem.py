"""Pins of the oracle's discretisation (Section 2): quadrature, patch test,
pressure resultant, tangent versus finite differences of the residual, and
quadratic Newton convergence."""
import numpy as np
import pytest

from oracle import elements as el
from oracle.assembly import FEProblem
from oracle.newton import newton_solve, direct_solver
from workloads import slab_problem


def test_gauss_rules_integrate_polynomials():
    for k in (1, 2):
        P, W = el.hex_volume_rule(k)
        deg = 2 * (k + 1) - 1
        for p in range(deg + 1):
            want = 0.0 if p % 2 else 2.0 / (p + 1) * 4.0
            assert np.isclose(np.sum(W * P[:, 0] ** p), want)


def test_shape_functions_partition_of_unity_and_nodal():
    for k in (1, 2):
        m = k + 1
        nodes = np.array([[-1 + 2 * a / k, -1 + 2 * b / k, -1 + 2 * c / k]
                          for c in range(m) for b in range(m) for a in range(m)])
        N, dN = el.hex_shape(k, nodes)
        assert np.allclose(N, np.eye(m ** 3), atol=1e-14)
        x = np.random.default_rng(0).uniform(-1, 1, (7, 3))
        N, dN = el.hex_shape(k, x)
        assert np.allclose(N.sum(1), 1.0)
        assert np.allclose(dN.sum(1), 0.0, atol=1e-13)
        # reproduces linear functions
        assert np.allclose(N @ nodes, x)
        assert np.allclose(np.einsum("qa,ai->qi", dN[:, :, 0], nodes[:, :]),
                           np.tile([1, 0, 0], (7, 1)), atol=1e-13)


def _patch_problem(k, jitter=0.25):
    prob = slab_problem(3, 3, 3, order=k, lengths=(1.0, 1.2, 0.9),
                        parts=(1, 1, 1), jitter=jitter, seed=11,
                        pressure=0.0, gamma=2.0e4, alpha_deg=(30.0, 30.0))
    prob["dirichlet_nodes"] = np.zeros(0, dtype=np.int32)
    return prob


@pytest.mark.parametrize("k", [1, 2])
def test_patch_test(k):
    # A homogeneous deformation gives constant P; interior nodal residuals
    # are P : sum_e int grad N_a = 0 on any (straight-sided) mesh.
    prob = _patch_problem(k)
    fe = FEProblem(prob)
    F0 = np.array([[1.05, 0.03, -0.02], [0.01, 0.97, 0.04], [-0.03, 0.02, 1.02]])
    u = fe.coords @ (F0 - np.eye(3)).T
    r = fe.residual(u.reshape(-1), 1.0).reshape(-1, 3)
    X = fe.coords
    interior = np.all((X > 1e-9) & (X < np.array([1.0, 1.2, 0.9]) - 1e-9), axis=1)
    assert interior.sum() > 0
    scale = np.abs(r).max()
    assert np.abs(r[interior]).max() <= 1e-11 * scale
    # and the total force vanishes (no pressure): sum_a int P grad N_a = 0
    assert np.abs(r.sum(0)).max() <= 1e-11 * scale


@pytest.mark.parametrize("k", [1, 2])
def test_pressure_resultant(k):
    # At d = 0 the stress vanishes (gamma = 0) and the residual is the
    # pressure load alone, whose resultant is p * area * e_z on the top face.
    p = 1234.5
    prob = slab_problem(3, 2, 2, order=k, lengths=(1.5, 0.8, 0.7), parts=(1, 1, 1),
                        jitter=0.2, pressure=p, gamma=0.0)
    prob["dirichlet_nodes"] = np.zeros(0, dtype=np.int32)
    fe = FEProblem(prob)
    r = fe.residual(np.zeros(fe.n_free), 1.0).reshape(-1, 3)
    assert np.allclose(r.sum(0), [0.0, 0.0, p * 1.5 * 0.8], rtol=1e-13, atol=1e-9)


@pytest.mark.parametrize("k", [1, 2])
def test_tangent_matches_residual_differences(k):
    prob = slab_problem(2, 3, 2, order=k, parts=(1, 1, 1), jitter=0.2,
                        pressure=2.0e3, gamma=3.0e4)
    fe = FEProblem(prob)
    rng = np.random.default_rng(3)
    d = 0.02 * rng.standard_normal(fe.n_free)
    K, _ = fe.tangent(d, 0.8)
    for _ in range(3):
        v = rng.standard_normal(fe.n_free)
        eps = 1e-6 * np.linalg.norm(d) / np.linalg.norm(v)
        fd = (fe.residual(d + eps * v, 0.8) - fe.residual(d - eps * v, 0.8)) / (2 * eps)
        kv = K @ v
        assert np.linalg.norm(kv - fd) <= 1e-7 * np.linalg.norm(kv)


def test_follower_pressure_is_nonsymmetric():
    prob = slab_problem(2, 2, 2, order=1, parts=(1, 1, 1), pressure=5.0e3, gamma=0.0)
    fe = FEProblem(prob)
    d = 0.03 * np.random.default_rng(5).standard_normal(fe.n_free)
    K, _ = fe.tangent(d, 1.0)
    asym = abs(K - K.T).max()
    assert asym > 1e-6 * abs(K).max()
    prob0 = dict(prob, pressure=0.0)
    fe0 = FEProblem(prob0)
    K0, _ = fe0.tangent(d, 1.0)
    assert abs(K0 - K0.T).max() <= 1e-12 * abs(K0).max()


def test_newton_converges_quadratically():
    prob = slab_problem(4, 4, 4, order=1, parts=(1, 1, 1), load_steps=2)
    d, log = newton_solve(prob, direct_solver, tol=1e-10)
    steps = [l for l in log if l["lam"] == 1.0]
    res = [s["res"] for s in steps] + [steps[-1]["res_new"]]
    assert len(steps) <= 6
    # estimated order log(r_{k+1}/r_k) / log(r_k/r_{k-1}) near 2
    orders = [np.log(res[i + 1] / res[i]) / np.log(res[i] / res[i - 1])
              for i in range(1, len(res) - 1)]
    assert max(orders) > 1.8
