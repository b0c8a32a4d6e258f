"""Pins of the oracle's time-dependent terms (Section 2): the consistent
mass matrix integrates to rho x volume, the Robin traction of Eq. (bc epi)
on a flat face gives area x [(N x N) K_perp + (I - N x N) K_par] c for a
translation c, the damping part acts on the backward-Euler velocity, and
the tangent with inertia and Robin terms matches central differences."""
import numpy as np
import pytest

from oracle.assembly import FEProblem
from workloads import slab_problem

ROBIN = dict(k_perp=2.0e5, k_par=2.0e4, c_perp=1.0e4, c_par=2.0e3)


def _free_slab(order, **kw):
    prob = slab_problem(3, 2, 2, order=order, lengths=(1.5, 0.8, 0.7), parts=(1, 1, 1),
                        jitter=0.2, pressure=0.0, gamma=0.0, **kw)
    prob["dirichlet_nodes"] = np.zeros(0, dtype=np.int32)
    return prob


def _top_faces(prob):
    nx, ny, nz = 3, 2, 2
    return np.array([[(nz - 1) * nx * ny + j * nx + i, 5, 0] for j in range(ny) for i in range(nx)])


@pytest.mark.parametrize("order", [1, 2])
def test_mass_matrix_integrates_to_rho_volume(order):
    prob = _free_slab(order)
    prob["rho"] = 1060.0
    fe = FEProblem(prob)
    dt = 1e-3
    c = np.array([0.3, -0.2, 0.5])
    d = np.tile(c, fe.n_free // 3)              # a translation: F = I, P = 0
    zero = np.zeros(fe.n_free)
    fe.set_time_state(dt, zero, zero)
    r = fe.residual(d, 1.0).reshape(-1, 3)
    vol = 1.5 * 0.8 * 0.7
    assert np.allclose(r.sum(0), 1060.0 / dt ** 2 * vol * c, rtol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_robin_traction_on_a_flat_face(order):
    prob = _free_slab(order)
    prob["robin_faces"] = _top_faces(prob)
    prob["robin"] = [ROBIN]
    fe = FEProblem(prob)
    c = np.array([0.3, -0.2, 0.5])
    d = np.tile(c, fe.n_free // 3)
    area = 1.5 * 0.8                             # top face z = 0.7, normal +z
    N = np.array([0.0, 0.0, 1.0])
    want = area * (ROBIN["k_perp"] * (N @ c) * N + ROBIN["k_par"] * (c - (N @ c) * N))
    r = fe.residual(d, 1.0).reshape(-1, 3)
    assert np.allclose(r.sum(0), want, rtol=1e-12)
    # damping acts on (d - d_prev) / dt: with d_prev = d it adds nothing,
    # with d_prev = 0 it adds area [(N x N) C_perp + (I - N x N) C_par] c / dt
    dt = 2e-3
    fe.set_time_state(dt, d, d)
    assert np.allclose(fe.residual(d, 1.0).reshape(-1, 3).sum(0), want, rtol=1e-12)
    fe.set_time_state(dt, np.zeros_like(d), np.zeros_like(d))
    damp = area * (ROBIN["c_perp"] * (N @ c) * N + ROBIN["c_par"] * (c - (N @ c) * N)) / dt
    assert np.allclose(fe.residual(d, 1.0).reshape(-1, 3).sum(0), want + damp, rtol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_time_dependent_tangent_matches_residual_differences(order):
    prob = slab_problem(3, 2, 2, order=order, parts=(1, 1, 1), jitter=0.15,
                        pressure=2.0e3, gamma=3.0e4)
    prob["rho"] = 1000.0
    prob["robin_faces"] = _top_faces(prob)
    prob["robin"] = [ROBIN]
    fe = FEProblem(prob)
    rng = np.random.default_rng(4)
    d, dp, dpp = (0.01 * rng.standard_normal(fe.n_free) for _ in range(3))
    fe.set_time_state(1e-3, dp, dpp)
    K, _ = fe.tangent(d, 0.7)
    for _ in range(2):
        v = rng.standard_normal(fe.n_free)
        eps = 1e-6 * np.linalg.norm(d) / np.linalg.norm(v)
        fd = (fe.residual(d + eps * v, 0.7) - fe.residual(d - eps * v, 0.7)) / (2 * eps)
        assert np.linalg.norm(K @ v - fd) <= 1e-7 * np.linalg.norm(K @ v)
