"""Pins of the oracle's constitutive law (Section 2) against facts that do
not come from the oracle itself: finite differences of the energy, frame
invariance, the stress-free reference state and the small-strain limit."""
import numpy as np
import pytest

from oracle import material as mat
from workloads import default_material

PAR = default_material()


def _rotation(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def _cases(n=6, seed=1):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        F = np.eye(3) + 0.25 * rng.standard_normal((3, 3))
        if np.linalg.det(F) < 0.3:
            F = np.eye(3) + 0.05 * rng.standard_normal((3, 3))
        R = _rotation(rng)
        yield F, R


@pytest.mark.parametrize("gamma", [0.0, 3.0e4])
def test_first_pk_is_energy_derivative(gamma):
    eps = 1e-6
    for F, R in _cases():
        P = mat.first_pk(F, R, PAR, gamma)
        Pfd = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                dF = np.zeros((3, 3))
                dF[i, j] = eps
                Pfd[i, j] = (mat.psi(F + dF, R, PAR, gamma)
                             - mat.psi(F - dF, R, PAR, gamma)) / (2 * eps)
        assert np.abs(P - Pfd).max() <= 1e-7 * np.abs(P).max()


@pytest.mark.parametrize("gamma", [0.0, 3.0e4])
def test_tangent_is_stress_derivative(gamma):
    eps = 1e-6
    for F, R in _cases(seed=2):
        A = mat.tangent(F, R, PAR, gamma)
        Afd = np.zeros((3, 3, 3, 3))
        for k in range(3):
            for l in range(3):
                dF = np.zeros((3, 3))
                dF[k, l] = eps
                Afd[:, :, k, l] = (mat.first_pk(F + dF, R, PAR, gamma)
                                   - mat.first_pk(F - dF, R, PAR, gamma)) / (2 * eps)
        assert np.abs(A - Afd).max() <= 1e-7 * np.abs(A).max()


def test_tangent_major_symmetry():
    # A = d^2 Psi / dF dF, so A_iJkL = A_kLiJ (the active part included).
    for F, R in _cases(seed=3):
        A = mat.tangent(F, R, PAR, 3.0e4)
        assert np.allclose(A, A.transpose(2, 3, 0, 1), rtol=0, atol=1e-9 * np.abs(A).max())


def test_frame_invariance():
    rng = np.random.default_rng(4)
    for F, R in _cases(seed=5):
        Qr = _rotation(rng)
        for g in (0.0, 3.0e4):
            assert np.isclose(mat.psi(Qr @ F, R, PAR, g), mat.psi(F, R, PAR, g),
                              rtol=1e-12, atol=1e-9)
            assert np.allclose(mat.first_pk(Qr @ F, R, PAR, g),
                               Qr @ mat.first_pk(F, R, PAR, g), rtol=1e-11, atol=1e-7)


def test_reference_state():
    R = _rotation(np.random.default_rng(6))
    I = np.eye(3)
    assert np.abs(mat.first_pk(I, R, PAR, 0.0)).max() == 0.0
    f = R[:, 0]
    assert np.allclose(mat.first_pk(I, R, PAR, 5.0), 5.0 * np.outer(f, f), atol=1e-12)


def test_small_strain_stiffness():
    # Psi ~ C/2 sum_ab W_ab eps'_ab^2 + B/2 (tr eps)^2 near F = I, so
    # eps : A(I) : eps = C sum W eps'^2 + B (tr eps)^2 for symmetric eps and
    # infinitesimal rotations cost nothing.
    rng = np.random.default_rng(7)
    R = _rotation(rng)
    A = mat.tangent(np.eye(3), R, PAR, 0.0)
    W = np.array([[PAR["bff"], PAR["bfs"], PAR["bfn"]],
                  [PAR["bfs"], PAR["bss"], PAR["bsn"]],
                  [PAR["bfn"], PAR["bsn"], PAR["bnn"]]])
    for _ in range(5):
        X = rng.standard_normal((3, 3))
        eps = 0.5 * (X + X.T)
        ep = R.T @ eps @ R
        want = PAR["C"] * np.sum(W * ep * ep) + PAR["B"] * np.trace(eps) ** 2
        got = np.einsum("iJ,iJkL,kL->", eps, A, eps)
        assert np.isclose(got, want, rtol=1e-12)
        skew = 0.5 * (X - X.T)
        assert abs(np.einsum("iJ,iJkL,kL->", skew, A, skew)) <= 1e-9 * abs(want)


def test_uniaxial_fibre_stretch_closed_form():
    # F = diag(l, 1, 1) along a fibre f = e_x with s = e_y, n = e_z:
    # E_ff = (l^2-1)/2, Q = b_ff E_ff^2, S_ff = C e^Q b_ff E_ff,
    # P_11 = l S_ff + B/2 (l log l + l - 1)/l + gamma.
    lam = 1.13
    F = np.diag([lam, 1.0, 1.0])
    R = np.eye(3)
    g = 1.7e4
    Eff = 0.5 * (lam ** 2 - 1)
    Q = PAR["bff"] * Eff ** 2
    want = (lam * PAR["C"] * np.exp(Q) * PAR["bff"] * Eff
            + 0.5 * PAR["B"] * (lam * np.log(lam) + lam - 1) / lam + g)
    P = mat.first_pk(F, R, PAR, g)
    assert np.isclose(P[0, 0], want, rtol=1e-13)
    assert abs(P[0, 1]) < 1e-9 and abs(P[1, 0]) < 1e-9


def test_slab_helix_frame():
    R = mat.slab_helix_frame(np.array([0.0, 0.5, 1.0]), 0.0, 1.0,
                             np.deg2rad(-60), np.deg2rad(60))
    for Rk in R:
        assert np.allclose(Rk.T @ Rk, np.eye(3), atol=1e-15)
        assert np.isclose(np.linalg.det(Rk), 1.0)
    assert np.allclose(R[0][:, 0], [0.5, -np.sqrt(3) / 2, 0])
    assert np.allclose(R[1][:, 0], [1, 0, 0])
    assert np.allclose(R[2][:, 0], [0.5, np.sqrt(3) / 2, 0])
