"""Guccione passive law plus active stress along fibres (Section 2).

All functions are vectorised over leading axes: F has shape (..., 3, 3),
R = [f | s | n] (..., 3, 3) holds the fibre frame as columns, and ``par``
is the material dictionary of ``workloads.material``.

* Kinematics: F = I + grad d, J = det F, E = (F^T F - I)/2.
* E_ab = (E a) . b for a, b in {f, s, n}.
* Q = b_ff E_ff^2 + b_ss E_ss^2 + b_nn E_nn^2 + b_fs (E_fs^2 + E_sf^2)
      + b_fn (E_fn^2 + E_nf^2) + b_sn (E_sn^2 + E_ns^2).
* Psi = C/2 (exp(Q) - 1) + B/2 (J - 1) log J,   P_pas = dPsi/dF.
* P_act = gamma (F f) (x) f / |F f|  (= d/dF of gamma |F f|).
"""
import numpy as np


def weight_matrix(par):
    """Symmetric 3x3 weights W with Q = sum_ab W_ab E_ab^2 in the fibre
    frame (ordering f, s, n)."""
    return np.array([
        [par["bff"], par["bfs"], par["bfn"]],
        [par["bfs"], par["bss"], par["bsn"]],
        [par["bfn"], par["bsn"], par["bnn"]],
    ])


def green_lagrange(F):
    I = np.eye(3)
    return 0.5 * (np.swapaxes(F, -1, -2) @ F - I)


def fiber_frame_strain(F, R):
    """E' = R^T E R, so E'_ab = (E a) . b."""
    E = green_lagrange(F)
    return np.swapaxes(R, -1, -2) @ E @ R


def q_value(F, R, par):
    Ep = fiber_frame_strain(F, R)
    W = weight_matrix(par)
    return np.sum(W * Ep * Ep, axis=(-1, -2))


def psi(F, R, par, gamma=0.0):
    """Strain energy density, including the active potential gamma |F f| so
    that the whole first Piola stress is its F-derivative."""
    Q = q_value(F, R, par)
    J = np.linalg.det(F)
    f = R[..., :, 0]
    Ff = np.einsum("...ij,...j->...i", F, f)
    return (0.5 * par["C"] * (np.exp(Q) - 1.0)
            + 0.5 * par["B"] * (J - 1.0) * np.log(J)
            + gamma * np.linalg.norm(Ff, axis=-1))


def second_pk_passive(F, R, par):
    """S = dPsi_iso/dE = C e^Q R (W o E') R^T  (from dQ/dE = 2 R (W o E') R^T)."""
    Ep = fiber_frame_strain(F, R)
    W = weight_matrix(par)
    Q = np.sum(W * Ep * Ep, axis=(-1, -2))
    Shat = R @ (W * Ep) @ np.swapaxes(R, -1, -2)
    return par["C"] * np.exp(Q)[..., None, None] * Shat, Q, Shat


def kappa(J, par):
    """J U'(J) for U = B/2 (J-1) log J:  B/2 (J log J + J - 1)."""
    return 0.5 * par["B"] * (J * np.log(J) + J - 1.0)


def dkappa(J, par):
    """d kappa / dJ = B/2 (log J + 2)."""
    return 0.5 * par["B"] * (np.log(J) + 2.0)


def first_pk(F, R, par, gamma=0.0):
    """P = F S + kappa(J) F^{-T} + gamma (F f)(x) f / |F f|."""
    S, _, _ = second_pk_passive(F, R, par)
    J = np.linalg.det(F)
    FinvT = np.swapaxes(np.linalg.inv(F), -1, -2)
    P = F @ S + kappa(J, par)[..., None, None] * FinvT
    if gamma != 0.0:
        f = R[..., :, 0]
        Ff = np.einsum("...ij,...j->...i", F, f)
        nrm = np.linalg.norm(Ff, axis=-1)
        P = P + gamma * np.einsum("...i,...j->...ij", Ff / nrm[..., None], f)
    return P


def tangent(F, R, par, gamma=0.0):
    """A_iJkL = dP_iJ / dF_kL in closed form, shape (..., 3, 3, 3, 3).

    Material part: delta_ik S_LJ + F_iM Csym_MJNL F_kN, with
      C_MJNL = C e^Q [ 2 Shat_MJ Shat_NL + sum_ab R_Ma R_Jb W_ab R_Na R_Lb ]
    symmetrised in (N, L) because only the symmetric part of dE acts.
    Volumetric part: J kappa'(J) Finv_Lk Finv_Ji - kappa Finv_Jk Finv_Li.
    Active part: gamma/|Ff| (delta_ik - m_i m_k) f_J f_L, m = Ff/|Ff|.
    """
    S, Q, Shat = second_pk_passive(F, R, par)
    W = weight_matrix(par)
    eQ = par["C"] * np.exp(Q)
    I = np.eye(3)
    lin = np.einsum("...Ma,...Jb,ab,...Na,...Lb->...MJNL", R, R, W, R, R)
    Cm = eQ[..., None, None, None, None] * (
        2.0 * np.einsum("...MJ,...NL->...MJNL", Shat, Shat) + lin)
    Cs = 0.5 * (Cm + np.swapaxes(Cm, -1, -2))
    A = np.einsum("ik,...LJ->...iJkL", I, S)
    A = A + np.einsum("...iM,...MJNL,...kN->...iJkL", F, Cs, F)
    J = np.linalg.det(F)
    Finv = np.linalg.inv(F)
    A = A + (J * dkappa(J, par))[..., None, None, None, None] * np.einsum(
        "...Lk,...Ji->...iJkL", Finv, Finv)
    A = A - kappa(J, par)[..., None, None, None, None] * np.einsum(
        "...Jk,...Li->...iJkL", Finv, Finv)
    if gamma != 0.0:
        f = R[..., :, 0]
        Ff = np.einsum("...ij,...j->...i", F, f)
        nrm = np.linalg.norm(Ff, axis=-1)
        m = Ff / nrm[..., None]
        proj = I - np.einsum("...i,...k->...ik", m, m)
        A = A + (gamma / nrm)[..., None, None, None, None] * np.einsum(
            "...ik,...J,...L->...iJkL", proj, f, f)
    return A


def slab_helix_frame(z, z0, z1, alpha0, alpha1):
    """Fibre frame of the slab workloads: the fibre angle rises linearly in
    the reference height z from alpha0 at z0 to alpha1 at z1,
    f = (cos a, sin a, 0), s = (-sin a, cos a, 0), n = e_z.  Returns R with
    columns f, s, n, shape (..., 3, 3)."""
    t = (np.asarray(z) - z0) / (z1 - z0)
    a = alpha0 + (alpha1 - alpha0) * t
    c, s = np.cos(a), np.sin(a)
    R = np.zeros(np.shape(a) + (3, 3))
    R[..., 0, 0] = c
    R[..., 1, 0] = s
    R[..., 0, 1] = -s
    R[..., 1, 1] = c
    R[..., 2, 2] = 1.0
    return R


def nodal_fiber_frame(f, n):
    """Fibre frame from interpolated nodal directions (the left-ventricle
    workloads): f normalised, n made orthogonal to f by one Gram-Schmidt
    step and normalised, s = n x f so that (f, s, n) is right-handed.
    Returns R with columns f, s, n, shape (..., 3, 3)."""
    f = f / np.linalg.norm(f, axis=-1, keepdims=True)
    n = n - np.sum(n * f, axis=-1, keepdims=True) * f
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    s = np.cross(n, f)
    return np.stack([f, s, n], axis=-1)


def fiber_frame(spec, X):
    """Fibre frame at reference points X (..., 3) from the analytic spec."""
    if spec["kind"] == "slab_helix":
        return slab_helix_frame(X[..., 2], spec["z0"], spec["z1"],
                                spec["alpha0"], spec["alpha1"])
    raise ValueError("unknown fibre spec %r" % spec["kind"])
