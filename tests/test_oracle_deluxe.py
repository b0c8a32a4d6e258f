"""Pins of the deluxe scaling of the oracle's BDDC (Section 3.2 names it as
the more robust alternative to counting): the scaling matrices of a class
sum to the identity; with two subdomains sharing one face and no primal
constraint, BDDC with deluxe scaling is the exact inverse (the averaged
local inverses sum to the inverse of the assembled Schur complement), also
for the nonsymmetric tangent, while counting is not; BDDC theory in the
symmetric case (M^-1 symmetric, spectrum >= 1); and the BDDC-GMRES solve
against a direct solve, including a multilevel method."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC
from oracle.krylov import gmres
from workloads import box_groups, lv_problem, slab_problem


def _setup(prob, d_scale=0.0, lam=1.0, seed=0):
    fe = FEProblem(prob)
    d = d_scale * np.random.default_rng(seed).standard_normal(fe.n_free)
    K, (Ke, Kf) = fe.tangent(d, lam)
    return fe, K, Ke, Kf


def test_class_scalings_sum_to_identity():
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), jitter=0.15, pressure=1e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 1e-3)
    pc = BDDC(fe, Ke, Kf, "VE", scaling="deluxe")
    total = {}
    for sub in pc.subs:
        gdofG = sub["gdof"][sub["ldofG"]]
        for pos, D in sub["deluxe"]:
            key = tuple(gdofG[pos])
            total[key] = total.get(key, 0) + D
    assert len(total) == len(pc.cl.edges) + len(pc.cl.faces)
    for D in total.values():
        assert np.abs(D - np.eye(D.shape[0])).max() <= 1e-10


@pytest.mark.parametrize("pressure,gamma", [(0.0, 0.0), (2e3, 3e4)])
def test_two_subdomains_deluxe_is_exact(pressure, gamma):
    # split in x, both halves clamped at z = 0: one face, no vertices or
    # edges, so the primal space is empty and the local Neumann problems
    # are nonsingular
    prob = slab_problem(4, 3, 3, parts=(2, 1, 1), jitter=0.1, pressure=pressure, gamma=gamma)
    fe, K, Ke, Kf = _setup(prob, 2e-3)
    r = np.random.default_rng(1).standard_normal(fe.n_free)
    dlx = BDDC(fe, Ke, Kf, "V", scaling="deluxe")
    assert dlx.n_pi == 0 and len(dlx.cl.faces) == 1
    z = dlx.apply(r)
    assert np.linalg.norm(K @ z - r) <= 1e-10 * np.linalg.norm(r)
    cnt = BDDC(fe, Ke, Kf, "V")
    assert np.linalg.norm(K @ cnt.apply(r) - r) > 1e-3 * np.linalg.norm(r)


@pytest.mark.parametrize("primal", ["VE", "VEF"])
def test_symmetric_case_spectrum_deluxe(primal):
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), jitter=0.15, pressure=0.0, gamma=0.0)
    fe, K, Ke, Kf = _setup(prob)
    pc = BDDC(fe, Ke, Kf, primal, scaling="deluxe")
    n = fe.n_free
    Minv = np.column_stack([pc.apply(e) for e in np.eye(n)])
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    ev = np.linalg.eigvals(Minv @ K.toarray())
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev).max()
    assert ev.real.min() >= 1.0 - 1e-9


def test_deluxe_solve_matches_direct_on_the_ventricle():
    prob = lv_problem(nt=3, ntheta=12, nu=6, n_parts=6, pressure=2.0e3, gamma=1.5e4)
    fe = FEProblem(prob)
    d = 1e-4 * np.random.default_rng(3).standard_normal(fe.n_free)
    K, (Ke, Kf) = fe.tangent(d, 1.0)
    r = np.random.default_rng(4).standard_normal(fe.n_free)
    x_ref = spla.spsolve(K.tocsc(), r)
    pc = BDDC(fe, Ke, Kf, "VEF", scaling="deluxe")
    x, its, _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-12)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_deluxe_with_multilevel_coarse_solve():
    prob = slab_problem(8, 8, 4, parts=(4, 4, 2), jitter=0.15, pressure=1e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 1e-3)
    part2, n2 = box_groups((4, 4, 2), (2, 2, 1))
    r = np.random.default_rng(5).standard_normal(fe.n_free)
    x_ref = spla.spsolve(K.tocsc(), r)
    pc = BDDC(fe, Ke, Kf, "VE", level2=dict(part=part2, n_parts=n2, primal="VEF"), scaling="deluxe")
    x, its, _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-12)
    assert np.linalg.norm(x - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
