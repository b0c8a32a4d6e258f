"""Pins of the oracle's BDDC (Section 3.2) and GMRES against what the theory
fixes: exactness of the block factorisation when the coarse space spans the
interface, one subdomain, symmetry and the lower spectral bound 1 of the
preconditioned operator in the symmetric case, the poly-logarithmic growth
in H/h, the ordering of primal spaces (Section 6.2) and agreement of the
BDDC-GMRES Newton solve with the direct one."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC, Classification
from oracle.krylov import gmres
from oracle.newton import newton_solve, direct_solver, make_bddc_solver
from workloads import slab_problem


def _setup(prob, d_scale=0.0, lam=1.0, seed=0):
    fe = FEProblem(prob)
    d = d_scale * np.random.default_rng(seed).standard_normal(fe.n_free)
    K, (Ke, Kf) = fe.tangent(d, lam)
    return fe, K, Ke, Kf


def test_classification_structured_boxes():
    # 2x2x2 boxes of an 8^3 cube clamped at z=0: one 8-fold cross point,
    # one on the top face and four on the lateral faces are vertices; the
    # remaining multiply-shared lines are edges, the rest faces.
    prob = slab_problem(8, 8, 8, parts=(2, 2, 2))
    fe = FEProblem(prob)
    cl = Classification(fe, prob["elem_part"], prob["n_parts"])
    X = fe.coords[cl.vertices]
    got = sorted(map(tuple, np.round(X * 8).astype(int)))
    want = sorted([(4, 4, 4), (4, 4, 8), (0, 4, 4), (8, 4, 4), (4, 0, 4), (4, 8, 4)])
    assert got == want
    # edges: four half-lines from the centre (x, y directions) and two
    # vertical segments below and above the centre
    assert len(cl.edges) == 6
    assert len(cl.faces) == 12


def test_single_subdomain_is_exact():
    prob = slab_problem(3, 3, 3, parts=(1, 1, 1), pressure=2e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 0.01)
    pc = BDDC(fe, Ke, Kf, "V")
    r = np.random.default_rng(1).standard_normal(fe.n_free)
    z = pc.apply(r)
    assert np.allclose(K @ z, r, rtol=0, atol=1e-10 * np.abs(r).max())
    x, its, _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-10)
    assert its == 1


def test_all_interface_primal_is_exact():
    # With every interface node primal, the local problems are Dirichlet
    # problems and Phi S_PiPi^-1 Phi^T is the whole Schur complement inverse.
    prob = slab_problem(4, 4, 4, parts=(2, 2, 2), pressure=2e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 0.01)
    cl = Classification(fe, prob["elem_part"], prob["n_parts"])
    cl.vertices = sorted(int(a) for a in np.nonzero(cl.interface)[0])
    cl.edges, cl.faces = [], []
    pc = BDDC(fe, Ke, Kf, "V", cl)
    r = np.random.default_rng(2).standard_normal(fe.n_free)
    z = pc.apply(r)
    assert np.linalg.norm(K @ z - r) <= 1e-10 * np.linalg.norm(r)


@pytest.mark.parametrize("primal", ["V", "VE", "VEF"])
def test_symmetric_case_spectrum(primal):
    # p = 0, gamma = 0, d = 0: the tangent is SPD, M^-1 is symmetric and the
    # eigenvalues of M^-1 A are real and >= 1 (BDDC theory).
    prob = slab_problem(4, 4, 4, parts=(2, 2, 2), pressure=0.0, gamma=0.0)
    fe, K, Ke, Kf = _setup(prob)
    pc = BDDC(fe, Ke, Kf, primal)
    n = fe.n_free
    Minv = np.column_stack([pc.apply(e) for e in np.eye(n)])
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    ev = np.linalg.eigvals(Minv @ K.toarray())
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev).max()
    assert ev.real.min() >= 1.0 - 1e-9


def _cond_estimate(prob, primal):
    fe, K, Ke, Kf = _setup(prob)
    pc = BDDC(fe, Ke, Kf, primal)
    op = spla.LinearOperator((fe.n_free,) * 2, matvec=lambda v: pc.apply(K @ v))
    lmax = spla.eigs(op, k=1, which="LM", tol=1e-6, return_eigenvectors=False)
    return abs(lmax[0])  # lambda_min >= 1, so this bounds the condition number


def test_condition_grows_polylogarithmically():
    # kappa <= c (1 + log(H/h))^2: with 2x2x2 subdomains and H/h = 2, 4, 6
    # the ratio kappa / (1 + log(H/h))^2 stays bounded while kappa grows.
    ks, ratios = [], []
    for hh in (2, 4, 6):
        prob = slab_problem(2 * hh, 2 * hh, 2 * hh, parts=(2, 2, 2),
                            pressure=0.0, gamma=0.0)
        kappa = _cond_estimate(prob, "VE")
        ks.append(kappa)
        ratios.append(kappa / (1 + np.log(hh)) ** 2)
    assert ks[0] < ks[1] < ks[2]
    assert max(ratios) / min(ratios) < 2.0


def test_primal_space_ordering():
    # Richer primal spaces need fewer iterations: V >= VE >= VEF (Section 6.2).
    prob = slab_problem(9, 9, 6, parts=(3, 3, 2), pressure=1e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 0.005)
    r = np.random.default_rng(4).standard_normal(fe.n_free)
    its = {}
    for primal in ("V", "VE", "VEF"):
        pc = BDDC(fe, Ke, Kf, primal)
        _, its[primal], _ = gmres(lambda v: K @ v, r, pc.apply, tol=1e-8)
    assert its["V"] >= its["VE"] >= its["VEF"]
    assert its["V"] > its["VEF"]


def test_flexible_matches_right_preconditioned():
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), pressure=1e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 0.005)
    pc = BDDC(fe, Ke, Kf, "VE")
    b = np.random.default_rng(6).standard_normal(fe.n_free)
    x1, i1, _ = gmres(lambda v: K @ v, b, pc.apply, tol=1e-10)
    x2, i2, _ = gmres(lambda v: K @ v, b, pc.apply, tol=1e-10, flexible=True)
    assert abs(i1 - i2) <= 1
    assert np.linalg.norm(K @ x1 - b) <= 1e-9 * np.linalg.norm(b)
    assert np.linalg.norm(x1 - x2) <= 1e-8 * np.linalg.norm(x1)


def test_gmres_restart_reaches_tolerance():
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), pressure=1e3, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 0.005)
    pc = BDDC(fe, Ke, Kf, "V")
    b = np.random.default_rng(7).standard_normal(fe.n_free)
    x, its, _ = gmres(lambda v: K @ v, b, pc.apply, tol=1e-9, restart=5)
    assert its > 5
    assert np.linalg.norm(K @ x - b) <= 2e-9 * np.linalg.norm(b)


def test_bddc_newton_matches_direct_newton():
    prob = slab_problem(6, 6, 6, parts=(2, 2, 2), primal="VE", load_steps=2)
    d1, log1 = newton_solve(prob, direct_solver, tol=1e-11)
    d2, log2 = newton_solve(prob, make_bddc_solver("VE", tol=1e-12), tol=1e-11)
    assert np.linalg.norm(d2 - d1) <= 1e-10 * np.linalg.norm(d1)
    assert all(l["gmres_its"] > 1 for l in log2)


def _ml_setup(nx=8, ny=8, nz=4, parts=(4, 4, 2), groups=(2, 2, 1), p=1e3, g=3e4):
    from workloads import box_groups
    prob = slab_problem(nx, ny, nz, parts=parts, pressure=p, gamma=g)
    fe, K, Ke, Kf = _setup(prob, 0.0 if p == 0 else 0.005)
    part2, n2 = box_groups(parts, groups)
    return prob, fe, K, Ke, Kf, part2, n2


def test_multilevel_with_one_level2_subdomain_equals_two_level():
    # One level-2 subdomain: the level-2 BDDC solves the coarse problem
    # exactly, so the multilevel apply must equal the two-level one.
    prob, fe, K, Ke, Kf, part2, n2 = _ml_setup(groups=(1, 1, 1))
    two = BDDC(fe, Ke, Kf, "VE")
    ml = BDDC(fe, Ke, Kf, "VE", level2=dict(part=part2, n_parts=n2, primal="VEF"))
    assert ml.coarse is not None and ml.coarse.n_pi == 0
    r = np.random.default_rng(11).standard_normal(fe.n_free)
    z2, zm = two.apply(r), ml.apply(r)
    assert np.linalg.norm(zm - z2) <= 1e-10 * np.linalg.norm(z2)


def test_multilevel_takes_at_least_the_two_level_iterations():
    # Section 7: approximating the coarse problem by BDDC raises the
    # iteration count relative to the exact coarse solve.
    prob, fe, K, Ke, Kf, part2, n2 = _ml_setup()
    b = np.random.default_rng(12).standard_normal(fe.n_free)
    two = BDDC(fe, Ke, Kf, "VE")
    ml = BDDC(fe, Ke, Kf, "VE", level2=dict(part=part2, n_parts=n2, primal="VEF"))
    assert ml.coarse.n_pi > 0
    _, i2, _ = gmres(lambda v: K @ v, b, two.apply, tol=1e-8)
    x, im, _ = gmres(lambda v: K @ v, b, ml.apply, tol=1e-8)
    assert im >= i2
    assert np.linalg.norm(K @ x - b) <= 2e-8 * np.linalg.norm(b)


def test_multilevel_symmetric_case():
    # Symmetric tangent: the multilevel preconditioner stays symmetric and
    # M^-1 A keeps a real spectrum bounded below by 1.
    prob, fe, K, Ke, Kf, part2, n2 = _ml_setup(6, 6, 4, parts=(3, 3, 2), groups=(2, 2, 1), p=0.0, g=0.0)
    ml = BDDC(fe, Ke, Kf, "VE", level2=dict(part=part2, n_parts=n2, primal="VEF"))
    n = fe.n_free
    Minv = np.column_stack([ml.apply(e) for e in np.eye(n)])
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    ev = np.linalg.eigvals(Minv @ K.toarray())
    assert np.abs(ev.imag).max() <= 1e-8 * np.abs(ev).max()
    assert ev.real.min() >= 1.0 - 1e-9


def _pcg(matvec, b, precond, tol, maxiter=500):
    """Textbook preconditioned conjugate gradients; returns the true relative
    residual after every iteration."""
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    p = z.copy()
    rz = r @ z
    hist = []
    for _ in range(maxiter):
        Ap = matvec(p)
        alpha = rz / (p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        hist.append(np.linalg.norm(b - matvec(x)) / np.linalg.norm(b))
        if hist[-1] <= tol:
            break
        z = precond(r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, hist


@pytest.mark.parametrize("primal", ["V", "VE"])
def test_symmetric_case_pcg_and_gmres_agree(primal):
    # SPD tangent (no follower pressure) and symmetric BDDC: right-
    # preconditioned GMRES minimises ||b - A x_k|| over the same affine
    # Krylov space PCG's x_k lies in, so GMRES never needs more iterations
    # than PCG for the same residual tolerance; PCG needs only a few more.
    prob = slab_problem(6, 6, 4, parts=(2, 2, 2), jitter=0.1, pressure=0.0, gamma=3e4)
    fe, K, Ke, Kf = _setup(prob, 1e-3)
    pc = BDDC(fe, Ke, Kf, primal)
    b = np.random.default_rng(9).standard_normal(fe.n_free)
    x_g, its_g, hist_g = gmres(lambda v: K @ v, b, pc.apply, tol=1e-9)
    x_c, hist_c = _pcg(lambda v: K @ v, b, pc.apply, tol=1e-9)
    its_c = len(hist_c)
    assert its_g <= its_c <= its_g + 3
    # after every step k, GMRES's residual (hist_g[k]; hist_g[0] = 1) is no
    # larger than PCG's (hist_c[k - 1])
    k = min(its_g, its_c)
    assert np.all(np.array(hist_g[1:k + 1]) <= np.array(hist_c[:k]) * (1 + 1e-6) + 1e-14)
    assert np.linalg.norm(x_g - x_c) <= 1e-7 * np.linalg.norm(x_c)
