"""GPU path versus the oracle on the tetrahedral ventricle meshes (P1, P2),
through the C ABI.  Tolerances as for the hexahedral slabs: 1e-12 for the
residual, tangent and SpMV; 1e-9 (FP64) and 1e-3 (FP32 operators) for the
BDDC apply; 1e-10 for FP64 Newton displacements."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC
from oracle.newton import newton_solve, direct_solver
from workloads import lv_problem

torch = pytest.importorskip("torch")
import paper_2208_06191_gb300 as pkg  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.build()
    pkg.load_library()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def lv_displacement(fe, amp=1.5e-3, noise=2e-5, seed=0):
    """A smooth field of about 2% strain plus small seeded noise."""
    X = fe.coords[fe.free_nodes]
    u = amp * np.sin(40.0 * X + np.array([0.3, 1.1, 2.0]))
    u += noise * np.random.default_rng(seed).standard_normal(u.shape)
    return u.reshape(-1)


SMALL = dict(nt=3, ntheta=12, nu=6, n_parts=6, pressure=2.0e3, gamma=3.0e4)


def _gpu_tangent(P):
    vals, rp, ci = P.tangent_to_host()
    n = P.n_free
    return sp.bsr_matrix((vals, ci, rp), shape=(n, n)).tocsr()


@pytest.mark.parametrize("order", [1, 2])
def test_tet_residual_tangent_spmv_parity(order):
    prob = lv_problem(order=order, **SMALL)
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    assert P.n_free == fe.n_free
    d = lv_displacement(fe, seed=order)
    assert fe.min_jacobian(d) > 0.5
    lam = 0.9
    r = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(_dev(d), lam, r)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    K_ref, _ = fe.tangent(d, lam)
    assert abs(_gpu_tangent(P) - K_ref).max() <= 1e-12 * abs(K_ref).max()
    x = np.random.default_rng(4).standard_normal(fe.n_free)
    y = torch.empty_like(r)
    P.spmv(_dev(x), y)
    assert np.abs(_host(y) - K_ref @ x).max() <= 1e-12 * np.abs(K_ref @ x).max()


def _tet_pair(order, primal, precision, **kw):
    args = dict(SMALL)
    args.update(kw)
    prob = lv_problem(order=order, **args)
    fe = FEProblem(prob)
    d = lv_displacement(fe, seed=7)
    K, (Ke, Kf) = fe.tangent(d, 0.8)
    ref = OracleBDDC(fe, Ke, Kf, primal)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), 0.8)
    pc = pkg.BDDC(P, precision=precision, primal=primal).setup()
    return fe, K, ref, P, pc


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("primal", ["V", "VEF", "VEFR"])
@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_tet_bddc_apply_parity(order, primal, precision, tol):
    fe, K, ref, P, pc = _tet_pair(order, primal, precision)
    info = P.info
    assert pc.info()["n_primal"] == ref.n_pi
    assert info["n_vertices"] == len(ref.cl.vertices)
    assert info["n_edges"] == len(ref.cl.edges) and info["n_faces"] == len(ref.cl.faces)
    r = np.random.default_rng(9).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(r), z)
    z_ref = ref.apply(r)
    assert np.linalg.norm(_host(z) - z_ref) <= tol * np.linalg.norm(z_ref)
    assert np.abs(_host(z) - z_ref).max() <= 2 * tol * np.abs(z_ref).max()


def test_tet_multilevel_apply_parity():
    prob = lv_problem(order=1, nt=3, ntheta=16, nu=8, n_parts=16, n_parts2=4,
                      pressure=2.0e3, gamma=3.0e4)
    fe = FEProblem(prob)
    d = lv_displacement(fe, seed=8)
    K, (Ke, Kf) = fe.tangent(d, 0.8)
    ref = OracleBDDC(fe, Ke, Kf, "VEF", level2=dict(part=prob["part2"], n_parts=4, primal="VEF"))
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), 0.8)
    pc = pkg.BDDC(P, precision=pkg.FP64, primal="VEF", levels=3, part2=prob["part2"],
                  n_parts2=4, primal2="VEF").setup()
    assert pc.info()["n_primal2"] == ref.coarse.n_pi > 0
    r = np.random.default_rng(10).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(r), z)
    z_ref = ref.apply(r)
    assert np.linalg.norm(_host(z) - z_ref) <= 1e-9 * np.linalg.norm(z_ref)
    assert np.abs(_host(z) - z_ref).max() <= 2 * 1e-9 * np.abs(z_ref).max()


@pytest.mark.parametrize("order", [1, 2])
def test_tet_newton_fp64_matches_oracle(order):
    prob = lv_problem(order=order, nt=3, ntheta=10, nu=5, n_parts=4, pressure=2.0e3,
                      gamma=3.0e4, load_steps=2)
    d_ref, _ = newton_solve(prob, direct_solver, tol=1e-11)
    P = pkg.Problem(prob)
    d, rep = P.solve(pkg.SolveOptions(precision=pkg.FP64, primal="VEF", load_steps=2,
                                      newton_rtol=1e-11, gmres_rtol=1e-12))
    assert rep["status"] == 0 and rep["load_steps_done"] == 2
    assert np.linalg.norm(_host(d) - d_ref) <= 1e-10 * np.linalg.norm(d_ref)


def test_tet_newton_fp32_within_two_iterations():
    prob = lv_problem(order=1, nt=3, ntheta=16, nu=8, n_parts=8, pressure=2.0e3, gamma=3.0e4)
    P = pkg.Problem(prob)
    d64, rep64 = P.solve(pkg.SolveOptions(precision=pkg.FP64, primal="VEF"))
    d32, rep32 = P.solve(pkg.SolveOptions(precision=pkg.FP32, primal="VEF"))
    assert rep32["status"] == 0 and rep32["final_rel_residual"] <= 1e-8
    its64 = [r["gmres_its"] for r in rep64["records"]]
    its32 = [r["gmres_its"] for r in rep32["records"]]
    assert len(its32) == len(its64)
    assert all(b <= a + 2 for a, b in zip(its64, its32))
