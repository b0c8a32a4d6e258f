"""Deluxe scaling on the GPU path versus the oracle, through the C ABI.

Tolerances as for the counting-scaled apply: FP64 operators relative 1e-9
(dense Gauss-Jordan inverses vs sparse LU and dense solves, rounding
amplified by the local condition numbers), FP32 operators relative 1e-3;
GMRES iterations of the FP64 path within one of the oracle's.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC
from oracle.krylov import gmres as oracle_gmres
from workloads import box_groups, lv_problem, slab_problem

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


def _smooth(fe, amp=0.03, seed=0):
    X = fe.coords[fe.free_nodes]
    u = np.stack([np.sin(2 * X[:, 1] + X[:, 2]), np.cos(3 * X[:, 0]) * X[:, 2],
                  np.sin(X[:, 0] + 2 * X[:, 2])], axis=1) * (amp * X[:, 2:3])
    u += 0.002 * np.random.default_rng(seed).standard_normal(u.shape)
    return u.reshape(-1)


RAGGED = dict(nx=5, ny=4, nz=3, parts=(2, 2, 2), jitter=0.2, pressure=2.0e3, gamma=3.0e4)


def _pair(prob, primal, precision, lam=0.8, disp=None, **kw):
    fe = FEProblem(prob)
    d = _smooth(fe) if disp is None else disp(fe)
    K, (Ke, Kf) = fe.tangent(d, lam)
    ref_kw = {k: v for k, v in kw.items() if k == "level2"}
    ref = OracleBDDC(fe, Ke, Kf, primal, scaling="deluxe", **ref_kw)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), lam)
    gpu_kw = {k: v for k, v in kw.items() if k != "level2"}
    pc = pkg.BDDC(P, precision=precision, primal=primal, scaling="deluxe", **gpu_kw).setup()
    return fe, K, ref, P, pc


def _apply_err(fe, ref, pc, seed):
    r = np.random.default_rng(seed).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(r), z)
    z_ref = ref.apply(r)
    zh = _host(z)
    # the larger of the norm-relative and half the largest-entry-relative
    # difference, so that one bound checks both
    return max(np.linalg.norm(zh - z_ref) / np.linalg.norm(z_ref),
               0.5 * np.abs(zh - z_ref).max() / np.abs(z_ref).max())


@pytest.mark.parametrize("primal", ["V", "VE", "VEF", "EF"])
@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_deluxe_apply_parity(primal, precision, tol):
    fe, K, ref, P, pc = _pair(slab_problem(order=1, **RAGGED), primal, precision)
    assert pc.info()["n_primal"] == ref.n_pi
    for seed in (11, 12):
        assert _apply_err(fe, ref, pc, seed) <= tol


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_deluxe_apply_parity_tets(order, precision, tol):
    prob = lv_problem(order=order, nt=3, ntheta=12, nu=6, n_parts=6, pressure=2.0e3, gamma=3.0e4)

    def disp(fe):
        X = fe.coords[fe.free_nodes]
        u = 1.5e-3 * np.sin(40.0 * X) * (X[:, 2:3] + 0.08)
        return u.reshape(-1)

    fe, K, ref, P, pc = _pair(prob, "VEF", precision, disp=disp)
    assert _apply_err(fe, ref, pc, 13) <= tol


def test_deluxe_q2_apply_parity():
    prob = slab_problem(4, 3, 2, order=2, parts=(2, 2, 1), jitter=0.1, pressure=1e3, gamma=2e4)
    fe, K, ref, P, pc = _pair(prob, "VEF", pkg.FP64)
    assert _apply_err(fe, ref, pc, 14) <= 1e-9


def test_two_subdomains_deluxe_is_exact_on_gpu():
    prob = slab_problem(4, 3, 3, order=1, parts=(2, 1, 1), jitter=0.1, pressure=2e3, gamma=3e4)
    fe, K, ref, P, pc = _pair(prob, "V", pkg.FP64)
    assert pc.info()["n_primal"] == 0
    b = np.random.default_rng(15).standard_normal(fe.n_free)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, rtol=1e-10)
    assert rep["converged"] and rep["iterations"] == 1
    assert np.linalg.norm(K @ _host(x) - b) <= 1e-9 * np.linalg.norm(b)


def test_deluxe_gmres_parity():
    fe, K, ref, P, pc = _pair(slab_problem(order=1, **RAGGED), "VE", pkg.FP64)
    b = np.random.default_rng(16).standard_normal(fe.n_free)
    x_ref, its_ref, _ = oracle_gmres(lambda v: K @ v, b, ref.apply, tol=1e-10)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, rtol=1e-10)
    assert rep["converged"]
    assert abs(rep["iterations"] - its_ref) <= 1
    assert np.linalg.norm(_host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_deluxe_multilevel_apply_parity():
    prob = slab_problem(8, 8, 4, order=1, parts=(4, 4, 2), jitter=0.15, pressure=1e3, gamma=3e4)
    part2, n2 = box_groups((4, 4, 2), (2, 2, 1))
    fe, K, ref, P, pc = _pair(prob, "VE", pkg.FP64, level2=dict(part=part2, n_parts=n2, primal="VEF"),
                              levels=3, part2=part2, n_parts2=n2, primal2="VEF")
    assert _apply_err(fe, ref, pc, 17) <= 1e-9


def test_deluxe_noalloc_matches_apply():
    fe, K, ref, P, pc = _pair(slab_problem(order=1, **RAGGED), "VEF", pkg.FP32)
    r = _dev(np.random.default_rng(18).standard_normal(fe.n_free))
    z1 = torch.empty_like(r)
    z2 = torch.empty_like(r)
    pc.apply(r, z1)
    pc.apply_noalloc(r, z2)
    assert torch.equal(z1, z2)


def test_deluxe_newton_solve_fp32():
    prob = slab_problem(6, 6, 3, order=1, parts=(2, 2, 1), pressure=1e3, gamma=3e4, load_steps=2)
    P = pkg.Problem(prob)
    opts = pkg.SolveOptions(precision=pkg.FP32, primal="VE", load_steps=2, scaling="deluxe")
    d, rep = P.solve(opts)
    assert rep["status"] == 0 and rep["final_rel_residual"] <= 1e-8
    fe = FEProblem(prob)
    r = fe.residual(_host(d), 1.0)
    f0 = fe.residual(np.zeros(fe.n_free), 1.0)
    assert np.linalg.norm(r) <= 1e-7 * np.linalg.norm(f0)
