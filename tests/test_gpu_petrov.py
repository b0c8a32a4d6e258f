"""Nonsymmetric BDDC with a left coarse basis (Petrov coarse space) on the
GPU path versus the oracle's, through the C ABI, on tangents made
nonsymmetric by the follower pressure on a face whose edges are free.

Tolerances as for the Galerkin apply: FP64 operators relative 1e-9, FP32
operators relative 1e-3; GMRES iterations of the FP64 path within one of
the oracle's.
"""
import numpy as np
import pytest

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC
from oracle.krylov import gmres as oracle_gmres
from workloads import box_groups, slab_problem

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


RAGGED = dict(nx=5, ny=4, nz=3, parts=(2, 2, 2), jitter=0.2, pressure=5.0e3, gamma=3.0e4)


def _pair(prob, primal, precision, scaling="counting", **kw):
    fe = FEProblem(prob)
    d = _smooth(fe)
    K, (Ke, Kf) = fe.tangent(d, 0.8)
    ref_kw = {k: v for k, v in kw.items() if k == "level2"}
    ref = OracleBDDC(fe, Ke, Kf, primal, scaling=scaling, coarse="petrov", **ref_kw)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), 0.8)
    gpu_kw = {k: v for k, v in kw.items() if k != "level2"}
    pc = pkg.BDDC(P, precision=precision, primal=primal, scaling=scaling, coarse="petrov",
                  **gpu_kw).setup()
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


@pytest.mark.parametrize("primal,scaling", [("VE", "counting"), ("VEF", "counting"),
                                            ("EF", "counting"), ("VE", "deluxe"), ("EFR", "counting")])
@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_petrov_apply_parity(primal, scaling, precision, tol):
    fe, K, ref, P, pc = _pair(slab_problem(order=1, **RAGGED), primal, precision, scaling)
    Kd = K.toarray()
    assert np.abs(Kd - Kd.T).max() > 1e-6 * np.abs(Kd).max()
    assert pc.info()["n_primal"] == ref.n_pi
    assert _apply_err(fe, ref, pc, 21) <= tol


def test_petrov_gmres_parity():
    fe, K, ref, P, pc = _pair(slab_problem(order=1, **RAGGED), "VE", pkg.FP64)
    b = np.random.default_rng(22).standard_normal(fe.n_free)
    x_ref, its_ref, _ = oracle_gmres(lambda v: K @ v, b, ref.apply, tol=1e-10)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, rtol=1e-10)
    assert rep["converged"]
    assert abs(rep["iterations"] - its_ref) <= 1
    assert np.linalg.norm(_host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_petrov_multilevel_apply_parity():
    prob = slab_problem(8, 8, 4, order=1, parts=(4, 4, 2), jitter=0.15, pressure=5e3, gamma=3e4)
    part2, n2 = box_groups((4, 4, 2), (2, 2, 1))
    fe, K, ref, P, pc = _pair(prob, "VE", pkg.FP64, level2=dict(part=part2, n_parts=n2, primal="VEF"),
                              levels=3, part2=part2, n_parts2=n2, primal2="VEF")
    assert _apply_err(fe, ref, pc, 23) <= 1e-9


def test_petrov_newton_solve_fp32():
    prob = slab_problem(6, 6, 3, order=1, parts=(2, 2, 1), pressure=1e3, gamma=3e4, load_steps=2)
    P = pkg.Problem(prob)
    opts = pkg.SolveOptions(precision=pkg.FP32, primal="VE", load_steps=2, coarse="petrov")
    d, rep = P.solve(opts)
    assert rep["status"] == 0 and rep["final_rel_residual"] <= 1e-8
