"""GPU path versus the oracle for the time-dependent terms (Section 2):
inertia with the consistent mass over dt^2 and the generalized Robin
condition of Eq. (bc epi), through fem_set_time_state and the Robin faces of
the problem description.  Bars as for the quasi-static path: 1e-12 for the
residual, tangent and SpMV, 1e-9 for the FP64 BDDC apply, 1e-10 for the
displacements of a short FP64 time-stepping solve."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC
from workloads import slab_problem, lv_problem

torch = pytest.importorskip("torch")
import paper_2208_06191_gb300 as pkg  # noqa: E402

pytestmark = pytest.mark.gpu

ROBIN = [dict(k_perp=2.0e5, k_par=2.0e4, c_perp=1.0e4, c_par=2.0e3),
         dict(k_perp=5.0e4, k_par=1.0e4, c_perp=2.0e3, c_par=5.0e2)]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.build()
    pkg.load_library()


def _dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def _slab(order):
    nx, ny, nz = 4, 3, 2
    prob = slab_problem(nx, ny, nz, order=order, parts=(2, 1, 2), jitter=0.15, pressure=2.0e3,
                        gamma=3.0e4)
    top = [[(nz - 1) * nx * ny + j * nx + i, 5, 0] for j in range(ny) for i in range(nx)]
    side = [[k * nx * ny + j * nx, 0, 1] for k in range(nz) for j in range(ny)]
    prob["robin_faces"] = np.array(top + side, dtype=np.int32)
    prob["robin"] = ROBIN
    prob["rho"] = 1.0e3
    return prob


def _lv(order):
    prob = lv_problem(nt=3, ntheta=12, nu=6, order=order, n_parts=4, pressure=2.0e3, gamma=1.5e4)
    X, E = prob["coords"], prob["elems"][:, :4]
    on_epi = np.abs((X[:, 0] ** 2 + X[:, 1] ** 2) / 0.035 ** 2 + X[:, 2] ** 2 / 0.080 ** 2 - 1) < 1e-9
    faces = [[e, f, 0] for e in range(E.shape[0]) for f in range(4)
             if all(on_epi[E[e, q]] for q in range(4) if q != f)]
    assert faces
    prob["robin_faces"] = np.array(faces, dtype=np.int32)
    prob["robin"] = ROBIN
    prob["rho"] = 1.0e3
    return prob


def _states(fe, amp, seed):
    rng = np.random.default_rng(seed)
    X = fe.coords[fe.free_nodes]
    base = amp * np.sin(7.0 * X / max(np.ptp(X), 1e-9) + 0.3)
    return [(base * s + 0.02 * amp * rng.standard_normal(X.shape)).reshape(-1) for s in (1.0, 0.8, 0.5)]


def _gpu_tangent(P):
    vals, rp, ci = P.tangent_to_host()
    n = P.n_free
    return sp.bsr_matrix((vals, ci, rp), shape=(n, n)).tocsr()


CASES = [("Q1", lambda: _slab(1), 0.02), ("Q2", lambda: _slab(2), 0.02),
         ("P1", lambda: _lv(1), 1.5e-3), ("P2", lambda: _lv(2), 1.5e-3)]


@pytest.mark.parametrize("name,make,amp", CASES)
def test_time_terms_residual_tangent_spmv_parity(name, make, amp):
    prob = make()
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    d, dp, dpp = _states(fe, amp, seed=len(name))
    assert fe.min_jacobian(d) > 0.5
    dt = 1e-3
    fe.set_time_state(dt, dp, dpp)
    dpg, dppg = _dev(dp), _dev(dpp)
    P.set_time_state(dt, dpg, dppg)
    lam = 0.6
    r = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(_dev(d), lam, r)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    K_ref, _ = fe.tangent(d, lam)
    assert abs(_gpu_tangent(P) - K_ref).max() <= 1e-12 * abs(K_ref).max()
    x = np.random.default_rng(1).standard_normal(fe.n_free)
    y = torch.empty_like(r)
    P.spmv(_dev(x), y)
    assert np.abs(_host(y) - K_ref @ x).max() <= 1e-12 * np.abs(K_ref @ x).max()
    # back to quasi-static: Robin springs only, no inertia
    fe.set_time_state(None, None, None)
    P.set_time_state(0.0)
    P.residual(_dev(d), lam, r)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()


@pytest.mark.parametrize("name,make,amp", [CASES[0], CASES[2]])
def test_time_terms_bddc_apply_parity(name, make, amp):
    prob = make()
    fe = FEProblem(prob)
    d, dp, dpp = _states(fe, amp, seed=5)
    dt = 1e-3
    fe.set_time_state(dt, dp, dpp)
    K, (Ke, Kf) = fe.tangent(d, 0.5)
    primal = "VE" if name == "Q1" else "VEF"
    ref = OracleBDDC(fe, Ke, Kf, primal)
    P = pkg.Problem(prob)
    dpg, dppg = _dev(dp), _dev(dpp)
    P.set_time_state(dt, dpg, dppg)
    P.assemble_tangent(_dev(d), 0.5)
    pc = pkg.BDDC(P, precision=pkg.FP64, primal=primal).setup()
    rhs = np.random.default_rng(6).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(rhs), z)
    z_ref = ref.apply(rhs)
    assert np.linalg.norm(_host(z) - z_ref) <= 1e-9 * np.linalg.norm(z_ref)
    assert np.abs(_host(z) - z_ref).max() <= 2 * 1e-9 * np.abs(z_ref).max()


def test_time_stepping_solve_matches_oracle():
    # three backward-Euler steps with the pressure and activation ramped in
    # time; each step is a Newton solve (GPU: BDDC-GMRES, FP64; oracle:
    # sparse LU) from the previous displacement
    prob = _slab(1)
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    opts = pkg.SolveOptions(precision=pkg.FP64, primal="VE", gmres_rtol=1e-12)
    dt, n = 1e-3, fe.n_free
    hist = [np.zeros(n), np.zeros(n)]
    hist_g = [torch.zeros(n, dtype=torch.float64, device="cuda") for _ in range(2)]
    for step in range(1, 4):
        lam = 0.3 * step
        fe.set_time_state(dt, hist[-1], hist[-2])
        d = hist[-1].copy()
        r0 = np.linalg.norm(fe.residual(d, lam))
        for _ in range(20):
            r = fe.residual(d, lam)
            if np.linalg.norm(r) <= 1e-12 * r0:
                break
            K, _ = fe.tangent(d, lam)
            d = d + spla.spsolve(K.tocsc(), -r)
        P.set_time_state(dt, hist_g[-1], hist_g[-2])
        dg = hist_g[-1].clone()
        rg = torch.empty_like(dg)
        for _ in range(20):
            P.residual(dg, lam, rg)
            if float(torch.linalg.vector_norm(rg)) <= 1e-12 * r0:
                break
            rec, _ = P.newton_step(dg, lam, opts)
            assert rec["status"] == 0
        assert np.linalg.norm(_host(dg) - d) <= 1e-10 * np.linalg.norm(d)
        hist.append(d)
        hist_g.append(dg)
    P.set_time_state(0.0)
