"""GPU path versus the oracle, element by element, through the C ABI.

Tolerances:
* residual, tangent, SpMV: FP64 throughout, relative 1e-12 of the largest
  entry (rounding order differs, nothing else);
* BDDC apply, FP64 operators: relative 1e-9 (dense Gauss-Jordan inverses vs
  sparse LU; both exact up to rounding amplified by the local condition
  numbers, about 1e4 here);
* BDDC apply, FP32 operators: relative 1e-3 (FP32 unit roundoff 6e-8 times
  the local condition numbers);
* Newton solve, FP64: displacement within 1e-10 relative of the oracle's
  direct-solver Newton solution (tolerances tightened to 1e-11 / 1e-12);
* Newton solve, FP32 operators: final relative residual <= 1e-8 and GMRES
  iterations within +2 of the FP64 path at every Newton step.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC, Classification
from oracle.krylov import gmres as oracle_gmres
from oracle.newton import newton_solve, direct_solver
from workloads import slab_problem, slab_config

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


def smooth_displacement(fe, amp=0.03, noise=0.002, seed=0):
    """A smooth field vanishing at z = 0 plus small seeded noise (keeps every
    element far from inversion on all test meshes)."""
    X = fe.coords[fe.free_nodes]
    u = np.stack([np.sin(2 * X[:, 1] + X[:, 2]), np.cos(3 * X[:, 0]) * X[:, 2],
                  np.sin(X[:, 0] + 2 * X[:, 2])], axis=1) * (amp * X[:, 2:3])
    u += noise * np.random.default_rng(seed).standard_normal(u.shape)
    return u.reshape(-1)


def _gpu_tangent(P):
    vals, rp, ci = P.tangent_to_host()
    n = P.n_free
    return sp.bsr_matrix((vals, ci, rp), shape=(n, n)).tocsr()


RAGGED = dict(nx=5, ny=4, nz=3, parts=(2, 2, 2), jitter=0.2, pressure=2.0e3, gamma=3.0e4)


@pytest.mark.parametrize("order", [1, 2])
def test_residual_and_tangent_parity(order):
    prob = slab_problem(order=order, **RAGGED)
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    assert P.n_free == fe.n_free
    rng = np.random.default_rng(10 + order)
    d = smooth_displacement(fe, seed=10 + order)
    assert fe.min_jacobian(d) > 0.5
    lam = 0.7
    r_gpu = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(_dev(d), lam, r_gpu)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r_gpu) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    K_ref, _ = fe.tangent(d, lam)
    K_gpu = _gpu_tangent(P)
    diff = abs(K_gpu - K_ref).max()
    assert diff <= 1e-12 * abs(K_ref).max()
    # SpMV with the assembled tangent
    x = rng.standard_normal(fe.n_free)
    y = torch.empty_like(r_gpu)
    P.spmv(_dev(x), y)
    assert np.abs(_host(y) - K_ref @ x).max() <= 1e-12 * np.abs(K_ref @ x).max()


def test_residual_only_matches_tangent_call():
    prob = slab_problem(order=1, **RAGGED)
    P = pkg.Problem(prob)
    d = _dev(smooth_displacement(FEProblem(prob), seed=3))
    r1 = torch.empty(P.n_free, dtype=torch.float64, device="cuda")
    r2 = torch.empty_like(r1)
    P.residual(d, 0.5, r1)
    P.assemble_tangent(d, 0.5, r2)
    assert torch.equal(r1, r2)


def _bddc_pair(prob, primal, precision, lam=0.8, seed=0):
    fe = FEProblem(prob)
    d = smooth_displacement(fe, seed=seed)
    K, (Ke, Kf) = fe.tangent(d, lam)
    ref = OracleBDDC(fe, Ke, Kf, primal)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), lam)
    pc = pkg.BDDC(P, precision=precision, primal=primal).setup()
    return fe, K, ref, P, pc


@pytest.mark.parametrize("primal", ["V", "VE", "VEF", "EF", "VER", "EFR"])
@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_bddc_apply_parity(primal, precision, tol):
    prob = slab_problem(order=1, **RAGGED)
    fe, K, ref, P, pc = _bddc_pair(prob, primal, precision)
    assert pc.info()["n_primal"] == ref.n_pi
    rng = np.random.default_rng(5)
    for _ in range(2):
        r = rng.standard_normal(fe.n_free)
        z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
        pc.apply(_dev(r), z)
        z_ref = ref.apply(r)
        assert np.linalg.norm(_host(z) - z_ref) <= tol * np.linalg.norm(z_ref)
        assert np.abs(_host(z) - z_ref).max() <= 2 * tol * np.abs(z_ref).max()


@pytest.mark.parametrize("order,parts", [(2, (2, 2, 1)), (1, (3, 1, 2))])
def test_bddc_apply_parity_q2_and_uneven(order, parts):
    prob = slab_problem(4, 3, 2, order=order, parts=parts, jitter=0.1, pressure=1e3, gamma=2e4)
    fe, K, ref, P, pc = _bddc_pair(prob, "VEF", pkg.FP64)
    r = np.random.default_rng(6).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(r), z)
    z_ref = ref.apply(r)
    assert np.linalg.norm(_host(z) - z_ref) <= 1e-9 * np.linalg.norm(z_ref)
    assert np.abs(_host(z) - z_ref).max() <= 2 * 1e-9 * np.abs(z_ref).max()


def test_single_subdomain_is_exact_solve():
    prob = slab_problem(3, 3, 3, order=1, parts=(1, 1, 1), pressure=1e3, gamma=2e4)
    fe, K, ref, P, pc = _bddc_pair(prob, "V", pkg.FP64)
    b = np.random.default_rng(2).standard_normal(fe.n_free)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, rtol=1e-10)
    assert rep["converged"] and rep["iterations"] == 1
    assert np.linalg.norm(K @ _host(x) - b) <= 1e-10 * np.linalg.norm(b)


@pytest.mark.parametrize("primal", ["V", "VE", "EFR"])
def test_gmres_parity(primal):
    prob = slab_problem(order=1, **RAGGED)
    fe, K, ref, P, pc = _bddc_pair(prob, primal, pkg.FP64)
    b = np.random.default_rng(7).standard_normal(fe.n_free)
    x_ref, its_ref, _ = oracle_gmres(lambda v: K @ v, b, ref.apply, tol=1e-10)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, rtol=1e-10)
    assert rep["converged"]
    assert abs(rep["iterations"] - its_ref) <= 1
    assert np.linalg.norm(K @ _host(x) - b) <= 2e-10 * np.linalg.norm(b)
    assert np.linalg.norm(_host(x) - x_ref) <= 1e-8 * np.linalg.norm(x_ref)


def test_gmres_restart_path():
    prob = slab_problem(order=1, **RAGGED)
    fe, K, ref, P, pc = _bddc_pair(prob, "V", pkg.FP64)
    b = np.random.default_rng(8).standard_normal(fe.n_free)
    x = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    rep = pc.gmres(_dev(b), x, restart=4, rtol=1e-9)
    assert rep["converged"] and rep["iterations"] > 4
    assert np.linalg.norm(K @ _host(x) - b) <= 2e-9 * np.linalg.norm(b)


def test_newton_solve_fp64_matches_oracle_cube():
    prob = slab_config("slab8_q1")
    d_ref, log = newton_solve(prob, direct_solver, tol=1e-11)
    P = pkg.Problem(prob)
    opts = pkg.SolveOptions(precision=pkg.FP64, primal="V", load_steps=4, newton_rtol=1e-11,
                            gmres_rtol=1e-12)
    d, rep = P.solve(opts)
    assert rep["status"] == 0 and rep["load_steps_done"] == 4
    assert np.linalg.norm(_host(d) - d_ref) <= 1e-10 * np.linalg.norm(d_ref)


def test_newton_solve_fp32_local_operators():
    prob = slab_config("slab8_q1")
    P = pkg.Problem(prob)
    d64, rep64 = P.solve(pkg.SolveOptions(precision=pkg.FP64, primal="V"))
    d32, rep32 = P.solve(pkg.SolveOptions(precision=pkg.FP32, primal="V"))
    assert rep32["status"] == 0 and rep32["load_steps_done"] == 4
    assert rep32["final_rel_residual"] <= 1e-8
    its64 = [r["gmres_its"] for r in rep64["records"]]
    its32 = [r["gmres_its"] for r in rep32["records"]]
    assert len(its32) == len(its64)
    assert all(b <= a + 2 for a, b in zip(its64, its32))
    # both solve the same nonlinear problem
    fe = FEProblem(prob)
    r = fe.residual(_host(d32), 1.0)
    r0 = fe.residual(np.zeros(fe.n_free), 1.0)
    assert np.linalg.norm(r) <= 1e-7 * np.linalg.norm(r0)


def test_zero_load_converges_immediately():
    prob = slab_problem(3, 3, 3, order=1, parts=(2, 1, 1), pressure=0.0, gamma=0.0)
    P = pkg.Problem(prob)
    d, rep = P.solve(pkg.SolveOptions(precision=pkg.FP64, primal="V", load_steps=2))
    assert rep["status"] == 0 and rep["newton_steps"] == 0
    assert float(torch.abs(d).max()) == 0.0


def test_inverted_element_is_reported():
    prob = slab_problem(2, 2, 2, order=1, parts=(1, 1, 1))
    P = pkg.Problem(prob)
    d = torch.zeros(P.n_free, dtype=torch.float64, device="cuda")
    d[2::3] = -5.0  # pushes every free node far below the clamped base
    r = torch.empty_like(d)
    with pytest.raises(pkg.CBDDCError) as ei:
        P.residual(d, 1.0, r)
    assert ei.value.code == pkg.EINVERTED


def test_invalid_inputs_are_rejected():
    prob = slab_problem(2, 2, 2, order=1, parts=(1, 1, 1))
    bad = dict(prob, elems=np.array(prob["elems"]) + 10_000)
    with pytest.raises(pkg.CBDDCError) as ei:
        pkg.Problem(bad)
    assert ei.value.code == pkg.EINVAL
    bad = dict(prob, elem_part=np.full(len(prob["elems"]), 3), n_parts=2)
    with pytest.raises(pkg.CBDDCError) as ei:
        pkg.Problem(bad)
    assert ei.value.code == pkg.EINVAL


def test_full_size_slab_residual_and_apply_sampled():
    # 48x48x12 Q1, 64 subdomains, VE: the launch configuration of the bench.
    prob = slab_config("slab48_q1")
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    assert P.info["n_vertices"] == 72 and P.info["n_edges"] == 108
    lam = 0.25
    d = np.zeros(fe.n_free)
    r_gpu = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(_dev(d), lam, r_gpu)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r_gpu) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    K_ref, (Ke, Kf) = fe.tangent(d, lam)
    ref = OracleBDDC(fe, Ke, Kf, "VE")
    for precision, tol in ((pkg.FP64, 1e-9), (pkg.FP32, 1e-3)):
        pc = pkg.BDDC(P, precision=precision, primal="VE").setup()
        assert pc.info()["n_primal"] == ref.n_pi == 540
        z = torch.empty_like(r_gpu)
        pc.apply(_dev(-r_ref), z)
        z_ref = ref.apply(-r_ref)
        assert np.linalg.norm(_host(z) - z_ref) <= tol * np.linalg.norm(z_ref)
        assert np.abs(_host(z) - z_ref).max() <= 2 * tol * np.abs(z_ref).max()


# ------------------------------------------------------------- multilevel

def _ml_pair(parts=(4, 4, 2), groups=(2, 2, 1), precision=None, primal="VE"):
    from workloads import box_groups
    prob = slab_problem(8, 8, 4, order=1, parts=parts, jitter=0.15, pressure=1e3, gamma=3e4)
    fe = FEProblem(prob)
    d = smooth_displacement(fe, seed=21)
    K, (Ke, Kf) = fe.tangent(d, 0.8)
    part2, n2 = box_groups(parts, groups)
    ref = OracleBDDC(fe, Ke, Kf, primal, level2=dict(part=part2, n_parts=n2, primal="VEF"))
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), 0.8)
    pc = pkg.BDDC(P, precision=precision if precision is not None else pkg.FP64, primal=primal,
                  levels=3, part2=part2, n_parts2=n2, primal2="VEF").setup()
    return fe, K, ref, P, pc


@pytest.mark.parametrize("precision,tol", [(pkg.FP64, 1e-9), (pkg.FP32, 1e-3)])
def test_multilevel_apply_parity(precision, tol):
    fe, K, ref, P, pc = _ml_pair(precision=precision)
    info = pc.info()
    assert info["n_primal"] == ref.n_pi and info["n_primal2"] == ref.coarse.n_pi > 0
    r = np.random.default_rng(31).standard_normal(fe.n_free)
    z = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    pc.apply(_dev(r), z)
    z_ref = ref.apply(r)
    assert np.linalg.norm(_host(z) - z_ref) <= tol * np.linalg.norm(z_ref)
    assert np.abs(_host(z) - z_ref).max() <= 2 * tol * np.abs(z_ref).max()


def test_rotations_refused_for_multilevel():
    from workloads import box_groups
    prob = slab_problem(4, 4, 2, order=1, parts=(2, 2, 1), pressure=1e3, gamma=3e4)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(np.zeros(P.n_free)), 0.5)
    part2, n2 = box_groups((2, 2, 1), (2, 1, 1))
    for primal, primal2 in (("VER", "VEF"), ("VE", "VEFR")):
        with pytest.raises(pkg.CBDDCError) as ei:
            pkg.BDDC(P, precision=pkg.FP64, primal=primal, levels=3, part2=part2, n_parts2=n2,
                     primal2=primal2).setup()
        assert ei.value.code == pkg.EINVAL


def test_multilevel_with_one_group_equals_two_level_on_gpu():
    from workloads import box_groups
    prob = slab_problem(8, 8, 4, order=1, parts=(4, 4, 2), pressure=1e3, gamma=3e4)
    fe = FEProblem(prob)
    d = smooth_displacement(fe, seed=22)
    P = pkg.Problem(prob)
    P.assemble_tangent(_dev(d), 0.7)
    part2, n2 = box_groups((4, 4, 2), (1, 1, 1))
    two = pkg.BDDC(P, precision=pkg.FP64, primal="VE").setup()
    ml = pkg.BDDC(P, precision=pkg.FP64, primal="VE", levels=3, part2=part2, n_parts2=n2).setup()
    r = _dev(np.random.default_rng(32).standard_normal(fe.n_free))
    z2 = torch.empty_like(r)
    zm = torch.empty_like(r)
    two.apply(r, z2)
    ml.apply(r, zm)
    torch.cuda.synchronize()
    assert float(torch.linalg.vector_norm(zm - z2)) <= 1e-10 * float(torch.linalg.vector_norm(z2))


def test_multilevel_newton_solve_fp32():
    from workloads import box_groups
    prob = slab_problem(8, 8, 8, order=1, parts=(4, 4, 4), pressure=1e3, gamma=3e4, load_steps=4)
    P = pkg.Problem(prob)
    part2, n2 = box_groups((4, 4, 4), (2, 2, 2))
    d2, rep2 = P.solve(pkg.SolveOptions(precision=pkg.FP32, primal="VE"))
    dm, repm = P.solve(pkg.SolveOptions(precision=pkg.FP32, primal="VE", levels=3, part2=part2,
                                        n_parts2=n2, primal2="VEF"))
    assert repm["status"] == 0 and repm["load_steps_done"] == 4
    assert repm["final_rel_residual"] <= 1e-8
    assert repm["total_gmres_its"] >= rep2["total_gmres_its"]
    assert float(torch.linalg.vector_norm(dm - d2)) <= 1e-6 * float(torch.linalg.vector_norm(d2))


@pytest.mark.parametrize("config", ["ragged", "slab48_q1"])
def test_tensor_core_setup_accuracy(config):
    """FP32 local operators from the tcgen05 setup GEMMs against those from
    FP32 CUDA-core GEMMs, by the BDDC apply's distance to the FP64 apply
    (element by element and in norm).  The Gauss-Jordan sweep updates on the
    tensor cores (one K-step per TMEM slice, slices summed in FP32 on the
    CUDA cores; mode 9 keeps the other products on the CUDA cores) are as
    accurate as on the CUDA cores.  The other products on the tensor cores
    (mode 1, the default) add a 32-wide K block per slice with truncation and
    lose a little more: within 16x the CUDA-core distance (measured: 11.3x
    on the ragged slab, 1.6x on slab48) and within the FP32 apply bar 1e-3.
    Mode 9 is held to 2x (measured at most 1.6x); mode 65 (the other
    products also one K-step per slice) measured 3.8x on the ragged slab."""
    prob = slab_problem(order=1, **RAGGED) if config == "ragged" else slab_config(config)
    P = pkg.Problem(prob)
    fe = FEProblem(prob)
    d = smooth_displacement(fe, seed=31) if config == "ragged" else np.zeros(fe.n_free)
    P.assemble_tangent(_dev(d), 0.75)
    r = _dev(np.random.default_rng(12).standard_normal(fe.n_free))
    primal = "VEF" if config == "ragged" else prob["primal"]

    def apply(precision, mode):
        prev = pkg.set_tensor_cores(mode)
        try:
            pc = pkg.BDDC(P, precision=precision, primal=primal).setup()
            z = torch.empty_like(r)
            pc.apply(r, z)
            return _host(z)
        finally:
            pkg.set_tensor_cores(prev)

    z64 = apply(pkg.FP64, 1)
    z_cc = apply(pkg.FP32, 0)
    e_cc = np.linalg.norm(z_cc - z64) / np.linalg.norm(z64)
    m_cc = np.abs(z_cc - z64).max() / np.abs(z64).max()
    assert e_cc <= 1e-3
    for mode, factor in ((9, 2.0), (1, 16.0), (65, 16.0)):
        z_tc = apply(pkg.FP32, mode)
        e_tc = np.linalg.norm(z_tc - z64) / np.linalg.norm(z64)
        m_tc = np.abs(z_tc - z64).max() / np.abs(z64).max()
        assert e_tc <= 1e-3
        assert e_tc <= factor * e_cc, (mode, e_tc, e_cc)
        assert m_tc <= factor * m_cc, (mode, m_tc, m_cc)
