"""The full-size workloads (Q2 slab, P1 and P2 ventricles) in the launch
configuration the benchmark times: outputs the oracle computes at full size
(residuals, BDDC applies on the Q2 slab) element by element, and properties
that hold at any size elsewhere (the tangent against central differences of
the residual, the Newton step's reported residual against the oracle's
residual at the updated state)."""
import numpy as np
import pytest

from oracle.assembly import FEProblem
from oracle.bddc import BDDC as OracleBDDC
from workloads import slab_config, lv_config

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


def test_slab24_q2_full_size_residual_and_apply():
    prob = slab_config("slab24_q2")
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    assert P.n_free == fe.n_free == 86436
    lam = 0.25
    d = np.zeros(fe.n_free)
    r = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(_dev(d), lam, r)
    r_ref = fe.residual(d, lam)
    assert np.abs(_host(r) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    K_ref, (Ke, Kf) = fe.tangent(d, lam)
    ref = OracleBDDC(fe, Ke, Kf, "VEF")
    z_ref = ref.apply(-r_ref)
    for precision, tol in ((pkg.FP64, 1e-9), (pkg.FP32, 1e-3)):
        pc = pkg.BDDC(P, precision=precision, primal="VEF").setup()
        assert pc.info()["n_primal"] == ref.n_pi
        z = torch.empty_like(r)
        pc.apply(_dev(-r_ref), z)
        assert np.linalg.norm(_host(z) - z_ref) <= tol * np.linalg.norm(z_ref)
        assert np.abs(_host(z) - z_ref).max() <= 2 * tol * np.abs(z_ref).max()


def _fd_tangent_check(P, d, lam, seed):
    """||K v - (F(d + e v) - F(d - e v)) / 2e|| relative, through the ABI."""
    n = P.n_free
    v = _dev(np.random.default_rng(seed).standard_normal(n))
    r = torch.empty(n, dtype=torch.float64, device="cuda")
    P.assemble_tangent(d, lam, r)
    kv = torch.empty_like(r)
    P.spmv(v, kv)
    eps = 1e-7 * float(torch.linalg.vector_norm(d)) / float(torch.linalg.vector_norm(v))
    rp, rm = torch.empty_like(r), torch.empty_like(r)
    P.residual(d + eps * v, lam, rp)
    P.residual(d - eps * v, lam, rm)
    fd = (rp - rm) / (2 * eps)
    return float(torch.linalg.vector_norm(kv - fd) / torch.linalg.vector_norm(kv))


@pytest.mark.parametrize("name", ["lv_p1", "lv_p2"])
def test_lv_full_size_newton_step(name):
    prob = lv_config(name)
    fe = FEProblem(prob)
    P = pkg.Problem(prob)
    assert P.n_free == fe.n_free
    lam = 1.0 / prob["load_steps"]
    d0 = np.zeros(fe.n_free)
    r = torch.empty(fe.n_free, dtype=torch.float64, device="cuda")
    P.residual(_dev(d0), lam, r)
    r_ref = fe.residual(d0, lam)
    assert np.abs(_host(r) - r_ref).max() <= 1e-12 * np.abs(r_ref).max()
    ml = {}
    if name == "lv_p2":
        ml = dict(levels=3, part2=prob["part2"], n_parts2=prob["n_parts2"], primal2="VEF",
                  precision2=pkg.FP32)
    opts = pkg.SolveOptions(precision=pkg.FP32, primal=prob["primal"], **ml)
    d = _dev(d0)
    rec, ctx = P.newton_step(d, lam, opts)
    assert rec["status"] == 0 and rec["gmres_its"] < 1000
    assert abs(rec["res"] - np.linalg.norm(r_ref)) <= 1e-12 * np.linalg.norm(r_ref)
    # residual at the updated state: GPU against the oracle, and progress
    dh = _host(d)
    r1 = fe.residual(dh, lam)
    P.residual(d, lam, r)
    assert np.abs(_host(r) - r1).max() <= 1e-11 * np.abs(r_ref).max()
    assert np.linalg.norm(r1) < 0.5 * np.linalg.norm(r_ref)
    # tangent at the new state against central differences of the residual
    assert _fd_tangent_check(P, d, lam, seed=3) <= 1e-6
