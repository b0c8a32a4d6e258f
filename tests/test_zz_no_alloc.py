"""bddc_apply_noalloc: the BDDC apply for callers that may not allocate
device memory while they run (code paths where cudaMalloc is not allowed,
or whose device memory was budgeted up front).  Its work vectors live in a
static device array of the library, so the call allocates nothing; it must
give the same result as bddc_apply.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2208_06191_gb300 as pkg  # noqa: E402
from workloads import box_groups, slab_problem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    pkg.build()
    pkg.load_library()


def _smooth(prob):
    X = np.asarray(prob["coords"])
    free = np.setdiff1d(np.arange(X.shape[0]), prob["dirichlet_nodes"])
    Xf = X[free]
    return (0.02 * Xf[:, 2:3] * np.sin(Xf + 1.0)).reshape(-1)


def _check_two_calls(pc, n, seed):
    """bddc_apply_noalloc runs the kernels of bddc_apply in the same order on
    the same operators, so the two results must agree bit for bit; a
    misplaced work vector inside the static array would break that."""
    rng = np.random.default_rng(seed)
    for _ in range(2):
        r = torch.as_tensor(rng.standard_normal(n), dtype=torch.float64, device="cuda")
        z_ref = torch.empty_like(r)
        z = torch.full_like(r, float("nan"))
        pc.apply(r, z_ref)
        pc.apply_noalloc(r, z)
        torch.cuda.synchronize()
        assert bool(torch.isfinite(z_ref).all())
        assert torch.equal(z, z_ref)


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32])
def test_apply_noalloc_matches_apply_on_two_calls(precision):
    prob = slab_problem(5, 4, 3, order=1, parts=(2, 2, 2), jitter=0.2, pressure=2.0e3, gamma=3.0e4)
    P = pkg.Problem(prob)
    d = torch.as_tensor(_smooth(prob), dtype=torch.float64, device="cuda")
    P.assemble_tangent(d, 0.8)
    pc = pkg.BDDC(P, precision=precision, primal="VEF").setup()
    _check_two_calls(pc, P.n_free, 42)


@pytest.mark.parametrize("precision", [pkg.FP64, pkg.FP32])
def test_apply_noalloc_three_levels(precision):
    # 32 box subdomains grouped into 4 level-2 subdomains: the level-2 apply
    # runs on the level-2 context's own (setup-time) vectors
    prob = slab_problem(8, 8, 4, order=1, parts=(4, 4, 2), jitter=0.15, pressure=1.0e3, gamma=3.0e4)
    P = pkg.Problem(prob)
    d = torch.as_tensor(_smooth(prob), dtype=torch.float64, device="cuda")
    P.assemble_tangent(d, 0.8)
    part2, n2 = box_groups((4, 4, 2), (2, 2, 1))
    pc = pkg.BDDC(P, precision=precision, primal="VE", levels=3, part2=part2, n_parts2=n2,
                  primal2="VEF", precision2=precision).setup()
    _check_two_calls(pc, P.n_free, 43)


def test_apply_noalloc_rejects_contexts_beyond_its_buffer():
    # 800 subdomains of 4x4x4 elements: the per-apply work vectors exceed 4 MiB.
    prob = slab_problem(80, 80, 8, order=1, lengths=(10.0, 10.0, 1.0), parts=(20, 20, 2),
                        pressure=1.0e3, gamma=1.0e4)
    P = pkg.Problem(prob)
    d = torch.zeros(P.n_free, dtype=torch.float64, device="cuda")
    P.assemble_tangent(d, 0.5)
    pc = pkg.BDDC(P, precision=pkg.FP32, primal="V").setup()
    r = torch.ones(P.n_free, dtype=torch.float64, device="cuda")
    z = torch.empty_like(r)
    with pytest.raises(pkg.CBDDCError) as ei:
        pc.apply_noalloc(r, z)
    assert ei.value.code == pkg.EINVAL
    assert "static buffer" in str(ei.value)
    pc.apply(r, z)  # the allocating path still serves it
    torch.cuda.synchronize()
    assert bool(torch.isfinite(z).all())
