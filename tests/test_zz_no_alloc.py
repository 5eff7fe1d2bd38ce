"""The allocation-free dual apply (feti_dual_apply_noalloc) against feti_dual_apply.

Some callers cannot allocate device memory once the solver is set up (a fixed
memory budget reserved at start-up, a latency-critical loop that must not hit
cudaMalloc's implicit synchronisation, or a phase in which another component
owns the allocator).  They call feti_dual_apply_noalloc, which keeps its
scratch in a static device array.  This file runs last in the suite so that a
failure here never hides the other tests; it passes in a fresh process and
after the rest of the suite alike.  Around every allocation-free call the
device's free memory (cudaMemGetInfo) must stay the same: the static array and
its module are set up by feti_create, not by the call.  Tolerance: the same kernels run on the
same data, so results agree to 1e-12 relative (the bound the other operator
tests use).  The allocation-free apply uses the full-row local kernels, so the
solver here keeps its FP32 applies on full rows too (symmetric="off"); with
the symmetric FP32 kernel the two would differ by FP32 rounding only.
"""
import numpy as np
import pytest

from feti_inputs import mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision,precond", [("fp64", "dirichlet"), ("mixed", "dirichlet"), ("fp64", "lumped")])
def test_noalloc_apply_matches_dual_apply_twice(precision, precond):
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(4, 16, 8, (2, 8, 2))
    rng = np.random.default_rng(41)
    with FetiSolver(prob, method="af", precond=precond, precision=precision, symmetric="off") as s:
        s.prepare()
        nl = s.sizes()["n_lambda"]
        for call in range(2):
            v = torch.tensor(rng.normal(size=nl), device="cuda", dtype=torch.float64)
            q_ref, z_ref = torch.empty_like(v), torch.empty_like(v)
            s.dual_apply(v, q_ref, z_ref, 1)
            q, z = torch.full_like(v, np.nan), torch.full_like(v, np.nan)
            torch.cuda.synchronize()
            free0, _ = torch.cuda.mem_get_info()
            s.dual_apply_noalloc(v, q, z)
            torch.cuda.synchronize()
            free1, _ = torch.cuda.mem_get_info()
            assert free1 == free0, (call, free0 - free1)
            assert torch.isfinite(q).all() and torch.isfinite(z).all()
            assert (q - q_ref).abs().max().item() <= 1e-12 * q_ref.abs().max().item(), call
            assert (z - z_ref).abs().max().item() <= 1e-12 * z_ref.abs().max().item(), call


def test_noalloc_rejects_oversized_decomposition():
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    prob = mesh.config_problem("jcyl32")   # about 0.9 M boundary DOFs: beyond the static scratch
    with FetiSolver(prob, method="af", precond="dirichlet") as s:
        v = torch.zeros(s.sizes()["n_lambda"], device="cuda", dtype=torch.float64)
        with pytest.raises(FetiError) as ei:
            s.dual_apply_noalloc(v, torch.empty_like(v), torch.empty_like(v))
        assert ei.value.status == 1 and "scratch" in str(ei.value)
