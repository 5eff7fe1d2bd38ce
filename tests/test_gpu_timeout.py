"""Bounded device waits that run out: FETI_ERR_TIMEOUT, then a usable context.

The streamed symmetric FP32 apply and the warp-specialised tensor-core block
GEMMs (one tile per CTA, and the persistent kernel) wait on mbarriers for their bulk / tensor-map copies and tensor-core
products.  Their main-loop waits give up after the context's spin timeout
(feti_options.spin_timeout_ns, feti_set_spin_timeout).  Here that budget is
set to zero after set-up, so every main-loop wait gives up at its first check
while the copies it waits for are still in flight; each kernel then stops its
pipeline, waits for what it issued (those drain waits keep their full
budget), releases tensor memory and flags the call.  The solve must return FETI_ERR_TIMEOUT (9), and the next solve on the
same context, with the default budget again, must match the FP64 oracle.
Nothing traps, faults or spins without a bound.
"""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import feti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture(scope="module")
def case():
    prob = mesh.cylinder_problem(4, 16, 8, (2, 8, 2))
    U_ref, _, _ = feti.FetiOracle(prob, feti.ALL_FLOATING, "dirichlet").solve(tol=1e-12)
    return prob, U_ref


def _rel(U, U_ref):
    return float(np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref))


def test_streamed_symmetric_apply_times_out_then_recovers(case):
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    prob, U_ref = case
    with FetiSolver(prob, method="af", precond="dirichlet", precision="mixed", symmetric="force_streamed",
                    tol=1e-10, maxit=60) as s:
        s.prepare()
        assert s.schedule()["fp32_F"][0] == -64          # the streamed kernel is the one in use
        s.set_spin_timeout(0)
        with pytest.raises(FetiError) as ei:
            s.solve()
        assert ei.value.status == 9 and "bounded wait" in str(ei.value)
        s.set_spin_timeout(100_000_000)
        U, rep = s.solve()
        assert rep["converged"] == 1
        assert _rel(U, U_ref) <= 1e-8


@pytest.mark.parametrize("variant,code", [("force_ws3", -3), ("force_persist", -5), ("force_persist_c3", -7)])
def test_tensor_core_block_gemm_times_out_then_recovers(case, variant, code):
    """The warp-specialised one-tile kernel and the persistent kernel."""
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    prob, U_ref = case
    scales = np.array([1.0, 2.5])
    with FetiSolver(prob, method="af", precond="dirichlet", precision="mixed", tensor_cores=variant,
                    tol=1e-10, maxit=60) as s:
        U, _ = s.solve_multi(scales)                     # tunes the block schedules with the default budget
        assert s.schedule()["block_fp32_F"][0] == code   # that tensor-core kernel
        s.set_spin_timeout(0)
        with pytest.raises(FetiError) as ei:
            s.solve_multi(scales)
        assert ei.value.status == 9 and "bounded wait" in str(ei.value)
        s.set_spin_timeout(100_000_000)
        U, rep = s.solve_multi(scales)
        assert rep["converged"] == 1
        for k, sc in enumerate(scales):
            assert _rel(U[k], sc * U_ref) <= 1e-8
