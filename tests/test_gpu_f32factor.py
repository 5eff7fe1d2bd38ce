"""FP32 local factorizations with FP64-refined K^+ (FETI_MIXED_F32FACTOR) against the FP64 oracle.

The local eliminations (interior columns, Schur complement, F_i = S[b',b']^-1
through the identity augmentation) run in FP32; the inner PCG uses the FP32
explicit operators; the dual right-hand side, the outer FP64 residual and the
recovery apply K^+ by FP32 triangular solves refined against the FP64 element
matrices.  The displacement must match the oracle (plain FP64, Sec. 4.3) to
1e-8 relative at PCG tolerance 1e-10, for classical and all-floating FETI and
every preconditioner, on structured and jittered uneven partitions.
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


def _rel(U, U_ref):
    return float(np.linalg.norm(U - U_ref) / np.linalg.norm(U_ref))


PROBS = {
    "cube6": lambda: mesh.cube_problem(6, (2, 2, 2)),
    "tube": lambda: mesh.cylinder_problem(4, 16, 8, (2, 8, 2)),
    "jtube": lambda: mesh.jittered_cylinder_problem(8, 32, 16, 24, 77, 78),
}


@pytest.mark.parametrize("name", list(PROBS))
@pytest.mark.parametrize("method", ["af", "classical"])
@pytest.mark.parametrize("precond", ["dirichlet", "lumped", "identity"])
def test_f32factor_solve_matches_oracle(name, method, precond):
    from paper_1508_02599_gb300 import FetiSolver
    if name == "jtube" and precond != "dirichlet":
        pytest.skip("preconditioner variants are covered on the structured meshes")
    prob = PROBS[name]()
    U_ref, res, _ = feti.FetiOracle(prob, method, precond).solve(tol=1e-12, maxit=3000)
    with FetiSolver(prob, method=method, precond=precond, precision="mixed_f32factor", tol=1e-10,
                    maxit=3000) as s:
        U, rep = s.solve()
        ref = s.refinement()
    assert rep["converged"] == 1
    assert 1 <= ref["steps"] <= 12 and ref["residual"] <= 1e-10, ref
    assert _rel(U, U_ref) <= 1e-8, (_rel(U, U_ref), rep, ref)


def test_f32factor_block_solve_matches_oracle():
    from paper_1508_02599_gb300 import FetiSolver
    prob = PROBS["tube"]()
    U_ref, _, _ = feti.FetiOracle(prob, "af", "dirichlet").solve(tol=1e-12)
    scales = np.array([1.0, 0.5, 3.0])
    with FetiSolver(prob, method="af", precond="dirichlet", precision="mixed_f32factor", tol=1e-10) as s:
        U, rep = s.solve_multi(scales)
    assert rep["converged"] == 1
    for k, sc in enumerate(scales):
        assert _rel(U[k], sc * U_ref) <= 1e-8


def test_f32factor_operators_close_to_fp64():
    """The FP32-eliminated F_i and S_i differ from the FP64 ones by FP32 rounding
    amplified by the local condition: one dual apply agrees to 1e-3 relative."""
    from paper_1508_02599_gb300 import FetiSolver
    prob = PROBS["tube"]()
    out = {}
    for prec in ("fp64", "mixed_f32factor"):
        with FetiSolver(prob, method="af", precond="dirichlet", precision=prec, symmetric="off") as s:
            s.prepare()
            n = s.sizes()["n_lambda"]
            g = torch.Generator(device="cuda").manual_seed(5)
            v = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
            q, z = torch.empty_like(v), torch.empty_like(v)
            s.dual_apply(v, q, z, 1)
            torch.cuda.synchronize()
            out[prec] = (q.cpu().numpy(), z.cpu().numpy())
    for i in range(2):
        a, b = out["fp64"][i], out["mixed_f32factor"][i]
        assert np.linalg.norm(a - b) <= 1e-3 * np.linalg.norm(a)
