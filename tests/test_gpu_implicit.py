"""The implicit local form against the explicit one and the oracle (Sec. 4.3).

Inside the PCG, y_i = K_i^+ B_i^T lambda is either the explicit
F_i = (S_i[b',b'])^-1 applied as a dense matvec (the default) or, with
local_form "implicit" (the paper's sparse-direct form), a forward and a
backward triangular sweep over the local Cholesky factor on the placed
boundary vector every iteration.  Both are F_i v up to rounding:
  * one dual apply agrees element-wise to 1e-12 of its largest entry;
  * solves match the FP64 oracle (iterations +-1 with the Dirichlet
    preconditioner, around the oracle's steps within 5 % of the threshold,
    see pcg_counts; displacement to 1e-9) for both FETI methods;
  * the implicit form is FP64 only: another precision is rejected.
"""
import numpy as np
import pytest

from feti_inputs import mesh
from pcg_counts import count_matches
from oracle import feti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _small():
    return mesh.cylinder_problem(4, 16, 8, (2, 8, 2))


def test_implicit_dual_apply_matches_explicit():
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.config_problem("cyl16")
    out = {}
    for form in ("explicit", "implicit"):
        with FetiSolver(prob, method="af", precond="dirichlet", local_form=form) as s:
            s.prepare()
            nl = s.sizes()["n_lambda"]
            v = torch.tensor(np.random.default_rng(3).normal(size=nl), device="cuda", dtype=torch.float64)
            q = torch.empty_like(v)
            z = torch.empty_like(v)
            s.dual_apply(v, q, z, 1)
            torch.cuda.synchronize()
            out[form] = (q.cpu().numpy(), z.cpu().numpy())
    for i in range(2):
        a, b = out["implicit"][i], out["explicit"][i]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), i


@pytest.mark.parametrize("method", ["classical", "af"])
def test_implicit_solve_matches_oracle(method):
    from paper_1508_02599_gb300 import FetiSolver
    prob = _small()
    m = feti.CLASSICAL if method == "classical" else feti.ALL_FLOATING
    o = feti.FetiOracle(prob, m, "dirichlet")
    _, res8, _ = o.solve(tol=1e-8, maxit=3000)
    U_ref, res12, _ = o.solve(tol=1e-12, maxit=3000)
    with FetiSolver(prob, method=method, precond="dirichlet", local_form="implicit", tol=1e-8, maxit=3000) as s:
        _, rep8 = s.solve()
    with FetiSolver(prob, method=method, precond="dirichlet", local_form="implicit", tol=1e-12, maxit=3000) as s:
        U, rep = s.solve()
    assert rep8["converged"] == 1 and rep["converged"] == 1
    assert count_matches(rep8["iterations"], res12.res_hist, 1e-8), (rep8["iterations"], res8.iterations)
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_implicit_form_needs_fp64():
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    with pytest.raises(FetiError) as ei:
        FetiSolver(_small(), method="af", precond="dirichlet", precision="mixed", local_form="implicit")
    assert ei.value.status == 1
