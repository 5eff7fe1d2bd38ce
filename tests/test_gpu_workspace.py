"""Grouped local factorizations and the compact interior factor (Sec. 4.4).

The dense elimination workspace holds one group of subdomains at a time
(workspace_mb); after each group the interior columns of its factor (L_II,
L_bI) are kept in a compact array and every K^+ solve takes the boundary block
through the explicit F_i.  Each subdomain's elimination is independent of the
others, so:
  * the solution is bit-identical whatever the grouping (one subdomain per
    group up to all in one), for every precision form, both methods and the
    lumped preconditioner (whose K_bb values are read per group);
  * with several groups the workspace is the largest group's, far below the
    whole dense workspace, and the compact factor is smaller still;
  * the FP64 solve through the compact factor matches the FP64 oracle
    (iterations +-1 around the oracle's steps within 5 % of the threshold,
    displacement to 1e-9);
  * the implicit local form keeps the whole factor in one group.
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


def _solve(prob, **kw):
    from paper_1508_02599_gb300 import FetiSolver
    with FetiSolver(prob, tol=1e-10, maxit=3000, **kw) as s:
        U, rep = s.solve()
        info = s.factor_info()
    assert rep["converged"] == 1
    return U, rep, info


@pytest.mark.parametrize("method,precond,precision", [
    ("af", "dirichlet", "fp64"), ("af", "dirichlet", "mixed"), ("af", "dirichlet", "mixed_f32factor"),
    ("classical", "dirichlet", "fp64"), ("af", "lumped", "fp64"), ("af", "lumped", "mixed_f32factor"),
])
def test_grouping_is_bit_identical(method, precond, precision):
    prob = _small()
    ref, rep_ref, info_ref = _solve(prob, method=method, precond=precond, precision=precision, workspace_mb=-1)
    assert info_ref["groups"] == 1 and info_ref["workspace"] == info_ref["full_workspace"]
    # 1 MiB: a few subdomains per group; every matrix here is well below it
    U, rep, info = _solve(prob, method=method, precond=precond, precision=precision, workspace_mb=1)
    assert info["groups"] > 4, info
    assert info["workspace"] * info["elem_bytes"] <= 1 << 20   # every subdomain's matrix is below 0.6 MiB here
    assert info["workspace"] < info["full_workspace"] // 4
    assert 0 < info["compact"] < info["full_workspace"]
    assert rep["iterations"] == rep_ref["iterations"]
    assert np.array_equal(U, ref)


def test_compact_factor_fp64_matches_oracle():
    prob = _small()
    o = feti.FetiOracle(prob, feti.ALL_FLOATING, "dirichlet")
    _, res8, _ = o.solve(tol=1e-8, maxit=3000)
    U_ref, res12, _ = o.solve(tol=1e-12, maxit=3000)
    from paper_1508_02599_gb300 import FetiSolver
    with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-8, maxit=3000, workspace_mb=1) as s:
        _, rep8 = s.solve()
    U, rep, info = _solve(prob, method="af", precond="dirichlet", precision="fp64", workspace_mb=1)
    assert info["groups"] > 4
    assert count_matches(rep8["iterations"], res12.res_hist, 1e-8), (rep8["iterations"], res8.iterations)
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)


def test_implicit_form_keeps_whole_factor():
    _, _, info = _solve(_small(), method="af", precond="dirichlet", precision="fp64", local_form="implicit",
                        workspace_mb=1)
    assert info["groups"] == 1 and info["compact"] == 0
    assert info["workspace"] == info["full_workspace"]


def test_workspace_option_rejected():
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    with pytest.raises(FetiError) as ei:
        FetiSolver(_small(), method="af", precond="dirichlet", workspace_mb=-2)
    assert ei.value.status == 1
