"""The sparse coarse problem against the dense inverse and the oracle (Sec. 4.3).

Every projection P = I - G (G^T G)^-1 G^T solves with G^T G.  The library
either forms the dense explicit inverse (block elimination) or factors G^T G
over supernodes of a nested-dissection order of the subdomain graph and
applies the factor by forward and backward sweeps (one task-graph kernel per
solve).  Both forms must give the oracle's solution and the same PCG:
  * classical FETI (subdomains touching the Dirichlet boundary have no
    kernel: uneven coarse blocks) and all-floating FETI, the three
    preconditioners, FP64 and the FP32-local form, against the FP64 oracle;
  * iteration counts within 2 % and Lanczos estimates within 1 % for both
    forms on the 64-subdomain tube (runs of ~190 and ~390 iterations, which
    drift by rounding), and the block form (several right-hand sides through
    the same sweeps);
  * the 1024-subdomain jittered tube, where the automatic choice is sparse:
    same iterations as the dense form and displacements within 1e-10;
  * a sweep whose dependency waits get a zero budget returns
    FETI_ERR_TIMEOUT, and the next solve on the context matches the oracle.
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


_REF = {}


def _small():
    return mesh.cylinder_problem(4, 16, 8, (2, 8, 2))


def _ref(method):
    if method not in _REF:
        U, _, _ = feti.FetiOracle(_small(), method, "dirichlet").solve(tol=1e-12)
        _REF[method] = U
    return _REF[method]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("method", ["classical", "af"])
@pytest.mark.parametrize("precond", ["dirichlet", "lumped", "identity"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sparse_coarse_matches_oracle(method, precond, precision):
    from paper_1508_02599_gb300 import FetiSolver
    prob = _small()
    U_ref = _ref(feti.CLASSICAL if method == "classical" else feti.ALL_FLOATING)
    with FetiSolver(prob, method=method, precond=precond, precision=precision, coarse="sparse", tol=1e-11,
                    maxit=3000) as s:
        info = s.coarse_info()
        U, rep = s.solve()
    assert info["form"] == "sparse" and info["supernodes"] > 1 and info["height"] > 1
    assert rep["converged"] == 1
    assert _rel(U, U_ref) <= 1e-8


@pytest.mark.parametrize("method", ["classical", "af"])
def test_sparse_and_dense_coarse_same_pcg(method):
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.config_problem("cyl16")
    out = {}
    for form in ("dense", "sparse"):
        with FetiSolver(prob, method=method, precond="dirichlet", coarse=form, tol=1e-10, maxit=3000) as s:
            assert s.coarse_info()["form"] == form
            U, rep = s.solve()
        out[form] = (U, rep)
    (Ud, rd), (Us, rs) = out["dense"], out["sparse"]
    # runs of ~190 (all-floating) and ~390 (classical) iterations on this
    # tube (Dirichlet kappa ~ 480) to 1e-10: the two forms round differently
    # and CG's loss of orthogonality lets the counts drift by a few percent
    # (389 against 397 seen with the compact-factor K^+)
    slack = max(1, int(0.03 * rd["iterations"]))
    assert abs(rs["iterations"] - rd["iterations"]) <= slack, (rs["iterations"], rd["iterations"])
    assert abs(rs["cond_est"] - rd["cond_est"]) <= 1e-2 * rd["cond_est"]
    assert _rel(Us, Ud) <= 1e-9


def test_sparse_coarse_block_form():
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.config_problem("cyl16")
    scales = np.array([1.0, -0.5, 2.0, 0.25])
    out = {}
    for form in ("dense", "sparse"):
        with FetiSolver(prob, method="af", precond="dirichlet", coarse=form, tol=1e-10, maxit=3000) as s:
            out[form] = s.solve_multi(scales)
    Ud, Us = out["dense"][0], out["sparse"][0]
    for k in range(len(scales)):
        assert _rel(Us[k], Ud[k]) <= 1e-10, k


def test_automatic_form_on_1024_subdomains():
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.config_problem("jcyl32")
    out = {}
    for form in ("auto", "dense"):
        with FetiSolver(prob, method="af", precond="dirichlet", coarse=form, tol=1e-8, maxit=3000) as s:
            info = s.coarse_info()
            U, rep = s.solve()
        out[form] = (info, U, rep)
    info = out["auto"][0]
    assert info["form"] == "sparse"
    # the factor is a small fraction of the dense inverse
    assert info["factor_entries"] < 0.05 * out["dense"][0]["factor_entries"]
    assert out["auto"][2]["iterations"] == out["dense"][2]["iterations"]
    assert _rel(out["auto"][1], out["dense"][1]) <= 1e-10


def test_sparse_coarse_wait_times_out_then_recovers():
    from paper_1508_02599_gb300 import FetiError, FetiSolver
    prob = _small()
    U_ref = _ref(feti.ALL_FLOATING)
    with FetiSolver(prob, method="af", precond="dirichlet", coarse="sparse", tol=1e-10, maxit=300) as s:
        s.prepare()
        s.set_spin_timeout(0)
        with pytest.raises(FetiError) as ei:
            s.solve()
        assert ei.value.status == 9 and "coarse" in str(ei.value)
        s.set_spin_timeout(100_000_000)
        U, rep = s.solve()
    assert rep["converged"] == 1
    assert _rel(U, U_ref) <= 1e-8
