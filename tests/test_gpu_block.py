"""Block form (several load cases sharing each operator apply) against the single-RHS path and the oracle.

The load cases are f_k = s_k f with homogeneous Dirichlet data, so the exact
answers are u_k = s_k u.  Tolerances: FP64 block vs oracle 1e-9 relative
(both at a projected residual of 1e-12); mixed block 1e-8; a block operator
apply equals the single-RHS apply column by column to 1e-12 (FP64: the same
products in a different association order).
"""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import feti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TUBE_FLOAT = mesh.cylinder_problem(4, 16, 8, (2, 8, 2))
SCALES = [1.0, 2.5, 0.7, 1.6]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision,precond,tol", [("fp64", "dirichlet", 1e-9), ("mixed", "dirichlet", 1e-8),
                                                   ("fp64", "lumped", 1e-9), ("fp64", "identity", 1e-9)])
def test_block_solve_matches_oracle(precision, precond, tol):
    from paper_1508_02599_gb300 import FetiSolver
    prob = TUBE_FLOAT
    o = feti.FetiOracle(prob, "af", precond)
    U_ref, _, _ = o.solve(tol=1e-12, maxit=3000)
    with FetiSolver(prob, method="af", precond=precond, tol=1e-12 if precision == "fp64" else 1e-11, maxit=5000,
                    precision=precision) as s:
        U, rep = s.solve_multi(SCALES)
    assert rep["converged"] == 1
    for k, sc in enumerate(SCALES):
        assert np.linalg.norm(U[k] - sc * U_ref) <= tol * np.linalg.norm(sc * U_ref)


def test_block_apply_equals_single_applies():
    from paper_1508_02599_gb300 import FetiSolver
    prob = TUBE_FLOAT
    rng = np.random.default_rng(2)
    with FetiSolver(prob, method="af", precond="dirichlet") as s:
        s.prepare()
        nl = s.sizes()["n_lambda"]
        V = torch.tensor(rng.normal(size=(nl, 5)), device="cuda", dtype=torch.float64)
        Q = torch.empty_like(V)
        Z = torch.empty_like(V)
        s.dual_apply_multi(V, Q, Z, 5, 2)
        for k in range(5):
            v = V[:, k].contiguous()
            q = torch.empty_like(v)
            z = torch.empty_like(v)
            s.dual_apply(v, q, z, 1)
            torch.cuda.synchronize()
            assert (Q[:, k] - q).abs().max().item() <= 1e-12 * q.abs().max().item()
            assert (Z[:, k] - z).abs().max().item() <= 1e-12 * z.abs().max().item()


JITTER = mesh.jittered_cylinder_problem(6, 24, 12, 24, mesh_seed=7, part_seed=8)


@pytest.mark.parametrize("prob", [TUBE_FLOAT, JITTER], ids=["tube", "jittered"])
@pytest.mark.parametrize("variant,code", [("force_reg", 0), ("force_bulk", -1), ("force_tma", -2),
                                          ("force_ws3", -3), ("force_ws2", -4), ("force_persist", -5),
                                          ("force_persist_q3", -6), ("force_persist_c3", -7)])
def test_tensor_core_block_gemm_matches_cuda_cores(prob, variant, code):
    """Each tcgen05 3xTF32 block GEMM (register-staged, bulk-copy staged,
    tensor-map fed, warp-specialised with 3 and 2 stages, persistent) against the CUDA-core FP32 GEMM on the same FP32 operator
    copies: agreement to 1e-5 relative (TF32 head + tail products reproduce
    FP32 products to about 2^-22 each), on subdomains whose boundary sizes are
    not multiples of the 32-column chunk or the 128-row tile; then a full
    block solve on the tensor cores against the oracle."""
    from paper_1508_02599_gb300 import FetiSolver
    outs = {}
    for tc in ("off", variant):
        with FetiSolver(prob, method="af", precond="dirichlet", precision="mixed", tensor_cores=tc) as s:
            s.prepare()
            nl = s.sizes()["n_lambda"]
            V = torch.tensor(np.random.default_rng(8).normal(size=(nl, 16)), device="cuda", dtype=torch.float64)
            Q = torch.empty_like(V)
            Z = torch.empty_like(V)
            s.dual_apply_multi(V, Q, Z, 16, 1)
            torch.cuda.synchronize()
            outs[tc] = (Q.cpu().numpy(), Z.cpu().numpy(), s.schedule())
    assert outs[variant][2]["block_fp32_F"][0] == code      # that tensor-core kernel ran
    assert outs[variant][2]["block_fp32_M"][0] == code
    assert outs["off"][2]["block_fp32_F"][0] > 0
    for i in range(2):
        a, b = outs[variant][i], outs["off"][i]
        assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()
    o = feti.FetiOracle(prob, "af", "dirichlet")
    U_ref, _, _ = o.solve(tol=1e-12, maxit=3000)
    with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-11, maxit=5000, precision="mixed",
                    tensor_cores=variant) as s:
        U, rep = s.solve_multi(SCALES)
    assert rep["converged"] == 1
    for k, sc in enumerate(SCALES):
        assert np.linalg.norm(U[k] - sc * U_ref) <= 1e-8 * np.linalg.norm(sc * U_ref)


def _linear_residual(prob, U, chunk=262144):
    """||K u - f|| / ||f|| on the free DOFs, K u formed element by element
    from the oracle's linear element matrices (chunked: bounded host memory)."""
    from oracle import fem
    Ur = U.reshape(-1, 3)
    out = np.zeros(U.size)
    E = prob.tets.shape[0]
    for s0 in range(0, E, chunk):
        t = prob.tets[s0:s0 + chunk]
        Ke = fem.linear_element(prob.coords[t], prob.material["E"], prob.material["nu"])
        fe = np.einsum("eij,ej->ei", Ke, Ur[t].reshape(-1, 12))
        np.add.at(out, (3 * t[:, :, None] + np.arange(3)[None, None, :]).reshape(-1), fe.ravel())
    f = fem.load_vector(prob)
    free = np.ones(U.size, bool)
    free[prob.dir_dof] = False
    return np.linalg.norm((out - f)[free]) / np.linalg.norm(f[free])


@pytest.mark.slow
def test_full_size_4096_subdomains_16_rhs():
    """The 48x192x96-cell jittered tube (2,737,728 DOFs) in 4096 uneven
    subdomains, 16 load cases p_k ~ U[8, 16] (seeded), FP32-local block PCG
    (FP64 outer residual) to 1e-10 on one GPU.  The load cases are collinear, so u_k / p_k must agree
    across k; each u_k is checked for equilibrium by the oracle's element
    route (K u_k formed element by element on the host)."""
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.config_problem("jcyl48")
    scales = np.random.Generator(np.random.PCG64(16)).uniform(8.0, 16.0, size=16)
    with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-10, maxit=6000, precision="mixed") as s:
        U, rep = s.solve_multi(scales)
        sz = s.sizes()
    assert rep["converged"] == 1
    assert sz["coarse_dim"] == 6 * 4096
    base = U[0] / scales[0]
    for k in range(16):
        assert np.linalg.norm(U[k] / scales[k] - base) <= 1e-7 * np.linalg.norm(base)
    for k in (0, 15):
        assert _linear_residual(prob, U[k] / scales[k]) <= 1e-6
