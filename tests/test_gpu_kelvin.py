"""Kelvin-solution cube with 512 sub-cubes (the shape of Sec. 5.1 / Table 2) on the GPU.

Parity with the oracle at 16^3 cells (both preconditioned forms), then the
trends and magnitudes of Table 2 and the P1 order of convergence from the GPU
solutions at 16^3 and 32^3 cells (closed-form exact solution).
"""
import os

import numpy as np
import pytest

from feti_inputs import mesh
from pcg_counts import count_matches
from oracle import fem, feti

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table2_cube_p1.txt")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _l2(prob, U):
    uex = mesh.kelvin_displacement(prob.coords, prob.material["E"], prob.material["nu"])
    e = U.reshape(-1, 3) - uex
    _, V = fem.shape_gradients(prob.coords[prob.tets])
    return np.sqrt((V * (e[prob.tets] ** 2).sum(axis=2).mean(axis=1)).sum())


def _table2():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or line.startswith("eoc") or not line.strip():
            continue
        lvl, m, pc, it, kappa = line.split()
        rows[int(lvl), m, pc] = (int(it), float(kappa))
    return rows


@pytest.mark.parametrize("method", ["af", "classical"])
def test_kelvin_512_matches_oracle(method):
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.kelvin_cube_problem(16)
    o = feti.FetiOracle(prob, method, "dirichlet")
    U_ref, res, _ = o.solve(tol=1e-12, maxit=2000)
    _, res8, _ = o.solve(tol=1e-8, maxit=2000)
    with FetiSolver(prob, method=method, precond="dirichlet", tol=1e-12) as s:
        U, rep = s.solve()
    with FetiSolver(prob, method=method, precond="dirichlet", tol=1e-8) as s:
        _, rep8 = s.solve()
    assert np.linalg.norm(U - U_ref) <= 1e-9 * np.linalg.norm(U_ref)
    assert count_matches(rep8["iterations"], res.res_hist, 1e-8), (rep8["iterations"], res8.iterations)


def test_kelvin_table2_trends_and_convergence():
    from paper_1508_02599_gb300 import FetiSolver
    paper = _table2()
    its, kap, err = {}, {}, {}
    for n in (16, 32):
        prob = mesh.kelvin_cube_problem(n)
        for method in ("af", "classical"):
            for pc in ("dirichlet", "lumped", "identity"):
                with FetiSolver(prob, method=method, precond=pc, tol=1e-8, maxit=2000) as s:
                    U, rep = s.solve()
                assert rep["converged"] == 1
                its[n, method, pc] = rep["iterations"]
                kap[n, method, pc] = rep["cond_est"]
                err[n, method, pc] = _l2(prob, U)
    for n in (16, 32):
        for m in ("af", "classical"):
            assert its[n, m, "dirichlet"] <= its[n, m, "lumped"] < its[n, m, "identity"]
        for pc in ("dirichlet", "lumped", "identity"):
            assert its[n, "af", pc] < its[n, "classical", pc]
            # magnitudes: within a factor of two of the paper's levels 1-2
            lo = min(paper[1, m, pc][0] for m in ("af", "classical"))
            hi = max(paper[2, m, pc][0] for m in ("af", "classical"))
            assert 0.5 * lo <= its[n, "af", pc] and its[n, "classical", pc] <= 2.0 * hi
    # P1 convergence of the GPU solutions: eoc ~ 2 (Table 2: 1.94-1.99)
    for key in (("af", "dirichlet"), ("classical", "dirichlet")):
        eoc = np.log2(err[(16,) + key] / err[(32,) + key])
        assert 1.85 < eoc < 2.1
