"""Load-stepped Newton runs on the GPU: load paths, long runs and checkpoint/resume.

Sec. 3.2 (Eq. loadStepping) ramps the load in steps tau = s / n; Sec. 5.3 runs
hundreds of such steps and compares the PCG iterations per step of classical
and all-floating FETI.  Here, on the two-fibre hyperelastic tube (Table 1
parameters unless stated):
  * a run stopped after a load step, written to a checkpoint (U, step, tau) and
    resumed with feti_newton_steps ends in the same state as the uninterrupted
    run on the same context, with the same per-step counts;
  * the pressure ramp 0 -> 16 kPa (the ramp of the 256-subdomain configuration)
    in 40 load steps on a small tube (the inner radius grows from 1 to about
    2.34), classical FETI, matches the oracle's Newton method on the assembled
    system along the same path.  (The oracle's FETI-increment Newton stops on
    this path: a local tangent loses positive definiteness under the
    prestress.  The GPU driver takes the full Newton step, shifts the local
    tangents of its FETI preconditioner where needed, and the flexible CG on
    the exact tangent still gives the Newton increment.  All-floating FETI,
    whose every subdomain floats, stalls on this path at 2 kPa: its shifted
    preconditioner is too weak there);
  * a long run (200 load steps, c = 6 kPa, kappa = 1000 kPa, as in Sec. 5.3)
    converges at every step under classical and all-floating FETI, with a
    checkpoint every 50 steps, and reports the PCG iterations per step.
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


def _tube(pressure, material=None):
    return mesh.cylinder_problem(2, 16, 4, (1, 4, 2), material=material or mesh.hgo_material(), pressure=pressure)


def test_resume_from_checkpoint_equals_uninterrupted_run(tmp_path):
    from paper_1508_02599_gb300 import FetiSolver, checkpoint_read, checkpoint_write
    prob = _tube(4.0)
    n = 10
    with FetiSolver(prob, method="classical", precond="dirichlet", tol=1e-12, maxit=3000, n_load_steps=n,
                    newton_tol=1e-7, newton_maxit=30) as s:
        U_full, rep_full, pcg_full, nwt_full = s.newton_steps(1, n)
        U_half, _, pcg_a, nwt_a = s.newton_steps(1, n // 2)
        path = tmp_path / "half.ckp"
        checkpoint_write(path, U_half, n // 2, n, (n // 2) / n)
        U0, step, n_steps, tau = checkpoint_read(path)
        assert (step, n_steps, tau) == (n // 2, n, 0.5)
        U_res, rep_res, pcg_b, nwt_b = s.newton_steps(step + 1, n_steps, U_start=U0)
    assert rep_full["newton_rel_res"] <= 1e-7 and rep_res["newton_rel_res"] <= 1e-7
    assert np.array_equal(U_res, U_full)
    assert list(pcg_a) + list(pcg_b) == list(pcg_full)
    assert list(nwt_a) + list(nwt_b) == list(nwt_full)
    assert np.all(nwt_full >= 1)


def test_pressure_ramp_to_16_kpa_matches_oracle():
    from oracle import feti
    from paper_1508_02599_gb300 import FetiSolver
    prob = _tube(16.0)
    n = 40
    U_ref, _ = feti.monolithic_newton(prob, n, follower=True, tol=1e-9, maxit=40)
    with FetiSolver(prob, method="classical", precond="dirichlet", tol=1e-10, maxit=3000, n_load_steps=n,
                    newton_tol=1e-8, newton_maxit=40) as s:
        U, rep, pcg, nwt = s.newton_steps(1, n)
    assert rep["newton_rel_res"] <= 1e-8
    assert np.linalg.norm(U - U_ref) <= 1e-6 * np.linalg.norm(U_ref)
    # the wall inflates: mean inner radius well above 1 at 16 kPa
    x, u = prob.coords, U.reshape(-1, 3)
    inner = np.abs(np.hypot(x[:, 0], x[:, 1]) - 1.0) < 1e-12
    assert np.hypot(x[inner, 0] + u[inner, 0], x[inner, 1] + u[inner, 1]).mean() > 1.5


def test_long_load_stepping_classical_and_all_floating(tmp_path):
    from paper_1508_02599_gb300 import FetiSolver, checkpoint_read, checkpoint_write
    prob = _tube(16.0, material=mesh.hgo_material(c=6.0, kappa=1000.0))
    n, block = 200, 50
    counts = {}
    for method in ("classical", "af"):
        with FetiSolver(prob, method=method, precond="dirichlet", tol=1e-10, maxit=3000, n_load_steps=n,
                        newton_tol=1e-7, newton_maxit=30) as s:
            U = None
            pcg_all, nwt_all = [], []
            for first in range(1, n + 1, block):
                last = first + block - 1
                U, rep, pcg, nwt = s.newton_steps(first, last, U_start=U)
                assert rep["newton_rel_res"] <= 1e-7, (method, last)
                path = tmp_path / f"{method}.ckp"
                checkpoint_write(path, U, last, n, last / n)
                U, step, _, _ = checkpoint_read(path)
                assert step == last
                pcg_all += list(pcg)
                nwt_all += list(nwt)
        counts[method] = (np.array(pcg_all), np.array(nwt_all))
        assert len(pcg_all) == n and min(nwt_all) >= 1
    # same equilibrium path: both methods solve the same discrete problem
    print("PCG iterations per load step: classical mean %.1f, all-floating mean %.1f"
          % (counts["classical"][0].mean(), counts["af"][0].mean()))
