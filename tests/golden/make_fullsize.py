"""Writes the full-size expected values of the GPU parity tests from the FP64 oracle.

For the 64-subdomain tube (16 x 64 x 32 cells, wedge partition) and the
1024-subdomain jittered tube (32 x 128 x 64 cells, jittered recursive
bisection), all-floating FETI, this script runs the oracle (oracle/feti.py,
Sec. 4 of the paper: projected PCG on the dual problem with the Dirichlet,
lumped and identity preconditioners) and records

  * the PCG iteration count at relative tolerance 1e-8 for each preconditioner
    (first k with ||P r_k|| <= 1e-8 ||P r_0||, the stopping rule of the solver);
  * the Lanczos condition estimate of each run;
  * ||U||_2 and U at 4096 seeded sample nodes (numpy PCG64, seed 4096), from
    the Dirichlet-preconditioned solve continued to 1e-12.

It imports only oracle/ and feti_inputs/.  Usage (from the repository root):
    python tests/golden/make_fullsize.py cyl16 jcyl32
writes tests/golden/fullsize_<name>.txt.  The 1024-subdomain case needs about
30 GB of host memory and about an hour on eight cores.
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from feti_inputs import mesh  # noqa: E402
from oracle import feti  # noqa: E402

N_SAMPLE = 4096
SAMPLE_SEED = 4096
TOL_COUNT = 1e-8
TOL_U = 1e-12


def sample_nodes(n_nodes: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    return np.sort(rng.choice(n_nodes, size=min(N_SAMPLE, n_nodes), replace=False))


def count_at(res_hist, tol: float) -> int:
    """Iterations the stopping rule ||P r_k|| <= tol ||P r_0|| needs."""
    w0 = res_hist[0]
    for k, w in enumerate(res_hist):
        if w <= tol * w0:
            return k
    raise RuntimeError("tolerance not reached")


def run(name: str) -> str:
    prob = mesh.config_problem(name)
    lines = [f"# full-size oracle values: {prob.name}, all-floating FETI, {prob.n_parts} subdomains,",
             f"# {prob.n_nodes} nodes; written by tests/golden/make_fullsize.py (oracle/ only)",
             f"# iterations: PCG count at ||P r_k|| <= {TOL_COUNT:g} ||P r_0||; cond: Lanczos estimate",
             f"# U: Dirichlet-preconditioned solve to {TOL_U:g}; sample: {N_SAMPLE} nodes, PCG64 seed {SAMPLE_SEED}"]
    U = None
    for precond in ("dirichlet", "lumped", "identity"):
        t0 = time.perf_counter()
        o = feti.FetiOracle(prob, feti.ALL_FLOATING, precond)
        o.assemble()
        # factorize one subdomain at a time and drop its dense K_i at once
        # (the oracle's own factorization of each subdomain, then its coarse
        # problem over all of them): the 1024-subdomain tube fits in host memory
        subs = o.subs
        for sd in subs:
            o.subs = [sd]
            o.factorize()
            sd.K = None
        o.subs = subs
        o._coarse()
        tol = TOL_U if precond == "dirichlet" else TOL_COUNT
        res = o.pcg(tol, 5000)
        assert res.converged, precond
        its = count_at(res.res_hist, TOL_COUNT)
        lines.append(f"iterations {precond} {its}")
        lines.append(f"cond {precond} {res.cond_est:.6f}")
        if precond == "dirichlet":
            us, _ = o.recover(res.lam)
            U = o.global_displacement(us)
        print(f"{name} {precond}: {its} iterations at {TOL_COUNT:g} ({res.iterations} to {tol:g}), "
              f"{time.perf_counter() - t0:.0f} s", flush=True)
        del o
    lines.append(f"unorm {np.linalg.norm(U):.17e}")
    lines.append(f"umax {np.abs(U).max():.17e}")
    u = U.reshape(-1, 3)
    for n in sample_nodes(prob.n_nodes):
        lines.append(f"u {n} {u[n, 0]:.17e} {u[n, 1]:.17e} {u[n, 2]:.17e}")
    return "\n".join(lines) + "\n"


if __name__ == "__main__":
    for name in sys.argv[1:] or ["cyl16", "jcyl32"]:
        text = run(name)
        with open(os.path.join(HERE, f"fullsize_{name}.txt"), "w") as f:
            f.write(text)
