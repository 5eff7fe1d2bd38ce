"""Full-size parity with the FP64 oracle on the 64-subdomain tube and the 1024-subdomain jittered tube.

Expected values come from tests/golden/make_fullsize.py, which runs only the
oracle (oracle/feti.py: projected PCG of Sec. 4.3 with the Dirichlet, lumped
and identity preconditioners of Sec. 4.4) on the same seeded meshes:
  * PCG iteration counts at ||P r_k|| <= 1e-8 ||P r_0||: the FP64 GPU form must
    need the same count +-1 with the Dirichlet preconditioner, and within 2 %
    with the lumped and identity ones (runs of hundreds of iterations, where
    the different summation orders of GPU and oracle shift the count by a few:
    on the 64-subdomain tube 237 vs 235 and 527 vs 518);
  * the displacement at 4096 seeded sample nodes (and ||U||, max|U|) from the
    oracle's solve to 1e-12: every precision form and preconditioner, solved
    to 1e-11, must match max |U - U_ref| <= 1e-8 max |U_ref| over the sample,
    element by element, and ||U|| to 1e-8 relative.
"""
import os

import numpy as np
import pytest

from feti_inputs import mesh

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ["cyl16", "jcyl32"]
_PROBS = {}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _golden(name):
    its, cond, nodes, vals = {}, {}, [], []
    unorm = umax = None
    with open(os.path.join(HERE, "golden", f"fullsize_{name}.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0] == "iterations":
                its[t[1]] = int(t[2])
            elif t[0] == "cond":
                cond[t[1]] = float(t[2])
            elif t[0] == "unorm":
                unorm = float(t[1])
            elif t[0] == "umax":
                umax = float(t[1])
            elif t[0] == "u":
                nodes.append(int(t[1]))
                vals.append([float(x) for x in t[2:5]])
    return {"iterations": its, "cond": cond, "unorm": unorm, "umax": umax, "nodes": np.array(nodes),
            "u": np.array(vals)}


def _prob(name):
    if name not in _PROBS:
        _PROBS[name] = mesh.config_problem(name)
    return _PROBS[name]


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precond", ["dirichlet", "lumped", "identity"])
def test_fullsize_iterations_match_oracle(name, precond):
    from paper_1508_02599_gb300 import FetiSolver
    g = _golden(name)
    with FetiSolver(_prob(name), method="af", precond=precond, precision="fp64", tol=1e-8, maxit=5000) as s:
        _, rep = s.solve()
    assert rep["converged"] == 1
    ref = g["iterations"][precond]
    # +-1 for the Dirichlet preconditioner; the long lumped and identity runs
    # (hundreds of iterations) drift by rounding (GPU and oracle sum in
    # different orders, and CG's loss of orthogonality amplifies it): +-2 %
    slack = 1 if precond == "dirichlet" else max(1, int(0.02 * ref))
    assert abs(rep["iterations"] - ref) <= slack, (rep["iterations"], ref)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("precond", ["dirichlet", "lumped", "identity"])
@pytest.mark.parametrize("precision", ["fp64", "mixed", "mixed_f32factor"])
def test_fullsize_displacement_matches_oracle(name, precond, precision):
    from paper_1508_02599_gb300 import FetiSolver
    g = _golden(name)
    with FetiSolver(_prob(name), method="af", precond=precond, precision=precision, tol=1e-11,
                    maxit=5000) as s:
        U, rep = s.solve()
    assert rep["converged"] == 1
    u = U.reshape(-1, 3)[g["nodes"]]
    err = np.abs(u - g["u"]).max()
    assert err <= 1e-8 * g["umax"], (err / g["umax"], rep)
    assert abs(np.linalg.norm(U) - g["unorm"]) <= 1e-8 * g["unorm"]
