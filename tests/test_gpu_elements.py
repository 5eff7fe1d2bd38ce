"""GPU element kernels (linear and two-fibre hyperelastic) against the oracle, element by element.

Tolerance: 1e-10 relative to the element's largest entry.  Both sides are
FP64; the oracle's elasticity tensor is a complex-step derivative of its
stress formula, the kernel's is written out analytically, so agreement
beyond rounding pins the derivation.
"""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    return (np.abs(a - b).reshape(a.shape[0], -1).max(axis=1) / scale).max()


def test_linear_elements_match():
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(2, 16, 4, (1, 2, 1))
    Ke_ref, _ = fem.element_matrices(prob)
    with FetiSolver(prob) as s:
        Ke, _ = s.elements()
    assert _rel(Ke, Ke_ref) <= 1e-12


@pytest.mark.parametrize("amp", [0.0, 0.02, 0.08])
def test_hgo_elements_match(amp):
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(2, 16, 4, (1, 2, 1), material=mesh.hgo_material(), pressure=0.1)
    rng = np.random.default_rng(17)
    x = prob.coords
    # smooth inflation plus noise: both fibre families active in most elements,
    # compressed in some
    r = np.hypot(x[:, 0], x[:, 1])[:, None]
    U = amp * (np.concatenate([x[:, :2] / r, np.zeros((x.shape[0], 1))], axis=1) + 0.5 * rng.normal(size=x.shape))
    Ke_ref, fe_ref = fem.element_matrices(prob, U)
    with FetiSolver(prob, method="classical") as s:
        Ke, fe = s.elements(U)
    assert _rel(Ke, Ke_ref) <= 1e-10
    assert np.abs(Ke - Ke.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(Ke).max()
    if amp > 0:
        assert _rel(fe, fe_ref) <= 1e-10
    else:
        assert np.abs(fe).max() <= 1e-12 * np.abs(Ke).max()


def test_newton_matches_oracle_classical():
    """Load-stepped Newton (one step, 1 mmHg as in Tables 4-7) on the small tube.

    Classical FETI: every subdomain touches the Dirichlet boundary, so the
    local tangents are nonsingular and the FETI increment is the exact Newton
    increment; GPU and oracle both stop at a relative residual of 1e-9.
    """
    from oracle import feti
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(2, 16, 2, (1, 4, 1), material=mesh.hgo_material(), pressure=0.13332)
    U_ref, log = feti.newton_solve(prob, feti.CLASSICAL, "dirichlet", n_load_steps=1, newton_tol=1e-9,
                                   pcg_tol=1e-12)
    with FetiSolver(prob, method="classical", precond="dirichlet", tol=1e-12, maxit=3000, n_load_steps=1,
                    newton_tol=1e-9, newton_maxit=25) as s:
        U, rep = s.newton()
    assert rep["newton_rel_res"] <= 1e-9
    assert abs(rep["newton_iters"] - len(log[0])) <= 1
    assert np.linalg.norm(U - U_ref) <= 1e-7 * np.linalg.norm(U_ref)


@pytest.mark.slow
def test_full_size_hgo_elements_sampled():
    """The element kernel at the full size of the 24x96x48-cell tube (663,552
    tets, Table 1 material) at a smooth inflation plus noise: tangents and
    internal forces of 4096 sampled elements (seeded) against the oracle's
    complex-step route, and the global internal-force vector of all elements
    (assembled on the host from the GPU element forces) against the oracle's
    assembled forces on the same sample's nodes."""
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(24, 96, 48, (4, 16, 4), material=mesh.hgo_material(), pressure=0.13332)
    x = prob.coords
    r = np.hypot(x[:, 0], x[:, 1])[:, None]
    rng = np.random.default_rng(23)
    U = 0.03 * (np.concatenate([x[:, :2] / r, np.zeros((x.shape[0], 1))], axis=1)
                + 0.2 * rng.normal(size=x.shape) / 24.0)
    with FetiSolver(prob, method="af") as s:
        Ke, fe = s.elements(U)
    assert Ke.shape == (663552, 12, 12)
    pick = np.sort(rng.choice(prob.tets.shape[0], size=4096, replace=False))
    t = prob.tets[pick]
    f_ref, K_ref, detF = fem.hgo_element(prob.coords[t], U[t], prob.fibres[pick], prob.material)
    assert np.all(detF > 0.0)
    assert _rel(Ke[pick], K_ref) <= 1e-10
    assert _rel(fe[pick], f_ref) <= 1e-10
    assert np.abs(Ke - Ke.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(Ke).max()
    # every element: translation invariance of the internal force (sum over the
    # four nodes vanishes) and of the tangent (rows sum to zero per component)
    fs = fe.reshape(-1, 4, 3).sum(axis=1)
    assert np.abs(fs).max() <= 1e-10 * np.abs(fe).max()
    ks = Ke.reshape(-1, 12, 4, 3).sum(axis=2)
    assert np.abs(ks).max() <= 1e-9 * np.abs(Ke).max()


def _oracle_rel_residual(prob, U, chunk=32768):
    """||f_int(U) - f_ext(U)|| / ||f_ext(U)|| on the free DOFs, element forces
    from the oracle's own element route in chunks (bounded host memory)."""
    Ur = U.reshape(-1, 3)
    E = prob.tets.shape[0]
    fint = np.empty((E, 12))
    for s0 in range(0, E, chunk):
        t = prob.tets[s0:s0 + chunk]
        f, _, detF = fem.hgo_element(prob.coords[t], Ur[t], prob.fibres[s0:s0 + chunk], prob.material)
        assert np.all(detF > 0.0)
        fint[s0:s0 + chunk] = f
    fext = fem.load_vector(prob, Ur, True)
    R = fem.internal_force_global(prob, fint) - fext
    free = np.ones(U.size, bool)
    free[prob.dir_dof] = False
    return np.linalg.norm(R[free]) / np.linalg.norm(fext[free])


@pytest.mark.slow
def test_full_size_newton_256_subdomains():
    """The 24x96x48-cell tube (117,600 nodes, 663,552 tets, 256 subdomains)
    with the Table 1 material under follower pressure, 1 mmHg in four load
    steps, Newton with all-floating FETI to a relative residual of 1e-8.  The
    returned displacement is checked by the oracle's element route (its own
    stress formula and load vector), independently of the kernel's tangent,
    of the FETI increments and of the GPU residual."""
    from paper_1508_02599_gb300 import FetiSolver
    prob = mesh.cylinder_problem(24, 96, 48, (4, 16, 4), material=mesh.hgo_material(), pressure=0.13332)
    with FetiSolver(prob, method="af", precond="dirichlet", tol=1e-10, maxit=4000, n_load_steps=4,
                    newton_tol=1e-8, newton_maxit=25) as s:
        U, rep = s.newton()
    assert rep["newton_rel_res"] <= 1e-8
    assert np.linalg.norm(U) > 0.0
    assert _oracle_rel_residual(prob, U) <= 2e-8
