"""Kelvin-solution cube (Sec. 5.1): FE convergence and FETI with inhomogeneous Dirichlet data."""
import numpy as np

from feti_inputs import mesh
from oracle import fem, feti


def _l2(prob, U):
    """L2 norm of the error against Kelvin's solution (vertex quadrature per element)."""
    uex = mesh.kelvin_displacement(prob.coords, prob.material["E"], prob.material["nu"])
    e = U.reshape(-1, 3) - uex
    _, V = fem.shape_gradients(prob.coords[prob.tets])
    return np.sqrt((V * (e[prob.tets] ** 2).sum(axis=2).mean(axis=1)).sum())


def _monolithic(prob):
    Ke, _ = fem.element_matrices(prob)
    return fem.monolithic_solve(prob, fem.assemble_global(prob, Ke), fem.load_vector(prob))


def test_kelvin_solution_satisfies_navier_equations():
    """The closed form is divergence-free in the stress sense: a finite-difference
    check of div sigma = 0 away from the source point."""
    E, nu = 210.0, 0.45
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    x0 = np.array([[0.3, 0.6, 0.4]])
    h = 1e-3

    def grad(x):
        G = np.zeros((3, 3))
        for j in range(3):
            d = np.zeros(3)
            d[j] = h
            G[:, j] = (mesh.kelvin_displacement(x + d, E, nu)[0] - mesh.kelvin_displacement(x - d, E, nu)[0]) / (2 * h)
        return G

    def stress(x):
        G = grad(x)
        eps = 0.5 * (G + G.T)
        return lam * np.trace(eps) * np.eye(3) + 2 * mu * eps

    div = np.zeros(3)
    for j in range(3):
        d = np.zeros(3)
        d[j] = h
        div += (stress(x0 + d)[:, j] - stress(x0 - d)[:, j]) / (2 * h)
    assert np.abs(div).max() <= 1e-4 * np.abs(stress(x0)).max()


def test_p1_order_of_convergence_matches_table2():
    """eoc ~ 2 for P1 (Table 2 prints 1.94-1.99)."""
    errs = [_l2(p, _monolithic(p)) for p in (mesh.kelvin_cube_problem(n, (1, 1, 1)) for n in (4, 8, 16))]
    eoc = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(eoc > 1.8) and np.all(eoc < 2.1)


def test_feti_with_inhomogeneous_dirichlet_equals_monolithic():
    """Classical elimination of u_D (f_i - K_iD u_D) and all-floating b = u_D rows."""
    prob = mesh.kelvin_cube_problem(8, (4, 4, 4))
    u_ref = _monolithic(prob)
    for method in (feti.CLASSICAL, feti.ALL_FLOATING):
        o = feti.FetiOracle(prob, method, "dirichlet")
        U, res, us = o.solve(tol=1e-12)
        assert np.linalg.norm(U - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
        assert o.jump(us) <= 1e-9 * np.linalg.norm(u_ref)
