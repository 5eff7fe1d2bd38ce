"""Pins of the oracle's P2 and P2-P0 tetrahedra (Sec. 3.2 static condensation; Sec. 5.1, Table 3).

The 10-node elements -- the displacement element and the one with a
piecewise-constant pressure condensed out -- are checked against what does
not depend on their code path:
  * shape functions: nodal interpolation (Kronecker delta at the ten nodes),
    partition of unity, gradients summing to zero;
  * element matrix: symmetric, the six rigid-body modes in its kernel and
    nothing else (rank 24), equal to the Schur complement of the mixed
    displacement-pressure element assembled with another quadrature rule;
  * energy of an affine displacement: V (2 mu eps:eps + lambda (tr eps)^2);
  * patch test: a quadratic, divergence-free equilibrium field (no body
    force) is reproduced exactly by P2-P0, which P1 cannot;
  * Kelvin's solution on the unit cube: L2 error order 3 for the displacement
    P2 element of Table 3 (eoc 2.97-3.01; tests/golden/table3_cube_p2.txt),
    order 2 for P2-P0 at nu = 0.45, and no locking of P2-P0 at nu = 0.4999
    where P1 locks;
  * FETI on P2-P0 (classical and all-floating) equals the monolithic solve.
"""
import os

import numpy as np
import pytest

from feti_inputs import mesh
from oracle import fem, feti

HERE = os.path.dirname(os.path.abspath(__file__))


def _random_tets(n=5, seed=2):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 4, 3))
    _, V = fem.shape_gradients(X)
    X[V < 0] = X[V < 0][:, [0, 2, 1, 3]]
    X10 = np.concatenate([X, np.stack([0.5 * (X[:, a] + X[:, b]) for a, b in fem.P2_EDGES], axis=1)], axis=1)
    return X10


def _collapsed_rule(n=4):
    """Conical-product rule on the unit tetrahedron from Gauss-Legendre points
    on [0,1]^3 (x = u, y = v (1-u), z = w (1-u)(1-v)); returns barycentric
    points [Q, 4] and weights [Q] summing to 1."""
    t, w = np.polynomial.legendre.leggauss(n)
    t, w = 0.5 * (t + 1.0), 0.5 * w
    U, Vv, W = np.meshgrid(t, t, t, indexing="ij")
    WU, WV, WW = np.meshgrid(w, w, w, indexing="ij")
    x, y, z = U, Vv * (1 - U), W * (1 - U) * (1 - Vv)
    wt = WU * WV * WW * (1 - U) ** 2 * (1 - Vv) * 6.0
    L = np.stack([1 - x - y - z, x, y, z], axis=-1).reshape(-1, 4)
    return L, wt.ravel()


def test_shape_functions_interpolate_and_sum_to_one():
    nodesL = np.vstack([np.eye(4)] + [0.5 * (np.eye(4)[a] + np.eye(4)[b]) for a, b in fem.P2_EDGES])
    N = fem.p2_shape_values(nodesL)
    assert np.allclose(N, np.eye(10), atol=1e-15)
    L, _ = _collapsed_rule(3)
    assert np.allclose(fem.p2_shape_values(L).sum(axis=1), 1.0, atol=1e-14)
    g, _ = fem.p2_shape_gradients(_random_tets(), L)
    assert np.abs(g.sum(axis=2)).max() <= 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("p0", [False, True])
def test_element_kernel_rank_and_symmetry(p0):
    X = _random_tets()
    K = fem.linear_p2_element(X, 3.0, 0.45, p0=p0)
    assert np.abs(K - K.transpose(0, 2, 1)).max() <= 1e-13 * np.abs(K).max()
    for e in range(X.shape[0]):
        R = feti.rigid_body_modes(X[e])
        assert np.abs(K[e] @ R).max() <= 1e-12 * np.abs(K[e]).max() * np.abs(R).max()
        ev = np.linalg.eigvalsh(K[e])
        assert np.sum(ev > 1e-10 * ev.max()) == 24


def test_element_is_schur_complement_of_mixed_element():
    """Mixed element [[A, B^T], [B, -V/lambda]] (displacement, P0 pressure),
    integrated with a 64-point conical-product rule, condensed by eliminating p."""
    E, nu = 3.0, 0.49
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    X = _random_tets()
    L, w = _collapsed_rule(4)
    g, V = fem.p2_shape_gradients(X, L)
    for e in range(X.shape[0]):
        A = np.zeros((30, 30))
        B = np.zeros(30)
        for q in range(L.shape[0]):
            Bq = np.zeros((6, 30))                 # Voigt strain rows xx yy zz yz xz xy
            for a in range(10):
                gx, gy, gz = g[e, q, a]
                Bq[0, 3 * a], Bq[1, 3 * a + 1], Bq[2, 3 * a + 2] = gx, gy, gz
                Bq[3, 3 * a + 1], Bq[3, 3 * a + 2] = gz, gy
                Bq[4, 3 * a], Bq[4, 3 * a + 2] = gz, gx
                Bq[5, 3 * a], Bq[5, 3 * a + 1] = gy, gx
            D = mu * np.diag([2, 2, 2, 1, 1, 1.0])   # 2 mu eps : eps in Voigt form
            A += w[q] * V[e] * Bq.T @ D @ Bq
            B += w[q] * V[e] * Bq[:3].sum(axis=0)     # int div N
        M = np.block([[A, B[:, None]], [B[None, :], np.array([[-V[e] / lam]])]])
        S = M[:30, :30] - np.outer(M[:30, 30], M[30, :30]) / M[30, 30]
        K = fem.linear_p2_element(X[e:e + 1], E, nu, p0=True)[0]
        assert np.abs(S - K).max() <= 1e-11 * np.abs(K).max()


def test_affine_field_energy():
    E, nu = 2.0, 0.3
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    X = _random_tets()
    rng = np.random.default_rng(9)
    G = rng.normal(size=(3, 3))
    eps = 0.5 * (G + G.T)
    _, V = fem.shape_gradients(X[:, :4])
    for p0 in (False, True):
        K = fem.linear_p2_element(X, E, nu, p0=p0)
        for e in range(X.shape[0]):
            u = (X[e] @ G.T).ravel()
            expect = V[e] * (2 * mu * np.sum(eps * eps) + lam * np.trace(eps) ** 2)
            assert np.isclose(u @ K[e] @ u, expect, rtol=1e-12)


def _monolithic(prob):
    Ke, _ = fem.element_matrices(prob)
    return fem.monolithic_solve(prob, fem.assemble_global(prob, Ke), fem.load_vector(prob))


def test_quadratic_patch_test():
    """u = s (x^2 - y^2, -2 x y, 0) + affine part: div u = const, Navier's
    equations hold without body force, Dirichlet data on the whole boundary
    of a jittered cube mesh; P2-P0 reproduces it at every node, P1 does not."""
    def field(x):
        u = np.stack([x[:, 0] ** 2 - x[:, 1] ** 2, -2 * x[:, 0] * x[:, 1], np.zeros(len(x))], axis=1)
        return 1e-2 * u + x @ np.array([[1e-3, 2e-3, 0.0], [0.0, -1e-3, 5e-4], [0.0, 0.0, 2e-3]]).T

    def with_data(prob):
        x = prob.coords
        on_b = np.any((x < 1e-12) | (x > 1 - 1e-12), axis=1)
        bn = np.nonzero(on_b)[0]
        dof = (3 * bn[:, None] + np.arange(3)).ravel()
        order = np.argsort(dof)
        prob.dir_dof = dof[order].astype(np.int32)
        prob.dir_val = field(x)[bn].ravel()[order]
        prob.trac_tri = prob.trac_tri[:0]
        prob.trac_owner = prob.trac_owner[:0]
        return prob

    def jittered():
        # interior vertices moved by up to 0.1 cell (uniform meshes make P1
        # exact at the nodes for harmonic quadratics; a jittered one does not)
        prob = mesh.cube_problem(4, (1, 1, 1), E=5.0, nu=0.4)
        x = prob.coords
        inner = np.all((x > 1e-12) & (x < 1 - 1e-12), axis=1)
        rng = np.random.default_rng(11)
        x[inner] += rng.uniform(-0.025, 0.025, size=(int(inner.sum()), 3))
        return prob

    p1 = with_data(jittered())
    err1 = np.abs(_monolithic(p1) - field(p1.coords).ravel()).max()
    assert err1 >= 1e-5 * np.abs(field(p1.coords)).max()
    for p0 in (False, True):
        p2 = with_data(mesh.p2_problem(jittered()))
        p2.material = mesh.linear_material(5.0, 0.4, p0=p0)
        err2 = np.abs(_monolithic(p2) - field(p2.coords).ravel()).max()
        assert err2 <= 1e-12 * np.abs(field(p2.coords)).max(), p0


def _l2_error(prob, U):
    L, w = _collapsed_rule(4)
    X = prob.coords[prob.tets]
    _, V = fem.shape_gradients(X[:, :4])
    N = fem.p2_shape_values(L)                          # [Q, 10]
    xq = np.einsum("qa,eai->eqi", N, X)
    uh = np.einsum("qa,eai->eqi", N, U.reshape(-1, 3)[prob.tets])
    ue = mesh.kelvin_displacement(xq.reshape(-1, 3), prob.material["E"], prob.material["nu"]).reshape(uh.shape)
    return np.sqrt(np.einsum("e,q,eqi->", V, w, (uh - ue) ** 2))


def _golden_eoc():
    for line in open(os.path.join(HERE, "golden", "table3_cube_p2.txt")):
        if line.startswith("eoc"):
            return [float(v) for v in line.split()[1:]]
    raise KeyError("eoc")


def test_p2_order_of_convergence_matches_table3():
    """Displacement P2 (Table 3's element): L2 error order 3."""
    errs = [_l2_error(p, _monolithic(p)) for p in (mesh.kelvin_cube_problem_p2(n, (1, 1, 1)) for n in (2, 4, 8))]
    eoc = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    paper = _golden_eoc()
    assert min(paper) >= 2.9 and max(paper) <= 3.1
    assert np.all(eoc > 2.8) and np.all(eoc < 3.2), eoc


def test_p2p0_is_locking_free():
    """P2-P0 (volumetric part condensed to P0): L2 order 2 at nu = 0.45 (the
    piecewise-constant pressure limits it); towards incompressibility
    (nu = 0.45 -> 0.4999) its error stays nearly constant (the P2-P0 pair is
    inf-sup stable, so the bound does not depend on lambda), while the
    displacement P2 element's error grows several-fold (volumetric locking)."""
    def kelvin(n, nu, p0):
        p = mesh.kelvin_cube_problem_p2(n, (1, 1, 1), nu=nu)
        p.material = mesh.linear_material(p.material["E"], nu, p0=p0)
        return p
    errs = [_l2_error(p, _monolithic(p)) for p in (kelvin(n, 0.45, True) for n in (2, 4, 8))]
    eoc = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(eoc > 1.7) and np.all(eoc < 2.4), eoc
    grow = {}
    for p0 in (True, False):
        e = [_l2_error(p, _monolithic(p)) for p in (kelvin(4, nu, p0) for nu in (0.45, 0.4999))]
        grow[p0] = e[1] / e[0]
    assert grow[True] <= 1.7 and grow[False] >= 3.0, grow


def _l1_error(prob, U):
    """L2 error of a P1 solution (conical-product rule, P1 interpolation)."""
    L, w = _collapsed_rule(4)
    X = prob.coords[prob.tets]
    _, V = fem.shape_gradients(X)
    xq = np.einsum("qa,eai->eqi", L, X)
    uh = np.einsum("qa,eai->eqi", L, U.reshape(-1, 3)[prob.tets])
    ue = mesh.kelvin_displacement(xq.reshape(-1, 3), prob.material["E"], prob.material["nu"]).reshape(uh.shape)
    return np.sqrt(np.einsum("e,q,eqi->", V, w, (uh - ue) ** 2))


@pytest.mark.parametrize("method", [feti.CLASSICAL, feti.ALL_FLOATING])
def test_feti_p2_equals_monolithic(method):
    prob = mesh.kelvin_cube_problem_p2(4, (2, 2, 2))
    u_ref = _monolithic(prob)
    o = feti.FetiOracle(prob, method, "dirichlet")
    U, res, us = o.solve(tol=1e-12)
    assert res.converged
    assert np.linalg.norm(U - u_ref) <= 1e-9 * np.linalg.norm(u_ref)
    assert o.jump(us) <= 1e-9 * np.linalg.norm(u_ref)
