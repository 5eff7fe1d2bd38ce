"""FP64 finite-element building blocks of the oracle (P1 and P2-P0 tetrahedra).

Follows Sec. 3 (kinematics, Eq. for F, C, J and the Flory split; the energy of
Eq. (isoaniso) with the volumetric penalty, neo-Hooke matrix and the two
exponential fibre families of Eqs. (aniso_1)-(aniso_2), active only in
tension) and Sec. 3.2 (Newton linearisation, tangent Eq. (Tangent), the
global matrices K'[i,j], residual K(U) and load vector).

Readings where the paper is silent:
* the elasticity tensor is not printed (Sec. 3.2 defers it); here it is the
  exact derivative 2 dS/dC of the stress formula, taken by complex-step
  differentiation, so it needs no hand derivation;
* a fibre family is active iff I4bar - 1 > 1e-12 (the paper's strict
  inequality, with the rounding of I4bar = 1 at zero strain kept inactive);
* for P1 tetrahedra F and J are constant per element, so the statically
  condensed P1-P0 element equals the pure displacement element with
  Psi_vol(J) (Sec. 3.2, static condensation);
* surface loads are P1-consistent: each vertex of a loaded triangle receives a
  third of (traction x area); a pressure acts along the area vector of the
  triangle that points into the solid, on the current geometry when the load
  follows the deformation (Sec. 3.2, last paragraph: load stiffness dropped).

Pins (tests/test_oracle_fem.py): linear patch test (exact affine fields),
Hooke stiffness against the classical 6x6 Voigt route, stress against a finite
difference of the energy, tangent against a finite difference of the internal
force, tangent at zero strain against Hooke with mu = c, lambda = kappa-2c/3.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

LINEAR_ISO = 0
HGO_TWO_FIBRE = 1
LINEAR_ISO_P0 = 2   # Hooke's law with the volumetric part condensed to a piecewise-constant pressure
FIBRE_ACTIVE_EPS = 1e-12

# Derivatives of the P1 shape functions w.r.t. barycentric reference coords.
_DN_DXI = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])


def shape_gradients(X: np.ndarray):
    """Gradients of the four P1 shape functions and the volume, per element.

    X: [E, 4, 3] vertex coordinates.  Returns g [E, 4, 3] (dN_a/dX) and V [E].
    """
    Jm = np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], axis=2)  # columns
    V = np.linalg.det(Jm) / 6.0
    g = np.einsum("ak,ekj->eaj", _DN_DXI, np.linalg.inv(Jm))
    return g, V


def linear_element(X: np.ndarray, E: float, nu: float) -> np.ndarray:
    """Isotropic Hooke element matrices K_e[E, 12, 12] (dof = 3*vertex + comp).

    K[a i, b j] = V (lam g_a,i g_b,j + mu (delta_ij g_a.g_b + g_a,j g_b,i)).
    """
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    g, V = shape_gradients(X)
    I3 = np.eye(3)
    gg = np.einsum("eak,ebk->eab", g, g)
    K = (lam * np.einsum("eai,ebj->eaibj", g, g)
         + mu * np.einsum("ij,eab->eaibj", I3, gg)
         + mu * np.einsum("eaj,ebi->eaibj", g, g))
    K *= V[:, None, None, None, None]
    return K.reshape(-1, 12, 12)


# P2-P0 tetrahedra (Sec. 3.2, static condensation; Sec. 5.1, Table 3).
# Ten nodes: the vertices, then the midpoints of the edges (0,1), (0,2), (0,3),
# (1,2), (1,3), (2,3).  In barycentric coordinates L_0..L_3 the shape
# functions are N_a = L_a (2 L_a - 1) at a vertex and N_ab = 4 L_a L_b at the
# midpoint of edge (a, b).
P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
# Degree-2 Gauss rule on the tetrahedron: the four points with barycentric
# coordinates (alpha, beta, beta, beta) and permutations, equal weights 1/4
# (alpha = (5 + 3 sqrt 5) / 20, beta = (5 - sqrt 5) / 20).
_Q2_ALPHA = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
_Q2_BETA = (5.0 - np.sqrt(5.0)) / 20.0
Q2_POINTS = np.array([[_Q2_ALPHA if j == i else _Q2_BETA for j in range(4)] for i in range(4)])
Q2_WEIGHTS = np.full(4, 0.25)


def p2_shape_values(Lq: np.ndarray) -> np.ndarray:
    """P2 shape function values [Q, 10] at barycentric points Lq [Q, 4]."""
    N = np.empty((Lq.shape[0], 10))
    for a in range(4):
        N[:, a] = Lq[:, a] * (2.0 * Lq[:, a] - 1.0)
    for e, (a, b) in enumerate(P2_EDGES):
        N[:, 4 + e] = 4.0 * Lq[:, a] * Lq[:, b]
    return N


def p2_shape_gradients(X: np.ndarray, Lq: np.ndarray = Q2_POINTS):
    """Gradients [E, Q, 10, 3] of the P2 shape functions at the barycentric
    points Lq and the volume [E] (straight-sided tetrahedra: X [E, >=4, 3],
    the vertices first).  grad N_a = (4 L_a - 1) grad L_a,
    grad N_ab = 4 (L_a grad L_b + L_b grad L_a)."""
    gL, V = shape_gradients(X[:, :4])           # gradients of the barycentric coordinates
    Q = Lq.shape[0]
    g = np.empty((X.shape[0], Q, 10, 3))
    for a in range(4):
        g[:, :, a, :] = (4.0 * Lq[None, :, a, None] - 1.0) * gL[:, None, a, :]
    for e, (a, b) in enumerate(P2_EDGES):
        g[:, :, 4 + e, :] = 4.0 * (Lq[None, :, a, None] * gL[:, None, b, :] + Lq[None, :, b, None] * gL[:, None, a, :])
    return g, V


def linear_p2_element(X: np.ndarray, E: float, nu: float, p0: bool = False) -> np.ndarray:
    """P2 element matrices K_e [E, 30, 30] (dof = 3 * node + comp) for Hooke's law.

    p0 = False: the displacement element of the linear cube study (Table 3),
    K[a i, b j] = int lambda g_a,i g_b,j + mu (delta_ij g_a . g_b + g_a,j g_b,i).
    p0 = True: P2-P0, the volumetric part carried by a piecewise-constant
    pressure p and condensed out element by element (Sec. 3.2, static
    condensation): with int q (div u - p / lambda) = 0, p = lambda (int div u) / V,
    so the lambda term becomes lambda V bbar_a,i bbar_b,j, bbar_a = (int g_a) / V.
    The integrands are of degree 2 in the coordinates, exact with the degree-2
    Gauss rule.
    """
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    g, V = p2_shape_gradients(X)
    w = Q2_WEIGHTS
    gg = np.einsum("q,eqak,eqbk->eab", w, g, g)
    K = mu * (np.einsum("ij,eab->eaibj", np.eye(3), gg) + np.einsum("q,eqaj,eqbi->eaibj", w, g, g))
    if p0:
        bbar = np.einsum("q,eqai->eai", w, g)
        K = K + lam * np.einsum("eai,ebj->eaibj", bbar, bbar)
    else:
        K = K + lam * np.einsum("q,eqai,eqbj->eaibj", w, g, g)
    return (K * V[:, None, None, None, None]).reshape(-1, 30, 30)


def hgo_energy(C: np.ndarray, a1: np.ndarray, a2: np.ndarray, mat: dict) -> np.ndarray:
    """Strain energy Psi(C) per element (Eq. isoaniso with its three terms)."""
    c, k1, k2, kappa = mat["c"], mat["k1"], mat["k2"], mat["kappa"]
    J = np.sqrt(np.linalg.det(C))
    J23 = J ** (-2.0 / 3.0)
    I1b = J23 * np.einsum("eii->e", C)
    psi = 0.5 * kappa * (J - 1.0) ** 2 + 0.5 * c * (I1b - 3.0)
    for a in (a1, a2):
        I4b = J23 * np.einsum("ei,eij,ej->e", a, C, a)
        act = np.real(I4b) - 1.0 > FIBRE_ACTIVE_EPS
        psi = psi + np.where(act, k1 / (2.0 * k2) * (np.exp(k2 * (I4b - 1.0) ** 2) - 1.0), 0.0)
    return psi


def hgo_stress(C: np.ndarray, a1: np.ndarray, a2: np.ndarray, mat: dict) -> np.ndarray:
    """Second Piola-Kirchhoff stress S = 2 dPsi/dC (works for complex C too).

    S = kappa (J-1) J C^-1 + c J^-2/3 (I - I1/3 C^-1)
        + sum_f 2 psi_f' J^-2/3 (a (x) a - I4/3 C^-1),
    psi_f' = k1 (I4bar-1) exp(k2 (I4bar-1)^2) for an active family, else 0.
    """
    c, k1, k2, kappa = mat["c"], mat["k1"], mat["k2"], mat["kappa"]
    Ci = np.linalg.inv(C)
    J = np.sqrt(np.linalg.det(C))
    J23 = J ** (-2.0 / 3.0)
    I1 = np.einsum("eii->e", C)
    I3 = np.eye(3)[None]
    S = (kappa * (J - 1.0) * J)[:, None, None] * Ci
    S = S + (c * J23)[:, None, None] * (I3 - (I1 / 3.0)[:, None, None] * Ci)
    for a in (a1, a2):
        I4 = np.einsum("ei,eij,ej->e", a, C, a)
        I4b = J23 * I4
        act = np.real(I4b) - 1.0 > FIBRE_ACTIVE_EPS
        dpsi = np.where(act, k1 * (I4b - 1.0) * np.exp(k2 * (I4b - 1.0) ** 2), 0.0)
        aa = np.einsum("ei,ej->eij", a, a)
        S = S + (2.0 * dpsi * J23)[:, None, None] * (aa - (I4 / 3.0)[:, None, None] * Ci)
    return S


def hgo_elasticity(C: np.ndarray, a1: np.ndarray, a2: np.ndarray, mat: dict) -> np.ndarray:
    """Material elasticity tensor CC[E,3,3,3,3] = 2 dS/dC by complex step.

    For a symmetric direction D, dS[D] = Im S(C + i h D) / h exactly up to
    rounding; CC_IJKK = 2 dS[E_KK]_IJ and CC_IJKL = dS[E_KL + E_LK]_IJ (K != L).
    """
    h = 1e-40
    CC = np.zeros(C.shape[:1] + (3, 3, 3, 3))
    Cc = C.astype(np.complex128)
    for K in range(3):
        for L in range(K, 3):
            D = np.zeros((3, 3))
            D[K, L] += 1.0
            D[L, K] += 1.0
            dS = np.imag(hgo_stress(Cc + 1j * h * D[None], a1, a2, mat)) / h
            if K == L:
                CC[:, :, :, K, K] = dS  # D = 2 E_KK, so dS = CC_IJKK
            else:
                CC[:, :, :, K, L] = dS
                CC[:, :, :, L, K] = dS
    return CC


def hgo_element(X: np.ndarray, U: np.ndarray, fib: np.ndarray, mat: dict):
    """Internal force f_e[E,12] and tangent K_e[E,12,12] of Eq. (Tangent).

    F = I + sum_a u_a (x) g_a;  f[a i] = V (F S g_a)_i;
    K[a i, b j] = V (delta_ij g_a.S g_b + F_iI g_a,J CC_IJKL F_jK g_b,L).
    """
    g, V = shape_gradients(X)
    F = np.eye(3)[None] + np.einsum("eai,eaJ->eiJ", U, g)
    C = np.einsum("eiI,eiJ->eIJ", F, F)
    a1, a2 = fib[:, 0:3], fib[:, 3:6]
    S = hgo_stress(C, a1, a2, mat)
    CC = hgo_elasticity(C, a1, a2, mat)
    f = np.einsum("e,eiI,eIJ,eaJ->eai", V, F, S, g).reshape(-1, 12)
    geo = np.einsum("eaI,eIJ,ebJ->eab", g, S, g)
    Kg = np.einsum("eab,ij->eaibj", geo, np.eye(3))
    Km = np.einsum("eiI,eaJ,eIJKL,ejK,ebL->eaibj", F, g, CC, F, g)
    K = (Kg + Km) * V[:, None, None, None, None]
    return f, K.reshape(-1, 12, 12), np.linalg.det(F)


def element_matrices(prob, U: np.ndarray | None = None):
    """Element tangents (and internal forces for the hyperelastic model).

    Returns (K_e [E,12,12], f_int [E,12] or None).
    """
    X = prob.coords[prob.tets]
    mat = prob.material
    if prob.tets.shape[1] == 10:
        if mat["kind"] not in (LINEAR_ISO, LINEAR_ISO_P0):
            raise NotImplementedError("P2 elements are built for the linear material")
        return linear_p2_element(X, mat["E"], mat["nu"], p0=mat["kind"] == LINEAR_ISO_P0), None
    if mat["kind"] in (LINEAR_ISO, LINEAR_ISO_P0):   # on P1 the element mean of div u is div u itself
        return linear_element(X, mat["E"], mat["nu"]), None
    if U is None:
        U = np.zeros_like(prob.coords)
    f, K, detF = hgo_element(X, U[prob.tets], prob.fibres, mat)
    if np.any(detF <= 0.0):
        raise FloatingPointError("inverted element: det F <= 0")
    return K, f


def surface_loads(prob, U: np.ndarray | None = None, follower: bool = True):
    """Consistent nodal loads per loaded triangle.

    Returns (owner tet [T], nodes [T,3] or [T,6], force per node [T,3] or
    [T,6,3]) for the pressure and traction triangles together.  P1 (3-node)
    triangles: a third of the force to each vertex.  P2 (6-node, flat)
    triangles under a constant load: int N = 0 at the vertices and A/3 at the
    edge midpoints.
    """
    if prob.trac_tri.shape[1:] == (6,) or prob.press_tri.shape[1:] == (6,):
        owners, nodes, forces = [], [], []
        if prob.press_tri.shape[0]:
            if U is not None and follower:
                raise NotImplementedError("follower pressure on P2 faces")
            x = prob.coords
            t = prob.press_tri
            av = 0.5 * np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]])
            f = np.zeros((t.shape[0], 6, 3))
            f[:, 3:, :] = (prob.pressure * av / 3.0)[:, None, :]
            owners.append(prob.press_owner)
            nodes.append(t)
            forces.append(f)
        if prob.trac_tri.shape[0]:
            x = prob.coords
            t = prob.trac_tri
            area = 0.5 * np.linalg.norm(np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]]), axis=1)
            f = np.zeros((t.shape[0], 6, 3))
            f[:, 3:, :] = (area[:, None] * prob.traction[None, :] / 3.0)[:, None, :]
            owners.append(prob.trac_owner)
            nodes.append(t)
            forces.append(f)
        if not owners:
            return np.zeros(0, np.int64), np.zeros((0, 6), np.int64), np.zeros((0, 6, 3))
        return np.concatenate(owners), np.concatenate(nodes), np.concatenate(forces)
    owners, verts, forces = [], [], []
    if prob.press_tri.shape[0]:
        x = prob.coords.copy()
        if U is not None and follower:
            x = x + U
        t = prob.press_tri
        area_vec = 0.5 * np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]])
        owners.append(prob.press_owner)
        verts.append(t)
        forces.append(prob.pressure * area_vec / 3.0)
    if prob.trac_tri.shape[0]:
        x = prob.coords
        t = prob.trac_tri
        area = 0.5 * np.linalg.norm(np.cross(x[t[:, 1]] - x[t[:, 0]], x[t[:, 2]] - x[t[:, 0]]), axis=1)
        owners.append(prob.trac_owner)
        verts.append(t)
        forces.append(area[:, None] * prob.traction[None, :] / 3.0)
    if not owners:
        return np.zeros(0, np.int64), np.zeros((0, 3), np.int64), np.zeros((0, 3))
    return np.concatenate(owners), np.concatenate(verts), np.concatenate(forces)


def assemble_global(prob, Ke: np.ndarray) -> sp.csr_matrix:
    """Global stiffness K'[i,j] (Sec. 3.2) as a sparse matrix on all 3N DOFs."""
    nd = 3 * prob.tets.shape[1]
    dofs = (3 * prob.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, nd)
    rows = np.repeat(dofs, nd, axis=1).ravel()
    cols = np.tile(dofs, (1, nd)).ravel()
    n = 3 * prob.n_nodes
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def load_vector(prob, U=None, follower=True) -> np.ndarray:
    """Global external load vector on all 3N DOFs."""
    _, verts, forces = surface_loads(prob, U, follower)
    f = np.zeros(3 * prob.n_nodes)
    if verts.shape[1:] == (6,):
        for v in range(6):
            np.add.at(f, (3 * verts[:, v][:, None] + np.arange(3)[None, :]).ravel(), forces[:, v, :].ravel())
        return f
    for v in range(3):
        np.add.at(f, (3 * verts[:, v][:, None] + np.arange(3)[None, :]).ravel(), forces.ravel())
    return f


def internal_force_global(prob, f_int: np.ndarray) -> np.ndarray:
    dofs = (3 * prob.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(-1)
    out = np.zeros(3 * prob.n_nodes)
    np.add.at(out, dofs, f_int.ravel())
    return out


def monolithic_solve(prob, K: sp.csr_matrix, f: np.ndarray) -> np.ndarray:
    """Direct solve of the assembled system with Dirichlet DOFs eliminated.

    u_D = prescribed values; K_FF u_F = f_F - K_FD u_D by sparse LU.
    """
    n = K.shape[0]
    is_d = np.zeros(n, dtype=bool)
    is_d[prob.dir_dof] = True
    u = np.zeros(n)
    u[prob.dir_dof] = prob.dir_val
    free = np.nonzero(~is_d)[0]
    Kff = K[free][:, free].tocsc()
    rhs = f[free] - K[free][:, np.nonzero(is_d)[0]] @ u[is_d]
    u[free] = spla.spsolve(Kff, rhs)
    return u
