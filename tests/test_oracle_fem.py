"""Pins of the oracle's element level against closed forms and independent routes."""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import fem

RNG = np.random.default_rng(7)


def _random_tets(n):
    X = RNG.normal(size=(n, 4, 3))
    vol = np.einsum("ij,ij->i", np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), X[:, 3] - X[:, 0])
    X[vol < 0, 2], X[vol < 0, 3] = X[vol < 0, 3].copy(), X[vol < 0, 2].copy()
    return X


def test_shape_gradients_partition_of_unity_and_volume():
    X = _random_tets(20)
    g, V = fem.shape_gradients(X)
    # sum_a grad N_a = 0 and sum_a X_a (x) grad N_a = I (P1 reproduces affine fields)
    assert np.abs(g.sum(axis=1)).max() < 1e-12
    ident = np.einsum("eai,eaj->eij", X, g)
    assert np.abs(ident - np.eye(3)).max() < 1e-11
    vol = np.abs(np.linalg.det(np.stack([X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 3] - X[:, 0]], 1))) / 6
    assert np.allclose(V, vol, rtol=1e-13)


def _voigt_stiffness(X, E, nu):
    """Textbook route: K = V B^T D B with engineering shear strains."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g, V = fem.shape_gradients(X)
    out = np.zeros((X.shape[0], 12, 12))
    for e in range(X.shape[0]):
        B = np.zeros((6, 12))
        for a in range(4):
            gx, gy, gz = g[e, a]
            c = 3 * a
            B[0, c] = gx
            B[1, c + 1] = gy
            B[2, c + 2] = gz
            B[3, c], B[3, c + 1] = gy, gx      # gamma_xy
            B[4, c + 1], B[4, c + 2] = gz, gy  # gamma_yz
            B[5, c], B[5, c + 2] = gz, gx      # gamma_xz
        out[e] = V[e] * B.T @ D @ B
    return out


def test_linear_element_matches_voigt_route():
    X = _random_tets(10)
    K = fem.linear_element(X, 2.7, 0.31)
    Kv = _voigt_stiffness(X, 2.7, 0.31)
    assert np.abs(K - Kv).max() <= 1e-12 * np.abs(Kv).max()


def test_linear_patch_energy_and_rigid_modes():
    X = _random_tets(5)
    E, nu = 1.3, 0.27
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    K = fem.linear_element(X, E, nu)
    _, V = fem.shape_gradients(X)
    A = RNG.normal(size=(3, 3))
    eps = 0.5 * (A + A.T)
    u = np.einsum("ij,eaj->eai", A, X).reshape(-1, 12)
    energy = 0.5 * np.einsum("ei,eij,ej->e", u, K, u)
    exact = 0.5 * V * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert np.allclose(energy, exact, rtol=1e-12)
    W = 0.5 * (A - A.T)  # infinitesimal rotation: zero force
    ur = (np.einsum("ij,eaj->eai", W, X) + RNG.normal(size=3)).reshape(-1, 12)
    f = np.einsum("eij,ej->ei", K, ur)
    assert np.abs(f).max() < 1e-12 * np.abs(K).max() * np.abs(ur).max()


def test_linear_patch_test_on_cube_mesh():
    """Affine displacement: internal nodes feel zero net force (exact for P1)."""
    prob = mesh.cube_problem(4, (1, 1, 1), E=1.0, nu=0.3)
    Ke, _ = fem.element_matrices(prob)
    K = fem.assemble_global(prob, Ke)
    A = RNG.normal(size=(3, 3))
    u = (prob.coords @ A.T).ravel()
    f = K @ u
    x = prob.coords
    interior = np.all((x > 1e-9) & (x < 1 - 1e-9), axis=1)
    idx = (3 * np.nonzero(interior)[0][:, None] + np.arange(3)).ravel()
    assert np.abs(f[idx]).max() < 1e-12


MAT = {"kind": fem.HGO_TWO_FIBRE, "c": 3.0, "k1": 2.3632, "k2": 0.8393, "kappa": 3000.0,
       "E": 0.0, "nu": 0.0}


def _fibres(n):
    a = RNG.normal(size=(n, 2, 3))
    a /= np.linalg.norm(a, axis=2, keepdims=True)
    return a.reshape(n, 6)


def _def_grad(n, scale=0.15):
    return np.eye(3)[None] + scale * RNG.normal(size=(n, 3, 3))


def test_hgo_stress_is_energy_derivative():
    n = 12
    Fm = _def_grad(n)
    C = np.einsum("eiI,eiJ->eIJ", Fm, Fm)
    fib = _fibres(n)
    a1, a2 = fib[:, :3], fib[:, 3:]
    S = fem.hgo_stress(C, a1, a2, MAT)
    h = 1e-6
    for I in range(3):
        for J in range(3):
            D = np.zeros((3, 3))
            D[I, J] += 0.5
            D[J, I] += 0.5
            dpsi = (fem.hgo_energy(C + h * D, a1, a2, MAT) - fem.hgo_energy(C - h * D, a1, a2, MAT)) / (2 * h)
            # dPsi[D] = S : D / 2
            assert np.allclose(dpsi, 0.5 * np.einsum("eij,ij->e", S, D), rtol=1e-6, atol=1e-6 * np.abs(S).max())


def test_hgo_tangent_is_force_derivative_and_symmetric():
    X = _random_tets(6)
    fib = _fibres(6)
    U = 0.08 * RNG.normal(size=(6, 4, 3))
    f, K, detF = fem.hgo_element(X, U, fib, MAT)
    assert np.all(detF > 0)
    h = 1e-7
    Kfd = np.zeros_like(K)
    for k in range(12):
        dU = np.zeros((6, 12))
        dU[:, k] = h
        fp, _, _ = fem.hgo_element(X, U + dU.reshape(6, 4, 3), fib, MAT)
        fm, _, _ = fem.hgo_element(X, U - dU.reshape(6, 4, 3), fib, MAT)
        Kfd[:, :, k] = (fp - fm) / (2 * h)
    assert np.abs(K - Kfd).max() <= 1e-6 * np.abs(K).max()
    assert np.abs(K - K.transpose(0, 2, 1)).max() <= 1e-12 * np.abs(K).max()


def test_hgo_tangent_at_zero_strain_is_hooke():
    X = _random_tets(8)
    fib = _fibres(8)
    _, K, _ = fem.hgo_element(X, np.zeros((8, 4, 3)), fib, MAT)
    c, kappa = MAT["c"], MAT["kappa"]
    mu, lam = c, kappa - 2 * c / 3
    E = mu * (3 * lam + 2 * mu) / (lam + mu)
    nu = lam / (2 * (lam + mu))
    Kh = fem.linear_element(X, E, nu)
    assert np.abs(K - Kh).max() <= 1e-12 * np.abs(Kh).max()


def test_fibres_inactive_in_compression():
    """Under fibre-direction compression the anisotropic terms vanish (Sec. 3.1)."""
    a = np.array([[1.0, 0.0, 0.0]])
    Fm = np.diag([0.9, 1.0 / np.sqrt(0.9), 1.0 / np.sqrt(0.9)])[None]
    C = np.einsum("eiI,eiJ->eIJ", Fm, Fm)
    with_f = fem.hgo_stress(C, a, a, MAT)
    no_f = fem.hgo_stress(C, a, a, dict(MAT, k1=0.0))
    assert np.array_equal(with_f, no_f)
    Fm = np.diag([1.1, 1.0 / np.sqrt(1.1), 1.0 / np.sqrt(1.1)])[None]
    C = np.einsum("eiI,eiJ->eIJ", Fm, Fm)
    assert not np.allclose(fem.hgo_stress(C, a, a, MAT), fem.hgo_stress(C, a, a, dict(MAT, k1=0.0)))


def test_table1_parameters_golden():
    vals = {}
    for line in open(__file__.replace("test_oracle_fem.py", "golden/table1_material.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    m = mesh.hgo_material()
    assert (m["c"], m["k1"], m["k2"]) == (vals["c"], vals["k1"], vals["k2"])
    assert m["kappa"] == 1e3 * vals["c"]


def test_pressure_load_resultant_on_tube():
    """Uniform pressure on the closed inner surface: zero net force, total |F_r| = p * area."""
    prob = mesh.cylinder_problem(2, 32, 4, (1, 1, 1))
    f = fem.load_vector(prob).reshape(-1, 3)
    assert np.abs(f.sum(axis=0)).max() < 1e-15 * 1e3
    x = prob.coords
    inner = np.abs(np.hypot(x[:, 0], x[:, 1]) - 1.0) < 1e-12
    fr = (f[:, 0] * x[:, 0] + f[:, 1] * x[:, 1]) / np.hypot(x[:, 0], x[:, 1])
    # polygonal inner surface of 32 facets: perimeter 64 sin(pi/32), length 2
    area = 32 * 2 * np.sin(np.pi / 32) * 2.0
    # nodal forces are normal to the facets; their radial parts at the nodes
    # sum to p * area * cos(pi/32)
    assert np.isclose(fr[inner].sum(), prob.pressure * area * np.cos(np.pi / 32), rtol=1e-12)
    assert np.abs(fr[~inner]).max() == 0.0


def test_traction_load_resultant_and_moment_on_cube():
    """Constant traction t on the face x = 1 of the unit cube (area 1): the
    P1-consistent nodal forces sum to t * area, their first moment sum_n x_n f_n
    equals t times the face's first moment of area (centroid (1, 1/2, 1/2)),
    and no force acts off the face."""
    prob = mesh.cube_problem(6, (1, 1, 1))
    t = np.asarray(prob.traction, dtype=float)
    assert np.abs(t).max() > 0.0
    f = fem.load_vector(prob).reshape(-1, 3)
    x = prob.coords
    on_face = np.abs(x[:, 0] - 1.0) < 1e-12
    assert np.abs(f[~on_face]).max() == 0.0
    assert np.allclose(f.sum(axis=0), t * 1.0, rtol=0.0, atol=1e-15)
    moment = np.einsum("na,nb->ab", x, f)           # sum_n x_n (outer) f_n
    expected = np.outer([1.0, 0.5, 0.5], t) * 1.0
    assert np.allclose(moment, expected, rtol=0.0, atol=1e-15)
    # corner nodes of the face carry less than edge and interior nodes
    # (fewer incident triangles): the split is not uniform over nodes
    fz = f[on_face, 2]
    assert fz.min() < fz.max() < 0.0 or fz.max() < fz.min() < 0.0 or np.ptp(fz) > 0.0
