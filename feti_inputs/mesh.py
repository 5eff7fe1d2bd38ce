"""Structured tetrahedral meshes, partitions and boundary data (seeded, synthetic).

Hexahedral cells are split into six tetrahedra along the index-space diagonal
(Kuhn/Freudenthal split), identical in every cell, so the mesh is conforming,
including across the periodic seam of the tube.  Nodes are numbered
lexicographically: i fastest, then j, then k.  Tetrahedra are oriented to
positive volume.  Boundary triangles are listed with the tetrahedron that owns
them and are oriented so that (x1-x0)x(x2-x0) points into the solid.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# The six Kuhn tetrahedra of the unit cell: start at corner (0,0,0), step
# along the axes in the order of a permutation, end at (1,1,1).
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]

LINEAR_ISO = 0
HGO_TWO_FIBRE = 1
LINEAR_ISO_P0 = 2

# Table 1 of the paper: matrix and fibre parameters of the media (kPa).
TABLE1_C = 3.0
TABLE1_K1 = 2.3632
TABLE1_K2 = 0.8393


@dataclass
class Problem:
    """One boundary-value problem: mesh + partition + material + boundary data."""
    name: str
    coords: np.ndarray            # float64 [n_nodes, 3], reference configuration
    tets: np.ndarray              # int32 [n_tets, 4], positive orientation
    part: np.ndarray              # int32 [n_tets], subdomain of each tetrahedron
    n_parts: int
    dir_dof: np.ndarray           # int32 [n_dir], sorted, dof = 3*node + component
    dir_val: np.ndarray           # float64 [n_dir], prescribed displacement
    press_tri: np.ndarray         # int32 [n_press, 3], oriented into the solid
    press_owner: np.ndarray       # int32 [n_press], owning tetrahedron
    pressure: float               # surface pressure magnitude on press_tri
    trac_tri: np.ndarray          # int32 [n_trac, 3]
    trac_owner: np.ndarray        # int32 [n_trac]
    traction: np.ndarray          # float64 [3], constant traction on trac_tri
    material: dict                # kind + parameters
    fibres: np.ndarray | None = None   # float64 [n_tets, 6]: a1, a2 per element
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def _kuhn_tets(ni: int, nj: int, nk: int, node_id, periodic_j: bool = False):
    """Split an ni x nj x nk block of cells into 6*ni*nj*nk tetrahedra.

    node_id(i, j, k) maps (broadcast) index triples to node numbers.  Returns
    (tets int64 [E,4], cell int64 [E,3]); cells are lexicographic (i fastest),
    six tetrahedra per cell in _PERMS order.
    """
    ci, cj, ck = np.meshgrid(np.arange(ni), np.arange(nj), np.arange(nk), indexing="ij")
    # lexicographic with i fastest: transpose to (k, j, i) order then flatten
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    ncell = ci.size
    tets = np.empty((ncell, 6, 4), dtype=np.int64)
    for t, perm in enumerate(_PERMS):
        off = np.zeros(3, dtype=np.int64)
        corners = [off.copy()]
        for ax in perm:
            off[ax] += 1
            corners.append(off.copy())
        for v, c in enumerate(corners):
            jj = cj + c[1]
            if periodic_j:
                jj = jj % nj
            tets[:, t, v] = node_id(ci + c[0], jj, ck + c[2])
    cells = np.stack([ci, cj, ck], axis=1)
    return tets.reshape(-1, 4), np.repeat(cells, 6, axis=0)


def _orient(coords: np.ndarray, tets: np.ndarray) -> np.ndarray:
    x = coords[tets]
    vol6 = np.einsum("ij,ij->i", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])
    if np.any(vol6 == 0):
        raise ValueError("degenerate tetrahedron in generated mesh")
    t = tets.copy()
    neg = vol6 < 0
    t[neg, 2], t[neg, 3] = tets[neg, 3], tets[neg, 2]
    return t


def _boundary_faces(coords: np.ndarray, tets: np.ndarray, on_surface: np.ndarray):
    """Faces of tetrahedra whose three nodes all satisfy on_surface.

    Returns (tri int32 [T,3] oriented into the solid, owner int32 [T]).
    """
    tris, owners = [], []
    for omit in range(4):
        keep = [v for v in range(4) if v != omit]
        f = tets[:, keep]
        sel = np.all(on_surface[f], axis=1)
        if not np.any(sel):
            continue
        f = f[sel].copy()
        opp = tets[sel, omit]
        x0, x1, x2 = coords[f[:, 0]], coords[f[:, 1]], coords[f[:, 2]]
        nrm = np.cross(x1 - x0, x2 - x0)
        inward = np.einsum("ij,ij->i", nrm, coords[opp] - (x0 + x1 + x2) / 3.0) > 0
        f[~inward, 1], f[~inward, 2] = f[~inward, 2], f[~inward, 1].copy()
        tris.append(f)
        owners.append(np.nonzero(sel)[0])
    tri = np.concatenate(tris).astype(np.int32)
    own = np.concatenate(owners).astype(np.int32)
    order = np.lexsort((tri[:, 0], own))
    return tri[order], own[order]


def _empty_tri():
    return np.zeros((0, 3), dtype=np.int32), np.zeros(0, dtype=np.int32)


def linear_material(E: float = 1.0, nu: float = 0.3, p0: bool = False) -> dict:
    """Hooke's law; p0: volumetric part condensed to a piecewise-constant pressure (P2-P0 on P2 meshes)."""
    return {"kind": LINEAR_ISO_P0 if p0 else LINEAR_ISO, "E": float(E), "nu": float(nu),
            "c": 0.0, "k1": 0.0, "k2": 0.0, "kappa": 0.0}


def hgo_material(c: float = TABLE1_C, k1: float = TABLE1_K1, k2: float = TABLE1_K2,
                 kappa: float | None = None) -> dict:
    """Neo-Hookean matrix + two exponential fibre families + volumetric penalty."""
    if kappa is None:
        kappa = 1e3 * c
    return {"kind": HGO_TWO_FIBRE, "E": 0.0, "nu": 0.0,
            "c": float(c), "k1": float(k1), "k2": float(k2), "kappa": float(kappa)}


def cube_problem(n: int = 12, parts=(2, 2, 2), E: float = 1.0, nu: float = 0.3,
                 traction=(0.0, 0.0, -1e-2)) -> Problem:
    """Unit cube, n^3 cells, face x=0 clamped, constant traction on face x=1.

    Partition into parts[0] x parts[1] x parts[2] blocks of cells.
    """
    m = n + 1
    node_id = lambda i, j, k: i + m * (j + m * k)
    g = np.arange(m) / n
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    coords = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                       Z.transpose(2, 1, 0).ravel()], axis=1)
    tets, cells = _kuhn_tets(n, n, n, node_id)
    tets = _orient(coords, tets)
    px, py, pz = parts
    if n % px or n % py or n % pz:
        raise ValueError("cells must divide evenly into the partition")
    sx, sy, sz = n // px, n // py, n // pz
    part = (cells[:, 0] // sx) + px * ((cells[:, 1] // sy) + py * (cells[:, 2] // sz))
    ii = np.arange(coords.shape[0]) % m
    clamp_nodes = np.nonzero(ii == 0)[0]
    dir_dof = np.sort((3 * clamp_nodes[:, None] + np.arange(3)[None, :]).ravel())
    trac_tri, trac_owner = _boundary_faces(coords, tets, ii == n)
    press_tri, press_owner = _empty_tri()
    return Problem(
        name=f"cube{n}_p{px}x{py}x{pz}", coords=coords, tets=tets.astype(np.int32),
        part=part.astype(np.int32), n_parts=px * py * pz,
        dir_dof=dir_dof.astype(np.int32), dir_val=np.zeros(dir_dof.size),
        press_tri=press_tri, press_owner=press_owner, pressure=0.0,
        trac_tri=trac_tri, trac_owner=trac_owner, traction=np.asarray(traction, dtype=np.float64),
        material=linear_material(E, nu), meta={"cells": (n, n, n), "parts": tuple(parts)})


def kelvin_displacement(x: np.ndarray, E: float, nu: float, x_star=(-0.5, -0.5, -0.5)) -> np.ndarray:
    """Kelvin's fundamental solution for a unit point force along x_1 at x_star.

    U_k = (1+nu)/(8 pi E (1-nu)) * [(3-4nu) delta_1k / rho + (x_1-x_1*)(x_k-x_k*) / rho^3],
    rho = |x - x_star| (Sec. 5.1, Eq. fundSol, with its index l read as k).
    Boundary data of the cube study; x_star lies outside the unit cube.
    """
    d = x - np.asarray(x_star, dtype=np.float64)[None, :]
    rho = np.linalg.norm(d, axis=1)
    c = (1.0 + nu) / (8.0 * math.pi * E * (1.0 - nu))
    u = c * d[:, 0:1] * d / rho[:, None] ** 3
    u[:, 0] += c * (3.0 - 4.0 * nu) / rho
    return u


def kelvin_cube_problem(n: int = 16, parts=(8, 8, 8), E: float = 210.0, nu: float = 0.45,
                        x_star=(-0.5, -0.5, -0.5)) -> Problem:
    """Unit cube, n^3 cells, Dirichlet data of Kelvin's solution on the whole surface.

    The shape of the linear cube study of Sec. 5.1 (E = 210, nu = 0.45,
    Gamma_D = boundary, 8 x 8 x 8 = 512 sub-cubes); no loads.
    """
    base = cube_problem(n, parts, E=E, nu=nu)
    m = n + 1
    idx = np.arange(base.n_nodes)
    i, j, k = idx % m, (idx // m) % m, idx // (m * m)
    on_b = (i == 0) | (i == n) | (j == 0) | (j == n) | (k == 0) | (k == n)
    bn = np.nonzero(on_b)[0]
    uD = kelvin_displacement(base.coords[bn], E, nu, x_star)
    dof = (3 * bn[:, None] + np.arange(3)[None, :]).ravel()
    order = np.argsort(dof)
    e_tri, e_own = _empty_tri()
    return Problem(
        name=f"kelvin{n}_p{parts[0]}x{parts[1]}x{parts[2]}", coords=base.coords, tets=base.tets, part=base.part,
        n_parts=base.n_parts, dir_dof=dof[order].astype(np.int32), dir_val=uD.ravel()[order],
        press_tri=e_tri, press_owner=e_own, pressure=0.0, trac_tri=e_tri.copy(), trac_owner=e_own.copy(),
        traction=np.zeros(3), material=linear_material(E, nu),
        meta={"cells": (n, n, n), "parts": tuple(parts), "x_star": tuple(x_star)})


def _cylinder_nodes(nr, nt, nz, r_in, r_out, length, jitter, rng):
    ii, jj, kk = np.meshgrid(np.arange(nr + 1), np.arange(nt), np.arange(nz + 1), indexing="ij")
    ii = ii.transpose(2, 1, 0).ravel().astype(np.float64)
    jj = jj.transpose(2, 1, 0).ravel().astype(np.float64)
    kk = kk.transpose(2, 1, 0).ravel().astype(np.float64)
    ri, ti, zi = ii.copy(), jj.copy(), kk.copy()
    if jitter > 0.0:
        d = rng.uniform(-jitter, jitter, size=(ii.size, 3))
        on_r = (ii == 0) | (ii == nr)
        on_z = (kk == 0) | (kk == nz)
        # symmetry planes of the boundary conditions stay planar
        on_t = np.isin(jj, [0, nt // 4, nt // 2, 3 * nt // 4])
        ri = ri + np.where(on_r, 0.0, d[:, 0])
        ti = ti + np.where(on_t, 0.0, d[:, 1])
        zi = zi + np.where(on_z, 0.0, d[:, 2])
    r = r_in + (r_out - r_in) * ri / nr
    th = 2.0 * math.pi * ti / nt
    z = length * zi / nz
    coords = np.stack([r * np.cos(th), r * np.sin(th), z], axis=1)
    return coords, ii.astype(np.int64), jj.astype(np.int64), kk.astype(np.int64)


def _cylinder_bc(ii, jj, kk, nr, nt, nz):
    """u_z = 0 on both ends, u_y = 0 on theta in {0, pi}, u_x = 0 on theta in {pi/2, 3pi/2}."""
    nodes = np.arange(ii.size)
    dofs = [3 * nodes[(kk == 0) | (kk == nz)] + 2,
            3 * nodes[(jj == 0) | (jj == nt // 2)] + 1,
            3 * nodes[(jj == nt // 4) | (jj == 3 * nt // 4)] + 0]
    return np.unique(np.concatenate(dofs))


def _helical_fibres(coords, tets, alpha_deg):
    cen = coords[tets].mean(axis=1)
    th = np.arctan2(cen[:, 1], cen[:, 0])
    ca, sa = math.cos(math.radians(alpha_deg)), math.sin(math.radians(alpha_deg))
    et = np.stack([-np.sin(th), np.cos(th), np.zeros_like(th)], axis=1)
    ez = np.array([0.0, 0.0, 1.0])
    a1 = ca * et + sa * ez
    a2 = ca * et - sa * ez
    a1 /= np.linalg.norm(a1, axis=1, keepdims=True)
    a2 /= np.linalg.norm(a2, axis=1, keepdims=True)
    return np.concatenate([a1, a2], axis=1)


def _rcb(cent, n_parts, rng, frac_jitter):
    """Recursive coordinate bisection of cell centroids (any n_parts >= 1).

    Each cut goes across the longest extent; the left share of cells aims at
    (n_left/n_parts) * (1 + U(-frac_jitter, frac_jitter)) and is moved to the
    nearest gap between distinct centroid coordinates, so every part is a box
    of whole cell layers (face-connected on a structured grid).
    """
    part = np.zeros(cent.shape[0], dtype=np.int64)

    def rec(idx, first, count):
        if count == 1:
            part[idx] = first
            return
        nl = count // 2
        ext = cent[idx].max(axis=0) - cent[idx].min(axis=0)
        ax = int(np.argmax(ext))
        u = rng.uniform(-frac_jitter, frac_jitter) if frac_jitter > 0 else 0.0
        frac = (nl / count) * (1.0 + u)
        order = idx[np.argsort(cent[idx, ax], kind="stable")]
        vals = cent[order, ax]
        gaps = np.nonzero(vals[1:] > vals[:-1])[0] + 1
        if gaps.size == 0:
            raise ValueError("cannot bisect a single layer of cells")
        target = frac * idx.size
        cut = int(gaps[np.argmin(np.abs(gaps - target))])
        rec(order[:cut], first, nl)
        rec(order[cut:], first + nl, count - nl)

    rec(np.arange(cent.shape[0]), 0, n_parts)
    return part


def cylinder_problem(nr: int = 16, nt: int = 64, nz: int = 32, parts=(4, 8, 2),
                     r_in: float = 1.0, r_out: float = 1.5, length: float = 2.0,
                     pressure: float = 0.01, material: dict | None = None,
                     fibre_angle_deg: float = 49.98) -> Problem:
    """Thick-walled tube under internal pressure, structured wedge partition.

    Cells: nr radial x nt circumferential (periodic) x nz axial.  Partition
    parts = (radial, circumferential, axial) blocks of cells.
    """
    if material is None:
        material = linear_material(1.0, 0.3)
    coords, ii, jj, kk = _cylinder_nodes(nr, nt, nz, r_in, r_out, length, 0.0, None)
    node_id = lambda i, j, k: i + (nr + 1) * (j + nt * k)
    tets, cells = _kuhn_tets(nr, nt, nz, node_id, periodic_j=True)
    tets = _orient(coords, tets)
    pr, pt, pz = parts
    if nr % pr or nt % pt or nz % pz:
        raise ValueError("cells must divide evenly into the partition")
    part = (cells[:, 0] // (nr // pr)) + pr * ((cells[:, 1] // (nt // pt)) + pt * (cells[:, 2] // (nz // pz)))
    dir_dof = _cylinder_bc(ii, jj, kk, nr, nt, nz)
    press_tri, press_owner = _boundary_faces(coords, tets, ii == 0)
    trac_tri, trac_owner = _empty_tri()
    fibres = None
    if material["kind"] == HGO_TWO_FIBRE:
        fibres = _helical_fibres(coords, tets, fibre_angle_deg)
    return Problem(
        name=f"cyl{nr}x{nt}x{nz}_p{pr}x{pt}x{pz}", coords=coords, tets=tets.astype(np.int32),
        part=part.astype(np.int32), n_parts=pr * pt * pz,
        dir_dof=dir_dof.astype(np.int32), dir_val=np.zeros(dir_dof.size),
        press_tri=press_tri, press_owner=press_owner, pressure=float(pressure),
        trac_tri=trac_tri, trac_owner=trac_owner, traction=np.zeros(3),
        material=material, fibres=fibres,
        meta={"cells": (nr, nt, nz), "parts": tuple(parts), "r_in": r_in, "r_out": r_out,
              "length": length})


def jittered_cylinder_problem(nr: int, nt: int, nz: int, n_parts: int, mesh_seed: int,
                              part_seed: int, jitter: float = 0.2, cut_jitter: float = 0.15,
                              r_in: float = 1.0, r_out: float = 1.5, length: float = 2.0,
                              pressure: float = 0.01) -> Problem:
    """Tube with nodes jittered by +-jitter cells (seeded) and a jittered RCB partition.

    Interior nodes move in all three index directions; nodes on r = r_in,
    r_out move only tangentially, nodes on the end faces only in r and theta,
    nodes on the four symmetry half-planes of the boundary conditions stay in
    their plane.  The partition bisects cell centroids in (r, 1.25*theta, z).
    """
    rng = np.random.Generator(np.random.PCG64(mesh_seed))
    coords, ii, jj, kk = _cylinder_nodes(nr, nt, nz, r_in, r_out, length, jitter, rng)
    node_id = lambda i, j, k: i + (nr + 1) * (j + nt * k)
    tets, cells = _kuhn_tets(nr, nt, nz, node_id, periodic_j=True)
    tets = _orient(coords, tets)
    # partition cells by their index-space centroid mapped to (r, 1.25 theta, z)
    ncell = nr * nt * nz
    cell_of_tet = np.arange(tets.shape[0]) // 6
    cc = cells[::6].astype(np.float64) + 0.5
    cent = np.stack([r_in + (r_out - r_in) * cc[:, 0] / nr,
                     1.25 * 2.0 * math.pi * cc[:, 1] / nt,
                     length * cc[:, 2] / nz], axis=1)
    prng = np.random.Generator(np.random.PCG64(part_seed))
    cpart = _rcb(cent, n_parts, prng, cut_jitter)
    assert cpart.size == ncell
    part = cpart[cell_of_tet]
    dir_dof = _cylinder_bc(ii, jj, kk, nr, nt, nz)
    press_tri, press_owner = _boundary_faces(coords, tets, ii == 0)
    trac_tri, trac_owner = _empty_tri()
    return Problem(
        name=f"jcyl{nr}x{nt}x{nz}_p{n_parts}", coords=coords, tets=tets.astype(np.int32),
        part=part.astype(np.int32), n_parts=int(n_parts),
        dir_dof=dir_dof.astype(np.int32), dir_val=np.zeros(dir_dof.size),
        press_tri=press_tri, press_owner=press_owner, pressure=float(pressure),
        trac_tri=trac_tri, trac_owner=trac_owner, traction=np.zeros(3),
        material=linear_material(1.0, 0.3),
        meta={"cells": (nr, nt, nz), "parts": n_parts, "mesh_seed": mesh_seed,
              "part_seed": part_seed, "jitter": jitter, "cut_jitter": cut_jitter,
              "r_in": r_in, "r_out": r_out, "length": length})


# Edges of a tetrahedron in the P2 node order: nodes 4..9 are the midpoints of
# the vertex pairs (0,1), (0,2), (0,3), (1,2), (1,3), (2,3).
P2_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def p2_problem(prob: Problem, dirichlet=None) -> Problem:
    """The same problem on 10-node (P2) tetrahedra: the P1 mesh's vertices keep
    their numbers, each edge gets a midpoint node numbered after them (edges in
    order of their sorted vertex pairs), tets become [E, 10] (vertices, then the
    midpoints of P2_EDGES) and loaded triangles [T, 6] (vertices v0 v1 v2, then
    the midpoints of (v0,v1), (v1,v2), (v2,v0)).  dirichlet(coords) -> (dofs,
    values) recomputes the Dirichlet data on the new node set (default: a DOF is
    prescribed iff both end vertices of its edge carry that DOF, with the mean
    of their values -- exact for homogeneous and affine data)."""
    N = prob.n_nodes
    t = prob.tets.astype(np.int64)
    pairs = np.concatenate([np.sort(t[:, [a, b]], axis=1) for a, b in P2_EDGES], axis=0)
    key = pairs[:, 0] * N + pairs[:, 1]
    uniq, inv = np.unique(key, return_inverse=True)
    ea, eb = uniq // N, uniq % N
    coords = np.concatenate([prob.coords, 0.5 * (prob.coords[ea] + prob.coords[eb])], axis=0)
    E = t.shape[0]
    mid = (N + inv).reshape(6, E).T
    tets10 = np.concatenate([t, mid], axis=1).astype(np.int32)
    edge_id = dict(zip(uniq.tolist(), range(uniq.size)))

    def midpoint(a, b):
        lo, hi = np.minimum(a, b), np.maximum(a, b)
        return N + np.array([edge_id[k] for k in (lo * N + hi).tolist()], dtype=np.int64)

    def faces6(tri):
        if tri.shape[0] == 0:
            return np.zeros((0, 6), np.int32)
        tri = tri.astype(np.int64)
        m01 = midpoint(tri[:, 0], tri[:, 1])
        m12 = midpoint(tri[:, 1], tri[:, 2])
        m20 = midpoint(tri[:, 2], tri[:, 0])
        return np.concatenate([tri, m01[:, None], m12[:, None], m20[:, None]], axis=1).astype(np.int32)

    if dirichlet is not None:
        dir_dof, dir_val = dirichlet(coords)
    else:
        pres = np.zeros(3 * N, bool)
        val = np.zeros(3 * N)
        pres[prob.dir_dof] = True
        val[prob.dir_dof] = prob.dir_val
        d, v = [prob.dir_dof.astype(np.int64)], [prob.dir_val]
        for c in range(3):
            both = pres[3 * ea + c] & pres[3 * eb + c]
            idx = np.nonzero(both)[0]
            d.append(3 * (N + idx) + c)
            v.append(0.5 * (val[3 * ea[idx] + c] + val[3 * eb[idx] + c]))
        d, v = np.concatenate(d), np.concatenate(v)
        order = np.argsort(d)
        dir_dof, dir_val = d[order], v[order]
    meta = dict(prob.meta)
    meta["order"] = 2
    return Problem(name=prob.name + "_p2", coords=coords, tets=tets10, part=prob.part.copy(), n_parts=prob.n_parts,
                   dir_dof=np.asarray(dir_dof, dtype=np.int32), dir_val=np.asarray(dir_val, dtype=np.float64),
                   press_tri=faces6(prob.press_tri), press_owner=prob.press_owner.copy(), pressure=prob.pressure,
                   trac_tri=faces6(prob.trac_tri), trac_owner=prob.trac_owner.copy(), traction=prob.traction.copy(),
                   material=dict(prob.material), fibres=None if prob.fibres is None else prob.fibres.copy(), meta=meta)


def kelvin_cube_problem_p2(n: int = 4, parts=(2, 2, 2), E: float = 210.0, nu: float = 0.45,
                           x_star=(-0.5, -0.5, -0.5)) -> Problem:
    """Kelvin-solution cube on P2 tetrahedra (the quadratic study of Sec. 5.1,
    Table 3): Dirichlet data of Kelvin's solution at every boundary node,
    vertices and edge midpoints."""
    base = kelvin_cube_problem(n, parts, E=E, nu=nu, x_star=x_star)

    def kelvin_data(coords):
        tol = 1e-12
        on_b = np.any((coords < tol) | (coords > 1.0 - tol), axis=1)
        bn = np.nonzero(on_b)[0]
        uD = kelvin_displacement(coords[bn], E, nu, x_star)
        dof = (3 * bn[:, None] + np.arange(3)[None, :]).ravel()
        order = np.argsort(dof)
        return dof[order], uD.ravel()[order]

    return p2_problem(base, kelvin_data)


def config_problem(name: str) -> Problem:
    """The named synthetic workloads (cube / tube sizes of the paper's experiments)."""
    if name == "cube12":          # 2197 nodes, 8 sub-cubes, H/h = 6
        return cube_problem(12, (2, 2, 2))
    if name == "cyl16":           # 35,904 nodes, 64 wedge subdomains
        return cylinder_problem(16, 64, 32, (4, 8, 2))
    if name == "cyl24_hgo":       # 117,600 nodes, 256 subdomains, Table 1 material
        return cylinder_problem(24, 96, 48, (4, 16, 4), material=hgo_material(), pressure=16.0)
    if name == "jcyl32":          # 274,560 nodes, 1024 uneven subdomains
        return jittered_cylinder_problem(32, 128, 64, 1024, 1508, 2599)
    if name == "jcyl16":          # 35,904 nodes, 128 uneven subdomains (jcyl32's subdomain sizes)
        return jittered_cylinder_problem(16, 64, 32, 128, 1510, 2601)
    if name == "jcyl48":          # 912,576 nodes, 4096 uneven subdomains
        return jittered_cylinder_problem(48, 192, 96, 4096, 1509, 2600)
    raise KeyError(name)
