"""FP64 CPU oracle of classical and all-floating FETI with projected PCG.

Follows Sec. 4 of the paper step by step:
  * Sec. 4 (reordering) and 4.1 (tearing): local matrices K_i' and loads f_i
    from each subdomain's own elements; continuity by the signed jump
    operator sum_i B_i u_i = 0 with entries in {0, 1, -1}, fully redundant
    (Fig. 3a: every pair of subdomains sharing a node gets a constraint);
  * Sec. 4.2 (all-floating): Dirichlet DOFs stay in every subdomain and get
    one extra constraint row per subdomain copy, right-hand side b = [0; b_D];
  * Sec. 4.3: generalized inverse K_i^+, rigid-body kernels r_{k,i}, dual
    operators F = sum B_i K_i^+ B_i^T, G = [B_i R_i], d = sum B_i K_i^+ f_i,
    e_{k,i} = (f_i, r_{k,i}); projection P = I - G (G^T G)^-1 G^T; initial
    lambda_0 = G (G^T G)^-1 e; CG on the projected dual problem; recovery of
    gamma = (G^T G)^-1 G^T (F lambda - d) and of the local solutions;
  * Sec. 4.4: preconditioner sum_i B_D,i Y_i B_D,i^T with multiplicity
    scaling, Y_i = K_i' (lumped), diag(0, S_i) (Dirichlet) or I.

Readings where the paper is silent, garbled or at odds with itself:
  1. the projection is printed with (G G^T)^-1, which has the wrong size; it
     is I - G (G^T G)^-1 G^T, as in the formulas for lambda_0 and gamma;
  2. G is the column blocks [B_1 R_1, ..., B_p R_p] (printed as a double sum);
  3. the solvability condition runs over the kernel index k, not i;
  4. B_D,i of the preconditioner is the multiplicity-scaled constraint
     operator, a different object from the Dirichlet block of B~_i;
  5. all-floating: the derivation gives F lambda - G gamma = d - b, so the dual
     right-hand side is d~ = d - b and gamma uses F lambda - d~;
  6. the generalized inverse "by fixing nodes" is K^+ = P^T diag(K_rr^-1, 0) P
     with k_i fixing DOFs chosen among the boundary DOFs by column-pivoted QR
     of R_b^T (largest remaining norm, ties within 1e-10 relative to the
     lowest local DOF);  any generalized inverse gives the same projected
     operator, so iterates and solution do not depend on the choice;
  7. stopping: ||P r_k||_2 <= tol ||P r_0||_2;
  8. preconditioner placement: y = P M^-1 P r (projection on both sides);
  9. multiplicity weights: 1/m(n) on interface rows at node n.  Under
     all-floating FETI the Dirichlet boundary is one more participant, of
     infinite stiffness (the limit of stiffness-weighted multiplicity
     scaling): at a Dirichlet DOF the Dirichlet rows weigh 1 and the
     interface rows 0.  With equal weights 1/(m+1) instead, all-floating
     FETI needed more iterations than classical FETI, against the trend of
     Tables 2 and 4;
 10. classical kernels: R_i = RBM_i N_i, N_i an orthonormal basis of the null
     space of the rigid-body modes restricted to the subdomain's Dirichlet
     DOFs (SVD, rank threshold 1e-10 sigma_max), so dim ker < 6 for
     subdomains touching the Dirichlet boundary in a vertex, edge or face;
 11. multiplier order: interface rows by global node, component, then
     subdomain pair (i < j, lexicographic), entries +1 on i and -1 on j;
     all-floating Dirichlet rows after them by (node, component, subdomain);
 12. shared nodes of the recovered displacement take the value of the lowest
     subdomain id (copies agree to the solver tolerance);
 13. the condition number is the Lanczos estimate from the CG coefficients.

Pins (tests/test_oracle_feti.py): FETI solution equals the monolithic direct
solve; K_i R_i = 0; K K^+ K = K; G^T lambda_k = e every iteration; P^2 = P,
P G = 0; jump B u - b -> 0; two fixing choices give the same solution and
iteration count; Lame closed form for the tube.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import time

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem

CLASSICAL = "classical"
ALL_FLOATING = "af"


def rigid_body_modes(x: np.ndarray) -> np.ndarray:
    """Six rigid-body modes [n_nodes*3, 6] about the mean node position.

    Columns: translations e_x, e_y, e_z, then rotations e_z x d, e_x x d,
    e_y x d with d = x - mean(x).
    """
    d = x - x.mean(axis=0)
    n = x.shape[0]
    R = np.zeros((n, 3, 6))
    R[:, 0, 0] = 1.0
    R[:, 1, 1] = 1.0
    R[:, 2, 2] = 1.0
    R[:, 0, 3], R[:, 1, 3] = -d[:, 1], d[:, 0]          # e_z x d
    R[:, 1, 4], R[:, 2, 4] = -d[:, 2], d[:, 1]          # e_x x d
    R[:, 2, 5], R[:, 0, 5] = -d[:, 0], d[:, 2]          # e_y x d
    return R.reshape(3 * n, 6)


def pivoted_rows(R: np.ndarray, k: int, tie_rel: float = 1e-10) -> list[int]:
    """k row indices of R chosen by column-pivoted QR of R^T (Gram-Schmidt)."""
    W = R.astype(np.float64).copy()
    chosen: list[int] = []
    for _ in range(k):
        nrm = np.einsum("ij,ij->i", W, W)
        nrm[chosen] = -1.0
        top = nrm.max()
        cand = np.nonzero(nrm >= top * (1.0 - tie_rel))[0]
        j = int(cand.min())
        chosen.append(j)
        q = W[j] / np.sqrt(nrm[j])
        W = W - np.outer(W @ q, q)
    return chosen


@dataclass
class Subdomain:
    nodes: np.ndarray          # global node ids, ascending
    free: np.ndarray           # local DOFs (into 3*n_nodes) kept in K_i
    bnd: np.ndarray            # positions (into free) of DOFs touched by B~_i
    fix: np.ndarray            # local DOFs (into 3*n_nodes) of the fixing set
    R: np.ndarray              # kernel basis on free DOFs [n_free, k]
    B: sp.csr_matrix = None    # [n_lambda, n_free]
    K: np.ndarray = None       # dense K_i' on free DOFs
    f: np.ndarray = None       # local load on free DOFs
    chol: tuple = None         # Cholesky of K_rr
    r_pos: np.ndarray = None   # positions (into free) of the non-fixing DOFs
    Y: np.ndarray = None       # preconditioner block on bnd


@dataclass
class IndexMaps:
    """Canonical multiplier numbering (reading 11): two entries per row, -1 padded."""
    row_sub: np.ndarray        # int32 [n_lambda, 2]
    row_ldof: np.ndarray       # int32 [n_lambda, 2], local DOF = 3*local node + comp
    row_sign: np.ndarray       # int8  [n_lambda, 2]
    b: np.ndarray              # float64 [n_lambda]
    weight: np.ndarray         # float64 [n_lambda]
    mult: np.ndarray           # int32 [n_nodes]


def build_index_maps(prob, method: str):
    """Local numbering, multiplicities and the signed constraint rows."""
    P, N = prob.n_parts, prob.n_nodes
    nodes = [np.unique(prob.tets[prob.part == s]) for s in range(P)]
    mult = np.zeros(N, dtype=np.int32)
    subs_of = [[] for _ in range(N)]
    for s in range(P):
        mult[nodes[s]] += 1
        for n in nodes[s]:
            subs_of[n].append(s)
    lidx = [dict(zip(nodes[s].tolist(), range(len(nodes[s])))) for s in range(P)]
    is_dir = np.zeros(3 * N, dtype=bool)
    is_dir[prob.dir_dof] = True
    dval = np.zeros(3 * N)
    dval[prob.dir_dof] = prob.dir_val
    af = method == ALL_FLOATING
    rs, rl, rg, rb, rw = [], [], [], [], []
    for n in range(N):
        S = subs_of[n]
        if len(S) < 2:
            continue
        for c in range(3):
            dof = 3 * n + c
            if not af and is_dir[dof]:
                continue
            w = 0.0 if (af and is_dir[dof]) else 1.0 / len(S)
            for a in range(len(S)):
                for bb in range(a + 1, len(S)):
                    i, j = S[a], S[bb]
                    rs.append((i, j))
                    rl.append((3 * lidx[i][n] + c, 3 * lidx[j][n] + c))
                    rg.append((1, -1))
                    rb.append(0.0)
                    rw.append(w)
    if af:
        for dof in np.sort(prob.dir_dof):
            n, c = int(dof) // 3, int(dof) % 3
            S = subs_of[n]
            w = 1.0
            for i in S:
                rs.append((i, -1))
                rl.append((3 * lidx[i][n] + c, -1))
                rg.append((1, 0))
                rb.append(dval[dof])
                rw.append(w)
    maps = IndexMaps(np.array(rs, dtype=np.int32).reshape(-1, 2),
                     np.array(rl, dtype=np.int32).reshape(-1, 2),
                     np.array(rg, dtype=np.int8).reshape(-1, 2),
                     np.array(rb, dtype=np.float64), np.array(rw, dtype=np.float64), mult)
    return nodes, maps, is_dir, dval


@dataclass
class PCGResult:
    lam: np.ndarray
    iterations: int
    converged: bool
    res_hist: list
    alphas: list
    betas: list
    cond_est: float
    compat_err: float = 0.0


class FetiOracle:
    """Classical / all-floating FETI on one problem (FP64, dense local algebra)."""

    def __init__(self, prob, method: str = ALL_FLOATING, precond: str = "dirichlet",
                 fix_override: dict | None = None):
        self.prob = prob
        self.method = method
        self.precond = precond
        self.timings = {}
        t0 = time.perf_counter()
        self.nodes, self.maps, self.is_dir, self.dval = build_index_maps(prob, method)
        self.n_lambda = self.maps.b.size
        self._build_subdomains(fix_override)
        self.timings["maps"] = time.perf_counter() - t0

    # ---- structure -----------------------------------------------------
    def _build_subdomains(self, fix_override):
        prob, maps = self.prob, self.maps
        af = self.method == ALL_FLOATING
        self.subs: list[Subdomain] = []
        for s, nod in enumerate(self.nodes):
            ndof = 3 * nod.size
            gdof = (3 * nod[:, None] + np.arange(3)[None, :]).ravel()
            free = np.arange(ndof) if af else np.nonzero(~self.is_dir[gdof])[0]
            pos = -np.ones(ndof, dtype=np.int64)
            pos[free] = np.arange(free.size)
            # B~_i as a sparse [n_lambda, n_free] matrix with +-1 entries
            rr, cc, vv = [], [], []
            for e in range(2):
                m = maps.row_sub[:, e] == s
                rows = np.nonzero(m)[0]
                rr.append(rows)
                cc.append(pos[maps.row_ldof[rows, e]])
                vv.append(maps.row_sign[rows, e].astype(np.float64))
            rr, cc, vv = np.concatenate(rr), np.concatenate(cc), np.concatenate(vv)
            if np.any(cc < 0):
                raise AssertionError("constraint row on an eliminated DOF")
            B = sp.csr_matrix((vv, (rr, cc)), shape=(self.n_lambda, free.size))
            bnd = np.unique(cc)
            # kernel (Sec. 4.3): six rigid-body modes, restricted for classical
            RBM = rigid_body_modes(prob.coords[nod])
            if af:
                N6 = np.eye(6)
            else:
                cons = np.nonzero(self.is_dir[gdof])[0]
                if cons.size == 0:
                    N6 = np.eye(6)
                else:
                    _, sv, Vt = np.linalg.svd(RBM[cons], full_matrices=True)
                    rank = int(np.sum(sv > 1e-10 * sv.max()))
                    N6 = Vt[rank:].T
            R = RBM[free] @ N6
            k = R.shape[1]
            if fix_override is not None and s in fix_override:
                fix = np.asarray(fix_override[s], dtype=np.int64)
            else:
                sel = pivoted_rows(R[bnd], k) if k else []
                fix = free[bnd[np.asarray(sel, dtype=np.int64)]] if k else np.zeros(0, np.int64)
            self.subs.append(Subdomain(nodes=nod, free=free, bnd=bnd, fix=fix, R=R, B=B))

    def coarse_dim(self) -> int:
        return int(sum(sd.R.shape[1] for sd in self.subs))

    # ---- local matrices (Sec. 4.1 / 4.2) -------------------------------
    def assemble(self, U: np.ndarray | None = None, tau: float = 1.0, follower: bool = True):
        """Local K_i' and f_i on the free DOFs from each subdomain's own elements.

        Linear: f_i = local load (minus K_iD u_D for classical elimination).
        Hyperelastic: f_i = tau * local load(U) - local internal force(U).
        """
        prob = self.prob
        Ke, fint = fem.element_matrices(prob, None if U is None else U.reshape(-1, 3))
        owners, verts, forces = fem.surface_loads(prob, None if U is None else U.reshape(-1, 3), follower)
        tri_part = prob.part[owners] if owners.size else np.zeros(0, np.int64)
        nd = 3 * prob.tets.shape[1]
        for s, sd in enumerate(self.subs):
            nod = sd.nodes
            ndof = 3 * nod.size
            els = np.nonzero(prob.part == s)[0]
            ln = np.searchsorted(nod, prob.tets[els])
            ld = (3 * ln[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, nd)
            Kfull = np.zeros((ndof, ndof))
            np.add.at(Kfull, (ld[:, :, None], ld[:, None, :]), Ke[els])
            ffull = np.zeros(ndof)
            tri = np.nonzero(tri_part == s)[0]
            if tri.size:
                lt = np.searchsorted(nod, verts[tri])
                if verts.shape[1] == 6:       # P2 faces: a force per face node
                    for v in range(6):
                        np.add.at(ffull, (3 * lt[:, v][:, None] + np.arange(3)[None, :]).ravel(),
                                  (tau * forces[tri][:, v, :]).ravel())
                else:
                    for v in range(3):
                        np.add.at(ffull, (3 * lt[:, v][:, None] + np.arange(3)[None, :]).ravel(),
                                  (tau * forces[tri]).ravel())
            if fint is not None:
                np.add.at(ffull, ld.ravel(), -fint[els].ravel())
            gdof = (3 * nod[:, None] + np.arange(3)[None, :]).ravel()
            if self.method == CLASSICAL and U is None:
                dcol = np.nonzero(self.is_dir[gdof])[0]
                ffull = ffull - Kfull[:, dcol] @ self.dval[gdof[dcol]]
            sd.K = Kfull[np.ix_(sd.free, sd.free)]
            sd.f = ffull[sd.free]

    def factorize(self):
        """Generalized inverses (reading 6) and preconditioner blocks (Sec. 4.4)."""
        t0 = time.perf_counter()
        for sd in self.subs:
            fixpos = np.searchsorted(sd.free, sd.fix)
            keep = np.ones(sd.free.size, dtype=bool)
            keep[fixpos] = False
            sd.r_pos = np.nonzero(keep)[0]
            sd.chol = sla.cho_factor(sd.K[np.ix_(sd.r_pos, sd.r_pos)], lower=True)
            b = sd.bnd
            if self.precond == "dirichlet":
                inner = np.setdiff1d(np.arange(sd.free.size), b)
                if inner.size:
                    KII = sla.cho_factor(sd.K[np.ix_(inner, inner)], lower=True)
                    KIb = sd.K[np.ix_(inner, b)]
                    sd.Y = sd.K[np.ix_(b, b)] - KIb.T @ sla.cho_solve(KII, KIb)
                else:
                    sd.Y = sd.K[np.ix_(b, b)].copy()
            elif self.precond == "lumped":
                sd.Y = sd.K[np.ix_(b, b)].copy()
            elif self.precond == "identity":
                sd.Y = np.eye(b.size)
            else:
                raise ValueError(self.precond)
        self._coarse()
        self.timings["factorize"] = time.perf_counter() - t0

    def kplus(self, sd: Subdomain, g: np.ndarray) -> np.ndarray:
        """K_i^+ g with the fixing-DOF generalized inverse (zero on fixing DOFs)."""
        x = np.zeros_like(g)
        x[sd.r_pos] = sla.cho_solve(sd.chol, g[sd.r_pos])
        return x

    def _coarse(self):
        """G = [B_1 R_1, ..., B_p R_p] (Sec. 4.3, read as column blocks), kept
        sparse: block i is nonzero only on the multiplier rows of subdomain i;
        G^T G is dense (cd x cd) and factored by Cholesky."""
        cols = [sp.csc_matrix(sd.B @ sd.R) for sd in self.subs if sd.R.shape[1]]
        self.G = sp.hstack(cols, format="csr") if cols else sp.csr_matrix((self.n_lambda, 0))
        self.GtG = (self.G.T @ self.G).toarray()
        self.GtG_chol = sla.cho_factor(self.GtG, lower=True) if self.G.shape[1] else None

    # ---- dual operators (Sec. 4.3) --------------------------------------
    def apply_F(self, lam: np.ndarray) -> np.ndarray:
        """F lambda = sum_i B_i K_i^+ B_i^T lambda."""
        q = np.zeros(self.n_lambda)
        for sd in self.subs:
            q += sd.B @ self.kplus(sd, sd.B.T @ lam)
        return q

    def apply_prec(self, w: np.ndarray) -> np.ndarray:
        """M^-1 w = sum_i B_D,i Y_i B_D,i^T w with B_D = W B (W: multiplicity weights)."""
        ww = self.maps.weight * w
        z = np.zeros(self.n_lambda)
        for sd in self.subs:
            v = (sd.B.T @ ww)[sd.bnd]
            y = np.zeros(sd.free.size)
            y[sd.bnd] = sd.Y @ v
            z += sd.B @ y
        return self.maps.weight * z

    def coarse_solve(self, v: np.ndarray) -> np.ndarray:
        return sla.cho_solve(self.GtG_chol, v)

    def project(self, v: np.ndarray) -> np.ndarray:
        """P v = v - G (G^T G)^-1 G^T v."""
        if self.G.shape[1] == 0:
            return v.copy()
        return v - self.G @ self.coarse_solve(self.G.T @ v)

    def rhs(self):
        """d~ = sum B_i K_i^+ f_i - b, e = (R_i^T f_i), lambda_0 = G (G^T G)^-1 e."""
        d = np.zeros(self.n_lambda)
        for sd in self.subs:
            d += sd.B @ self.kplus(sd, sd.f)
        d -= self.maps.b
        e = np.concatenate([sd.R.T @ sd.f for sd in self.subs if sd.R.shape[1]] or [np.zeros(0)])
        lam0 = self.G @ self.coarse_solve(e) if e.size else np.zeros(self.n_lambda)
        return d, e, lam0

    def pcg(self, tol: float = 1e-10, maxit: int = 1000, check_compat: bool = False) -> PCGResult:
        """Projected preconditioned CG on P^T F lambda = P^T d~ (readings 7, 8)."""
        d, e, lam = self.rhs()
        r = d - self.apply_F(lam)
        hist, alphas, betas = [], [], []
        w = self.project(r)
        w0 = np.linalg.norm(w)
        hist.append(w0)
        p = None
        rho_prev = None
        it = 0
        converged = w0 == 0.0
        compat = 0.0
        while not converged and it < maxit:
            z = self.apply_prec(w)
            y = self.project(z)
            rho = float(w @ y)
            if p is None:
                p = y.copy()
                beta = 0.0
            else:
                beta = rho / rho_prev
                p = y + beta * p
            q = self.apply_F(p)
            pq = float(p @ q)
            if not (pq > 0.0) or not np.isfinite(pq):
                raise FloatingPointError("PCG breakdown: (p, Fp) <= 0")
            alpha = rho / pq
            lam = lam + alpha * p
            r = r - alpha * q
            it += 1
            alphas.append(alpha)
            betas.append(beta)
            rho_prev = rho
            w = self.project(r)
            nw = np.linalg.norm(w)
            hist.append(nw)
            if check_compat and e.size:
                compat = max(compat, float(np.linalg.norm(self.G.T @ lam - e) / max(np.linalg.norm(e), 1e-300)))
            converged = nw <= tol * w0
        return PCGResult(lam, it, converged, hist, alphas, betas, lanczos_cond(alphas, betas), compat)

    def recover(self, lam: np.ndarray):
        """gamma = (G^T G)^-1 G^T (F lambda - d~); u_i = K_i^+(f_i - B_i^T lambda) + R_i gamma_i."""
        d, _, _ = self.rhs()
        res = self.apply_F(lam) - d
        gamma = self.coarse_solve(self.G.T @ res) if self.G.shape[1] else np.zeros(0)
        us = []
        off = 0
        for sd in self.subs:
            k = sd.R.shape[1]
            u = self.kplus(sd, sd.f - sd.B.T @ lam)
            if k:
                u = u + sd.R @ gamma[off:off + k]
                off += k
            us.append(u)
        return us, gamma

    def global_displacement(self, us) -> np.ndarray:
        """Owner rule (reading 12): lowest subdomain id wins; Dirichlet DOFs get u_D."""
        N = self.prob.n_nodes
        U = np.full(3 * N, np.nan)
        for s in range(len(self.subs) - 1, -1, -1):
            sd = self.subs[s]
            gdof = (3 * sd.nodes[:, None] + np.arange(3)[None, :]).ravel()
            U[gdof[sd.free]] = us[s]
        if self.method == CLASSICAL:
            U[self.prob.dir_dof] = self.prob.dir_val
        return U

    def jump(self, us) -> float:
        """||sum_i B~_i u_i - b||_2."""
        v = -self.maps.b.copy()
        for sd, u in zip(self.subs, us):
            v += sd.B @ u
        return float(np.linalg.norm(v))

    def solve(self, tol: float = 1e-10, maxit: int = 1000, check_compat: bool = False):
        """Linear solve: assemble, factorize, PCG, recover.  Returns (U, PCGResult, us)."""
        t0 = time.perf_counter()
        self.assemble()
        self.factorize()
        t1 = time.perf_counter()
        res = self.pcg(tol, maxit, check_compat)
        t2 = time.perf_counter()
        us, _ = self.recover(res.lam)
        self.timings.update(local=t1 - t0, pcg=t2 - t1, total=time.perf_counter() - t0)
        return self.global_displacement(us), res, us


def lanczos_cond(alphas, betas) -> float:
    """Condition estimate from CG coefficients (tridiagonal Lanczos matrix).

    T_jj = 1/alpha_j + beta_j/alpha_{j-1}, T_j,j+1 = sqrt(beta_{j+1})/alpha_j.
    """
    m = len(alphas)
    if m == 0:
        return 1.0
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / alphas[j] + (betas[j] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j + 1]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return float(ev.max() / ev.min())


def newton_solve(prob, method: str = ALL_FLOATING, precond: str = "dirichlet",
                 n_load_steps: int = 10, newton_tol: float = 1e-8, newton_maxit: int = 25,
                 pcg_tol: float = 1e-10, pcg_maxit: int = 3000, follower: bool = True,
                 min_step: float = 1.0 / 64):
    """Load-stepped Newton (Eq. loadStepping) with a FETI solve per step.

    tau = s / n_load_steps; stop when ||R||_2 <= newton_tol ||tau f_ext||_2 on
    the free DOFs, R = f_int(U) - tau f_ext(U).  Increments satisfy homogeneous
    Dirichlet conditions (b = 0).  Kernels, fixing DOFs and G stay those of the
    reference configuration.

    Reading: the paper's tangent is positive definite only near equilibrium;
    with the volumetric penalty the full first step from U = 0 overshoots and
    leaves local tangents indefinite (the Cholesky factorization of K_rr
    fails).  The step length is therefore halved (down to min_step) until the
    local tangents at U + a dU factorize.  Returns (U, log) with one list per
    load step of (relative residual, PCG iterations, step length).
    """
    N = prob.n_nodes
    U = np.zeros(3 * N)
    if np.any(prob.dir_val != 0.0):
        raise NotImplementedError("inhomogeneous Dirichlet data in the nonlinear driver")
    solver = FetiOracle(prob, method, precond)
    free = np.ones(3 * N, dtype=bool)
    free[prob.dir_dof] = False

    def residual(U, tau):
        _, fint = fem.element_matrices(prob, U.reshape(-1, 3))
        fext = fem.load_vector(prob, U.reshape(-1, 3), follower)
        R = fem.internal_force_global(prob, fint) - tau * fext
        return np.linalg.norm(R[free]) / np.linalg.norm(tau * fext[free])

    def factorizes(U, tau):
        solver.assemble(U, tau, follower)
        try:
            solver.factorize()
            return True
        except (np.linalg.LinAlgError, sla.LinAlgError):
            return False

    log = []
    for step in range(1, n_load_steps + 1):
        tau = step / n_load_steps
        its = []
        if not factorizes(U, tau):
            raise RuntimeError("local tangent not positive definite at the start of a load step")
        rel = residual(U, tau)
        for k in range(newton_maxit + 1):
            if rel <= newton_tol:
                break
            if k == newton_maxit:
                raise RuntimeError(f"Newton did not converge: {its}")
            res = solver.pcg(pcg_tol, pcg_maxit)
            us, _ = solver.recover(res.lam)
            dU = solver.global_displacement(us)
            dU[~free] = 0.0
            a = 1.0
            while not factorizes(U + a * dU, tau):
                a *= 0.5
                if a < min_step:
                    raise RuntimeError("no step keeps the local tangents positive definite")
            U = U + a * dU
            rel = residual(U, tau)
            its.append((rel, res.iterations, a))
        log.append(its)
    return U, log


def monolithic_newton(prob, n_load_steps: int = 1, follower: bool = True, tol: float = 1e-10,
                      maxit: int = 30):
    """Load-stepped Newton on the assembled global system (the plain definition).

    tau = s / n_load_steps (Eq. loadStepping); per step, Newton on
    R(U) = f_int(U) - tau f_ext(U) over the non-Dirichlet DOFs with the
    assembled element tangents (Sec. 3.2, Eq. NewtonRecursion) and a sparse
    direct solve, until ||R|| <= tol ||tau f_ext|| or maxit iterations (the
    follower pressure's load stiffness is left out, as in the paper, so the
    convergence is linear rather than quadratic in follower mode).  Returns
    (U, history) with the relative residuals of every step.
    """
    import scipy.sparse.linalg as spla
    N = prob.n_nodes
    U = np.zeros(3 * N)
    free = np.ones(3 * N, bool)
    free[prob.dir_dof] = False
    idx = np.nonzero(free)[0]
    hist = []
    for s in range(1, n_load_steps + 1):
        tau = s / n_load_steps
        h = []
        for _ in range(maxit):
            Ke, fint = fem.element_matrices(prob, U.reshape(-1, 3))
            fext = fem.load_vector(prob, U.reshape(-1, 3), follower)
            R = fem.internal_force_global(prob, fint) - tau * fext
            h.append(np.linalg.norm(R[free]) / np.linalg.norm(tau * fext[free]))
            if h[-1] <= tol:
                break
            K = fem.assemble_global(prob, Ke)
            dU = np.zeros(3 * N)
            dU[idx] = spla.spsolve(K[idx][:, idx].tocsc(), -R[idx])
            U = U + dU
        hist.append(h)
    return U, hist
