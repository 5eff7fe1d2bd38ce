"""Python face of the C ABI: same calls as include/feti.h, numpy/torch marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


class FetiError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def library_path() -> str:
    return L.LIB_PATH


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None and a.size else None


_METHODS = {"classical": L.CLASSICAL, "af": L.ALL_FLOATING, "all_floating": L.ALL_FLOATING}
_PRECONDS = {"identity": L.PREC_IDENTITY, "lumped": L.PREC_LUMPED, "dirichlet": L.PREC_DIRICHLET}


class FetiSolver:
    """One problem on the current CUDA device (feti_create ... feti_destroy).

    prob: any object with the fields of a boundary-value problem: coords
    [N,3] float64, tets [E,4] int32, part [E] int32, n_parts, dir_dof,
    dir_val, press_tri, press_owner, pressure, trac_tri, trac_owner,
    traction, material (dict: kind, E, nu, c, k1, k2, kappa), fibres.
    plan_only: the host decomposition only, without a device
    (feti_create_plan); the size, map, fixing, coarse and factor getters
    answer, every solve raises.
    """

    def __init__(self, prob, method: str = "af", precond: str = "dirichlet", tol: float = 1e-10,
                 maxit: int = 1000, chunk: int = 16, stream=None, follower: bool = True,
                 n_load_steps: int = 10, newton_tol: float = 1e-8, newton_maxit: int = 25,
                 precision: str = "fp64", inner_tol: float = 0.0, max_outer: int = 0,
                 tensor_cores="auto", batched: bool = True, symmetric="auto", spin_timeout_ns: int = 0,
                 coarse: str = "auto", local_form: str = "auto", workspace_mb: int = 0,
                 plan_only: bool = False):
        self._lib = L.load()
        self._ctx = C.c_void_p()
        self._keep = []
        keep = self._keep.append
        coords = np.ascontiguousarray(prob.coords, dtype=np.float64); keep(coords)
        tets = np.ascontiguousarray(prob.tets, dtype=np.int32); keep(tets)
        part = np.ascontiguousarray(prob.part, dtype=np.int32); keep(part)
        self.n_nodes = coords.shape[0]
        self._n_tets = tets.shape[0]
        self._npe = tets.shape[1]
        mesh = L.FetiMesh(coords.shape[0], _ptr(coords, C.c_double), tets.shape[0], _ptr(tets, C.c_int32),
                          _ptr(part, C.c_int32), int(prob.n_parts), int(self._npe))
        m = prob.material
        fib = None
        if getattr(prob, "fibres", None) is not None:
            fib = np.ascontiguousarray(prob.fibres, dtype=np.float64); keep(fib)
        mat = L.FetiMaterial(int(m["kind"]), float(m["E"]), float(m["nu"]), float(m["c"]), float(m["k1"]),
                             float(m["k2"]), float(m["kappa"]), _ptr(fib, C.c_double))
        dd = np.ascontiguousarray(prob.dir_dof, dtype=np.int32); keep(dd)
        dv = np.ascontiguousarray(prob.dir_val, dtype=np.float64); keep(dv)
        fpn = 6 if tets.shape[1] == 10 else 3
        pt = np.ascontiguousarray(prob.press_tri, dtype=np.int32).reshape(-1, fpn); keep(pt)
        po = np.ascontiguousarray(prob.press_owner, dtype=np.int32); keep(po)
        tt = np.ascontiguousarray(prob.trac_tri, dtype=np.int32).reshape(-1, fpn); keep(tt)
        to = np.ascontiguousarray(prob.trac_owner, dtype=np.int32); keep(to)
        bc = L.FetiBC(dd.size, _ptr(dd, C.c_int32), _ptr(dv, C.c_double), pt.shape[0], _ptr(pt, C.c_int32),
                      _ptr(po, C.c_int32), float(prob.pressure), tt.shape[0], _ptr(tt, C.c_int32),
                      _ptr(to, C.c_int32), (C.c_double * 3)(*[float(v) for v in prob.traction]))
        prec = {"fp64": L.FP64, "mixed": L.MIXED, "mixed_f32factor": L.MIXED_F32FACTOR}[precision]
        opt = L.FetiOptions(_METHODS[method], _PRECONDS[precond], prec, float(tol), int(maxit), int(chunk),
                            int(bool(follower)), int(n_load_steps), float(newton_tol), int(newton_maxit),
                            float(inner_tol), int(max_outer),
                            {"auto": 0, False: 1, "off": 1, True: 2, "force": 2, "force_reg": 3,
                             "force_bulk": 4, "force_tma": 5, "force_ws3": 6, "force_ws2": 7,
                             "force_persist": 8, "force_persist_q3": 9, "force_persist_c3": 10}[tensor_cores],
                            int(not batched), {"auto": 0, "off": 1, False: 1, "force": 2, True: 2, "force_streamed": 3, "force_cta": 4}[symmetric],
                            int(spin_timeout_ns), {"auto": 0, "dense": 1, "sparse": 2}[coarse],
                            {"auto": 0, "explicit": 1, "implicit": 2}[local_form], int(workspace_mb))
        if plan_only:
            # host decomposition only (no device): the getters work, solves do not
            self._check(self._lib.feti_create_plan(C.byref(self._ctx), C.byref(mesh), C.byref(mat), C.byref(bc),
                                                   C.byref(opt)))
            return
        st = None if stream is None else C.c_void_p(int(stream))
        self._check(self._lib.feti_create(C.byref(self._ctx), C.byref(mesh), C.byref(mat), C.byref(bc),
                                          C.byref(opt), st))

    # -- helpers ---------------------------------------------------------------
    def _check(self, status: int):
        if status != L.FETI_OK:
            msg = self._lib.feti_last_error(self._ctx).decode() if self._ctx else ""
            raise FetiError(status, msg)

    def close(self):
        if self._ctx:
            self._lib.feti_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -----------------------------------------------------------------
    def sizes(self) -> dict:
        out = (C.c_int64 * 5)()
        self._check(self._lib.feti_get_sizes(self._ctx, out))
        return dict(zip(["n_lambda", "coarse_dim", "n_local", "n_boundary", "n_parts"], list(out)))

    def coarse_info(self) -> dict:
        """Form of the coarse problem: 'none', 'dense' or 'sparse', with the
        sparse factor's supernodes, assembly-tree height, factor entries,
        sweep tasks and set-up workspace (doubles)."""
        out = (C.c_int64 * 6)()
        self._check(self._lib.feti_get_coarse_info(self._ctx, out))
        v = list(out)
        return {"form": ["none", "dense", "sparse"][v[0]], "supernodes": v[1], "height": v[2],
                "factor_entries": v[3], "tasks": v[4], "workspace": v[5]}

    def factor_info(self) -> dict:
        """Storage of the local factorizations: groups eliminated one after
        another in the reused workspace, its elements, the elements of the
        whole dense workspace, the compact interior factor's elements (0 when
        the whole factor is kept) and bytes per element."""
        out = (C.c_int64 * 5)()
        self._check(self._lib.feti_get_factor_info(self._ctx, out))
        return dict(zip(["groups", "workspace", "full_workspace", "compact", "elem_bytes"], list(out)))

    def index_maps(self) -> dict:
        n = self.sizes()["n_lambda"]
        rs = np.empty((n, 2), np.int32)
        rl = np.empty((n, 2), np.int32)
        sg = np.empty((n, 2), np.int8)
        w = np.empty(n, np.float64)
        b = np.empty(n, np.float64)
        self._check(self._lib.feti_get_index_maps(self._ctx, rs.ctypes.data, rl.ctypes.data, sg.ctypes.data,
                                                  w.ctypes.data, b.ctypes.data))
        return {"row_sub": rs, "row_ldof": rl, "row_sign": sg, "weight": w, "b": b}

    def fixing(self) -> list:
        P = self.sizes()["n_parts"]
        ptr = np.empty(P + 1, np.int32)
        self._check(self._lib.feti_get_fixing(self._ctx, ptr.ctypes.data, None))
        ld = np.empty(max(int(ptr[-1]), 1), np.int32)
        self._check(self._lib.feti_get_fixing(self._ctx, None, ld.ctypes.data))
        return [ld[ptr[s]:ptr[s + 1]].copy() for s in range(P)]

    def elements(self, U=None, n_tets: int | None = None, out=None):
        """Element tangents [E,12,12] and internal forces [E,12] (hyperelastic) at U.

        Host arrays by default; with out = (Ke, fe) torch CUDA float64 tensors
        of those shapes, U must be a torch CUDA tensor (or None) and the
        results stay on the device."""
        E = n_tets if n_tets is not None else self._n_tets
        nd = 3 * self._npe
        if out is not None:
            Ke, fe = out
            up = None if U is None else C.c_void_p(U.data_ptr())
            self._check(self._lib.feti_elements(self._ctx, up, 1, C.c_void_p(Ke.data_ptr()),
                                                C.c_void_p(fe.data_ptr()), 1))
            return Ke, fe
        Ke = np.empty((E, nd, nd), np.float64)
        fe = np.empty((E, nd), np.float64)
        Uc = None if U is None else np.ascontiguousarray(U, dtype=np.float64).ravel()
        self._check(self._lib.feti_elements(self._ctx, None if Uc is None else Uc.ctypes.data, 0, Ke.ctypes.data,
                                            fe.ctypes.data, 0))
        return Ke, fe

    def prepare(self):
        self._check(self._lib.feti_prepare(self._ctx))

    def refinement(self) -> dict:
        """FP32-factor form: refinement corrections per K^+ application and the residual they reach."""
        n, r = C.c_int32(), C.c_double()
        self._check(self._lib.feti_get_refinement(self._ctx, C.byref(n), C.byref(r)))
        return {"steps": n.value, "residual": r.value}

    def set_spin_timeout(self, ns: int):
        """Main-loop wait budget (ns, literal; 100_000_000 = the default; 0 = give up at once) of the
        kernels with bounded mbarrier waits."""
        self._check(self._lib.feti_set_spin_timeout(self._ctx, int(ns)))

    def _report(self, rep: L.FetiReport) -> dict:
        return {k: getattr(rep, k) for k, _ in L.FetiReport._fields_}

    def solve(self, out=None, check: bool = True):
        """Linear solve.  out: torch CUDA tensor [N*3] float64 (device) or None (returns numpy)."""
        rep = L.FetiReport()
        if out is None:
            u = np.empty(3 * self.n_nodes, np.float64)
            st = self._lib.feti_solve(self._ctx, u.ctypes.data, 0, C.byref(rep))
        else:
            u = out
            st = self._lib.feti_solve(self._ctx, C.c_void_p(out.data_ptr()), 1, C.byref(rep))
        if check:
            self._check(st)
        return u, self._report(rep)

    def solve_multi(self, scales, out=None):
        """Block solve of len(scales) load cases f_k = scales[k] * f; returns [nrhs, 3N]."""
        sc = np.ascontiguousarray(scales, dtype=np.float64)
        rep = L.FetiReport()
        if out is None:
            u = np.empty((sc.size, 3 * self.n_nodes), np.float64)
            self._check(self._lib.feti_solve_multi(self._ctx, sc.ctypes.data, sc.size, u.ctypes.data, 0,
                                                   C.byref(rep)))
        else:
            u = out
            self._check(self._lib.feti_solve_multi(self._ctx, sc.ctypes.data, sc.size,
                                                   C.c_void_p(out.data_ptr()), 1, C.byref(rep)))
        return u, self._report(rep)

    def dual_apply_noalloc(self, v, q, z):
        """q = F v, z = M^-1 q without any device allocation (static scratch; see feti.h).

        Enqueued on the solver's stream; synchronise before reading q and z.
        """
        self._check(self._lib.feti_dual_apply_noalloc(self._ctx, C.c_void_p(v.data_ptr()), C.c_void_p(q.data_ptr()),
                                                      C.c_void_p(z.data_ptr())))

    def dual_apply_multi(self, v, q, z, nrhs: int, n_apply: int) -> float:
        ms = C.c_double()
        self._check(self._lib.feti_dual_apply_multi(self._ctx, C.c_void_p(v.data_ptr()), C.c_void_p(q.data_ptr()),
                                                    C.c_void_p(z.data_ptr()), int(nrhs), int(n_apply),
                                                    C.byref(ms)))
        return ms.value

    def solve_host(self, u_host):
        """feti_solve into a caller-owned host buffer (e.g. pinned torch tensor)."""
        rep = L.FetiReport()
        ptr = u_host.data_ptr() if hasattr(u_host, "data_ptr") else u_host.ctypes.data
        self._check(self._lib.feti_solve(self._ctx, C.c_void_p(ptr), 0, C.byref(rep)))
        return self._report(rep)

    def newton(self, out=None):
        rep = L.FetiReport()
        if out is None:
            u = np.empty(3 * self.n_nodes, np.float64)
            self._check(self._lib.feti_newton(self._ctx, u.ctypes.data, 0, C.byref(rep)))
        else:
            u = out
            self._check(self._lib.feti_newton(self._ctx, C.c_void_p(out.data_ptr()), 1, C.byref(rep)))
        return u, self._report(rep)

    def newton_steps(self, first: int, last: int, U_start=None):
        """Load steps first..last of the load-stepped Newton method from U_start (host array
        [3N] or None = unloaded); returns (U, report, pcg_per_step, newton_per_step)."""
        n = last - first + 1
        pcg = np.zeros(max(n, 1), np.int32)
        nwt = np.zeros(max(n, 1), np.int32)
        u = np.empty(3 * self.n_nodes, np.float64)
        u0 = None if U_start is None else np.ascontiguousarray(U_start, dtype=np.float64).ravel()
        rep = L.FetiReport()
        self._check(self._lib.feti_newton_steps(self._ctx, None if u0 is None else u0.ctypes.data, int(first),
                                                int(last), u.ctypes.data, 0, pcg.ctypes.data, nwt.ctypes.data,
                                                C.byref(rep)))
        return u, self._report(rep), pcg[:n], nwt[:n]

    def dual_apply(self, v, q, z, n_apply: int) -> float:
        """q = F v, z = M^-1 q, n_apply times on device tensors; returns ms per apply."""
        ms = C.c_double()
        self._check(self._lib.feti_dual_apply(self._ctx, C.c_void_p(v.data_ptr()), C.c_void_p(q.data_ptr()),
                                              C.c_void_p(z.data_ptr()), int(n_apply), C.byref(ms)))
        return ms.value

    def schedule(self) -> dict:
        out = np.zeros(12, np.int32)
        self._check(self._lib.feti_get_schedule(self._ctx, out.ctypes.data))
        o = [int(x) for x in out]
        return {"fp64_F": o[0:2], "fp64_M": o[2:4], "fp32_F": o[4:6], "fp32_M": o[6:8],
                "block_fp32_F": o[8:10], "block_fp32_M": o[10:12]}

    def element_stats(self) -> dict:
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.feti_element_stats(self._ctx, C.byref(a), C.byref(b), C.byref(c)))
        return {"elem_ms": a.value, "elem_bytes": b.value, "n_elements": int(c.value)}

    def kernel_stats(self) -> dict:
        a, b, c = C.c_double(), C.c_double(), C.c_double()
        self._check(self._lib.feti_kernel_stats(self._ctx, C.byref(a), C.byref(b), C.byref(c)))
        return {"gemv_ms": a.value, "gemv_bytes": b.value, "gemv_flops": c.value}


def checkpoint_write(path: str, U, step: int, n_load_steps: int, tau: float) -> None:
    """feti_checkpoint_write: the state (U, step, tau) of a load-stepped run (host-only call)."""
    lib = L.load()
    u = np.ascontiguousarray(U, dtype=np.float64).ravel()
    st = lib.feti_checkpoint_write(str(path).encode(), u.ctypes.data, u.size, int(step), int(n_load_steps),
                                   float(tau))
    if st != L.FETI_OK:
        raise FetiError(st, f"checkpoint_write {path}")


def checkpoint_read(path: str):
    """feti_checkpoint_read: returns (U, step, n_load_steps, tau); raises FetiError on a bad file."""
    lib = L.load()
    info = L.FetiCheckpointInfo()
    st = lib.feti_checkpoint_read(str(path).encode(), None, 0, C.byref(info))
    if st != L.FETI_OK:
        raise FetiError(st, f"checkpoint_read {path}")
    u = np.empty(info.n_dofs, np.float64)
    st = lib.feti_checkpoint_read(str(path).encode(), u.ctypes.data, u.size, C.byref(info))
    if st != L.FETI_OK:
        raise FetiError(st, f"checkpoint_read {path}")
    return u, info.step, info.n_load_steps, info.tau
