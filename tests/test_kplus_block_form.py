"""The block form of K_rr^-1 that the K^+ sweeps compute, emulated on the CPU.

The local solves keep only the interior columns of the Cholesky factor
L = [[L_II, 0], [L_bI, L_bb]] of K_rr (interior DOFs first) plus the explicit
F_i = S_i[b',b']^-1 = (L_bb L_bb^T)^-1 (Sec. 4.4), and apply
    y_I = L_II^-1 g_I,  z_b = g_b - L_bI y_I,  x_b = F_i z_b,
    x_I = L_II^-T (y_I - L_bI^T x_b).
The GPU kernels run the two triangular solves right-looking over 32-column
blocks (solve a diagonal block, then update the rows below it / the columns
left of it) on the compact layout: rows [0, n_I + n_b') x columns [0, n_I),
row stride n_I rounded up to 4, zero above the diagonal.  This test runs the
same steps in numpy, in the same block order, and checks the result against a
dense solve of K_rr x = g, for interior sizes below, at and across multiples
of 32 (and no interior at all).
"""
import numpy as np
import pytest


def _compact(Lf, nI, nbp):
    ld = (nI + 3) & ~3
    A = np.zeros((nI + nbp, ld))
    for r in range(nI + nbp):
        cmax = r if r < nI else nI - 1
        A[r, :cmax + 1] = Lf[r, :cmax + 1]
    return A


def _fwd_interior(A, nI, g):
    ys = g[:nI].copy()
    for I0 in range(0, nI, 32):
        nb = min(32, nI - I0)
        D = np.tril(A[I0:I0 + nb, I0:I0 + nb])
        b = ys[I0:I0 + nb].copy()
        x = np.zeros(nb)
        for c in range(nb):           # warp 0: one column per step
            x[c] = b[c] / D[c, c]
            b[c + 1:] -= D[c + 1:, c] * x[c]
        ys[I0:I0 + nb] = x
        if I0 + 32 < nI:              # rows below, with this block's 32 values
            ys[I0 + 32:] -= A[I0 + 32:nI, I0:I0 + 32] @ x
    return ys


def _bwd_interior(A, nI, t):
    ys = t.copy()
    last = ((nI - 1) // 32) * 32 if nI > 0 else -32
    for I0 in range(last, -1, -32):
        nb = min(32, nI - I0)
        D = np.tril(A[I0:I0 + nb, I0:I0 + nb])
        b = ys[I0:I0 + nb].copy()
        x = np.zeros(nb)
        for c in range(nb - 1, -1, -1):
            x[c] = b[c] / D[c, c]
            b[:c] -= D[c, :c] * x[c]
        ys[I0:I0 + nb] = x
        if I0 > 0:                    # columns left of the block
            ys[:I0] -= A[I0:I0 + nb, :I0].T @ x
    return ys


@pytest.mark.parametrize("nI,nbp", [(0, 17), (5, 40), (32, 32), (33, 9), (70, 50), (96, 31), (131, 77)])
def test_block_form_equals_dense_solve(nI, nbp):
    rng = np.random.default_rng(nI * 1000 + nbp)
    n = nI + nbp
    M = rng.normal(size=(n, n))
    K = M @ M.T + n * np.eye(n)
    Lf = np.linalg.cholesky(K)
    A = _compact(Lf, nI, nbp)
    # F_i from the Schur complement of the interior block (not from L_bb)
    S = K[nI:, nI:] - K[nI:, :nI] @ np.linalg.solve(K[:nI, :nI], K[:nI, nI:]) if nI else K.copy()
    F = np.linalg.inv(S)
    g = rng.normal(size=n)
    yI = _fwd_interior(A, nI, g)
    zb = g[nI:] - A[nI:, :nI] @ yI
    xb = F @ zb
    tI = yI - A[nI:, :nI].T @ xb
    xI = _bwd_interior(A, nI, tI)
    x = np.concatenate([xI, xb])
    ref = np.linalg.solve(K, g)
    assert np.abs(x - ref).max() <= 1e-12 * np.abs(ref).max()


def test_compact_layout_keeps_only_what_the_sweeps_read():
    rng = np.random.default_rng(7)
    nI, nbp = 45, 20
    n = nI + nbp
    M = rng.normal(size=(n, n))
    Lf = np.linalg.cholesky(M @ M.T + n * np.eye(n))
    A = _compact(Lf, nI, nbp)
    assert A.shape == (n, 48)                       # stride: n_I rounded up to 4
    assert np.array_equal(A[:nI, :nI], np.tril(Lf[:nI, :nI]))
    assert np.array_equal(A[nI:, :nI], Lf[nI:, :nI])
    assert not A[:, nI:].any()                      # padding


@pytest.mark.parametrize("method", ["af", "classical"])
def test_block_form_equals_oracle_kplus_on_tube_subdomains(method):
    """On the subdomains of a small tube (with their fixing DOFs): the dense
    local order [interior | boundary minus fixing], the compact interior
    factor and F_i = S_i[b',b']^-1 give the oracle's generalized inverse
    K_i^+ g (Sec. 4.3, fixing-DOF inverse zero on the fixing DOFs), and the
    boundary block of K_i^+ is F_i itself."""
    from feti_inputs import mesh
    from oracle import feti
    prob = mesh.cylinder_problem(4, 16, 8, (2, 4, 2))
    o = feti.FetiOracle(prob, feti.ALL_FLOATING if method == "af" else feti.CLASSICAL, "dirichlet")
    o.assemble()
    o.factorize()
    rng = np.random.default_rng(11)
    for sd in o.subs[:6]:
        n = sd.free.size
        fixpos = np.searchsorted(sd.free, sd.fix)
        bp = np.setdiff1d(sd.bnd, fixpos)                         # boundary minus fixing
        inner = np.setdiff1d(np.arange(n), np.union1d(sd.bnd, fixpos))
        order = np.concatenate([inner, bp])
        nI, nbp = inner.size, bp.size
        Krr = sd.K[np.ix_(order, order)]
        Lf = np.linalg.cholesky(Krr)
        A = _compact(Lf, nI, nbp)
        S = Krr[nI:, nI:] - (Krr[nI:, :nI] @ np.linalg.solve(Krr[:nI, :nI], Krr[:nI, nI:]) if nI else 0.0)
        F = np.linalg.inv(S)
        g = rng.normal(size=n)
        yI = _fwd_interior(A, nI, g[order])
        zb = g[bp] - A[nI:, :nI] @ yI
        xb = F @ zb
        xI = _bwd_interior(A, nI, yI - A[nI:, :nI].T @ xb)
        x = np.zeros(n)
        x[order] = np.concatenate([xI, xb])
        ref = o.kplus(sd, g)
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
        assert not x[fixpos].any()
        # the boundary block of the generalized inverse is F_i
        E = np.zeros((n, nbp))
        E[bp, np.arange(nbp)] = 1.0
        KpB = np.column_stack([o.kplus(sd, E[:, j]) for j in range(nbp)])[bp]
        assert np.abs(KpB - F).max() <= 1e-10 * np.abs(F).max()
