"""The zero structure the GPU factorization skips, checked on subdomain matrices.

The dense local factorization works in the order [interior | boundary minus
fixing | fixing | augmentation] and updates, per 32-column block, only the
rows that block can reach:
  * interior columns: a row is zero left of the first interior column it
    couples to through an element, and Cholesky fill stays inside that
    envelope (boundary DOFs are ordered by that first column);
  * boundary columns of the identity-augmented matrix [[K, 0], [E^T, 0]]:
    augmentation row n + a is zero left of column nI + a until that column is
    eliminated.
Both claims are checked here on the local stiffness matrices of a tube
subdomain built by the oracle's element routine, with a plain blocked
elimination (all rows) and the restricted one (reachable rows only), and on
the complement: the blocked result equals the Schur complement inverse.
"""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import fem
from oracle.feti import pivoted_rows, rigid_body_modes

NB = 32


def _subdomain(prob, s):
    """Dense order, envelope table and the local matrix of subdomain s (all-floating)."""
    P = prob.n_parts
    nodes = [np.unique(prob.tets[prob.part == t]) for t in range(P)]
    mult = np.zeros(prob.n_nodes, int)
    for t in range(P):
        mult[nodes[t]] += 1
    isd = np.zeros(3 * prob.n_nodes, bool)
    isd[prob.dir_dof] = True
    nd = nodes[s]
    loc = {g: i for i, g in enumerate(nd)}
    isb = np.repeat((mult[nd] > 1) | isd.reshape(-1, 3).any(1)[nd], 3)
    interior = [d for d in range(3 * len(nd)) if not isb[d]]
    bl = [d for d in range(3 * len(nd)) if isb[d]]
    R = rigid_body_modes(prob.coords[nd] - prob.coords[nd].mean(0))
    fix = [bl[i] for i in pivoted_rows(R[bl], 6)]
    nI = len(interior)
    own = np.full(len(nd), nI)
    for i, d in enumerate(interior):
        own[d // 3] = min(own[d // 3], i)
    first_node = np.full(len(nd), nI)
    elems = [[loc[g] for g in t] for t in prob.tets[prob.part == s]]
    for t in elems:
        m = min(own[a] for a in t)
        for a in t:
            first_node[a] = min(first_node[a], m)
    first = np.repeat(first_node, 3)
    bsort = sorted([d for d in bl if d not in fix], key=lambda d: first[d])
    order = interior + bsort + fix
    Ke = fem.element_matrices(prob)
    Ke = Ke[0] if isinstance(Ke, tuple) else Ke
    K = np.zeros((3 * len(nd),) * 2)
    for e in np.nonzero(prob.part == s)[0]:
        idx = np.array([3 * loc[g] + c for g in prob.tets[e] for c in range(3)])
        K[np.ix_(idx, idx)] += Ke[e]
    return K[np.ix_(order, order)], nI, len(bsort), first[order]


def _eliminate(A, c0, c1, rows_of):
    """Right-looking blocked Cholesky of columns [c0, c1) of the lower triangle of A."""
    for t, kb in enumerate(range(c0, c1, NB)):
        nk = min(NB, c1 - kb)
        D = np.tril(A[kb:kb + nk, kb:kb + nk])
        L = np.linalg.cholesky(D + np.tril(D, -1).T)
        A[kb:kb + nk, kb:kb + nk] = L
        rows = rows_of(t, kb + nk)
        cols = np.arange(kb, kb + nk)
        X = A[np.ix_(rows, cols)].copy()
        for j in range(nk):                      # row-wise forward substitution, fixed order
            v = X[:, j].copy()
            for l in range(j):
                v -= X[:, l] * L[j, l]
            X[:, j] = v / L[j, j]
        A[np.ix_(rows, cols)] = X
        U = np.zeros((len(rows), len(rows)))
        for l in range(nk):                      # rank-nk update, fixed order per entry
            U += np.outer(X[:, l], X[:, l])
        A[np.ix_(rows, rows)] -= np.tril(U)
    return A


@pytest.mark.parametrize("s", [0, 9])
def test_restricted_elimination_is_bit_identical(s):
    prob = mesh.cylinder_problem(6, 24, 12, (2, 4, 2))
    K, nI, nbp, first = _subdomain(prob, s)
    n = K.shape[0]
    k = n - nI - nbp
    ld = n + nbp
    # the envelope claim itself: the factor of K_rr is exactly zero left of it
    Lrr = np.linalg.cholesky(K[:nI + nbp, :nI + nbp])
    for r in range(nI, nI + nbp):
        assert not np.any(Lrr[r, :min(first[r], nI)])
    assert list(first[nI:nI + nbp]) == sorted(first[nI:nI + nbp])
    # per-step reachable rows of the interior elimination, as the host tabulates them
    last = np.full(nI + 1, -1)
    for r in range(nI):
        last[first[r] + 1] = max(last[first[r] + 1], r)
    last = np.maximum.accumulate(last)
    bfirst = first[nI:nI + nbp]

    def reach0(t, r0):
        eI = max(r0, last[r0] + 1)
        nb = int(np.searchsorted(bfirst, r0, "left"))
        return np.concatenate([np.arange(r0, eI), np.arange(nI, nI + nb), np.arange(nI + nbp, n)])

    def reach1(t, r0):
        return np.arange(r0, min(ld, n + r0 - nI))

    A0 = np.zeros((ld, ld))
    A0[:n, :n] = np.tril(K)
    A0[n + np.arange(nbp), nI + np.arange(nbp)] = 1.0
    full = A0.copy()
    _eliminate(full, 0, nI, lambda t, r0: np.arange(r0, n))
    _eliminate(full, nI, nI + nbp, lambda t, r0: np.arange(r0, ld))
    part = A0.copy()
    _eliminate(part, 0, nI, reach0)
    _eliminate(part, nI, nI + nbp, reach1)
    assert np.array_equal(np.tril(full), np.tril(part))
    # and the augmentation block is minus the inverse of the Schur complement on b'
    S = K[nI:, nI:] - K[nI:, :nI] @ np.linalg.solve(K[:nI, :nI], K[:nI, nI:])
    F = -np.tril(part[n:, n:])
    F = F + np.tril(F, -1).T
    Fi = np.linalg.inv(S[:nbp, :nbp])
    assert np.abs(F - Fi).max() <= 1e-10 * np.abs(Fi).max()
    assert k == 6
