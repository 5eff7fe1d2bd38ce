"""The host decomposition of feti_create, run without a device (feti_create_plan).

feti_create_plan runs the argument checks and the whole host decomposition of
feti_create (local numbering, the fully redundant multiplier rows of Sec. 4.1,
kernels and fixing DOFs of Sec. 4.3 / 5.2, the dense local order, the coarse
ordering, the elimination workspace groups) and stops before the first device
call.  On the CPU, against the oracle and the mathematics:
  * the multiplier index maps, weights, b and the fixing DOFs equal the
    oracle's bit for bit, and the sizes its own (cube and tube, both methods);
  * the multiplier counts of the 64- and 1024-subdomain tubes follow the
    node-multiplicity rule (C(m, 2) rows per DOF, plus one row per subdomain
    copy of a Dirichlet DOF under all-floating FETI) and the coarse dimension
    is 6 per floating subdomain;
  * the workspace groups: the whole workspace is the sum of (n + n_b')^2 over
    the subdomains, a group never exceeds the budget unless it holds a single
    subdomain, the compact factor is (n_I + n_b') x n_I rounded up to 4 per
    subdomain, the implicit form keeps one group and no compact copy;
  * a host plan refuses every call that needs the device.
"""
import numpy as np
import pytest

from feti_inputs import mesh
from oracle import feti


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


CUBE = mesh.cube_problem(6, (2, 2, 2))
TUBE = mesh.cylinder_problem(4, 16, 8, (2, 8, 2))


def _plan(prob, method="af", precond="dirichlet", **kw):
    from paper_1508_02599_gb300 import FetiSolver
    return FetiSolver(prob, method=method, precond=precond, plan_only=True, **kw)


def _layout(sd):
    """(n, n_I, n_b', k) of an oracle subdomain in the dense local order:
    interior, boundary minus fixing, fixing."""
    n = len(sd.free)
    pos = {int(d): i for i, d in enumerate(sd.free)}
    fixpos = {pos[int(d)] for d in sd.fix}
    nbp = len(set(int(b) for b in sd.bnd) - fixpos)
    k = len(sd.fix)
    return n, n - nbp - k, nbp, k


@pytest.mark.parametrize("prob", [CUBE, TUBE], ids=lambda p: p.name)
@pytest.mark.parametrize("method", ["classical", "af"])
def test_plan_maps_and_fixing_equal_the_oracle(prob, method):
    o = feti.FetiOracle(prob, method)
    with _plan(prob, method) as s:
        m = s.index_maps()
        for key in ("row_sub", "row_ldof", "row_sign", "weight", "b"):
            assert np.array_equal(m[key], getattr(o.maps, key)), key
        for sd, f in zip(o.subs, s.fixing()):
            assert np.array_equal(np.asarray(sd.fix, np.int32), f)
        sz = s.sizes()
        assert sz["n_lambda"] == o.n_lambda and sz["coarse_dim"] == o.coarse_dim()
        assert sz["n_parts"] == prob.n_parts


def _rule_counts(prob):
    mult = np.zeros(prob.n_nodes, np.int64)
    for s in range(prob.n_parts):
        mult[np.unique(prob.tets[prob.part == s])] += 1
    is_dir = np.zeros(3 * prob.n_nodes, bool)
    is_dir[prob.dir_dof] = True
    m3 = np.repeat(mult, 3)
    return int((m3 * (m3 - 1) // 2).sum() + m3[is_dir].sum())


@pytest.mark.parametrize("name", ["cyl16", "jcyl32"])
def test_plan_sizes_of_the_benchmark_tubes(name):
    prob = mesh.config_problem(name)
    with _plan(prob) as s:
        sz = s.sizes()
        ci = s.coarse_info()
    assert sz["n_lambda"] == _rule_counts(prob)
    assert sz["coarse_dim"] == 6 * prob.n_parts
    assert ci["form"] == ("sparse" if 6 * prob.n_parts >= 1536 else "dense")


def test_plan_workspace_groups():
    o = feti.FetiOracle(TUBE, "af")
    lays = [_layout(sd) for sd in o.subs]
    full = sum((n + nbp) ** 2 for n, _, nbp, _ in lays)
    compact = sum((nI + nbp) * ((nI + 3) & ~3) for _, nI, nbp, _ in lays)
    biggest = max((n + nbp) ** 2 for n, _, nbp, _ in lays)
    with _plan(TUBE, workspace_mb=-1) as s:
        one = s.factor_info()
    assert one == {"groups": 1, "workspace": full, "full_workspace": full, "compact": compact, "elem_bytes": 8}
    with _plan(TUBE, workspace_mb=1) as s:
        g = s.factor_info()
    cap = (1 << 20) // 8
    assert g["full_workspace"] == full and g["compact"] == compact
    assert g["workspace"] <= max(cap, biggest)
    # every matrix here is below the budget, so each group holds at most cap
    # elements and there are at least full / cap groups
    assert g["groups"] >= -(-full // cap)
    with _plan(TUBE, precision="mixed_f32factor", workspace_mb=1) as s:
        g32 = s.factor_info()
    assert g32["elem_bytes"] == 4 and g32["groups"] < g["groups"]
    assert g32["workspace"] <= max((1 << 20) // 4, biggest)
    with _plan(TUBE, precision="fp64", local_form="implicit", workspace_mb=1) as s:
        imp = s.factor_info()
    assert imp["groups"] == 1 and imp["compact"] == 0 and imp["workspace"] == full


def test_plan_refuses_device_calls():
    from paper_1508_02599_gb300 import FetiError
    with _plan(CUBE) as s:
        with pytest.raises(FetiError) as ei:
            s.solve()
        assert ei.value.status == 12   # FETI_ERR_STATE
        with pytest.raises(FetiError):
            s.prepare()


def test_plan_checks_arguments():
    from paper_1508_02599_gb300 import FetiError
    with pytest.raises(FetiError) as ei:
        _plan(CUBE, workspace_mb=-2)
    assert ei.value.status == 1
    with pytest.raises(FetiError) as ei:
        _plan(CUBE, precision="mixed", local_form="implicit")
    assert ei.value.status == 1
