"""Tracing and checking on the GPU: the per-solve JSON log has one line per solved system with
the solve's own figures; the checked build (device index checks) solves parity cases with no bad
index and matches the oracle; a non-finite right-hand side ends a solve with PM_BREAKDOWN, not a
hang or a fault."""
import json

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1207_0486_gb300 as pm  # noqa: E402
from paper_1207_0486_gb300 import api, build  # noqa: E402
from oracle import fem, pcg as opcg  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu


def _lines(path):
    return [json.loads(s) for s in open(path).read().splitlines()]


def test_solve_log_has_one_line_per_system(tmp_path):
    op = pm.assemble_operator(box_basin())
    log = tmp_path / "solves.jsonl"
    pm.set_log(str(log), hbm_peak_gbs=6800.0)
    try:
        b = torch.from_numpy(random_vector(op.n, 3)).cuda()
        x = torch.zeros_like(b)
        st = op.solve(pm.OP_PRESSURE, b, x, pm.Options(rtol=1e-10, prec=pm.PREC_LINE))
        bt = pm.Batch([op, op], [pm.OP_VEL_U1, pm.OP_MASS], pm.Options(rtol=1e-10), prec=[pm.PREC_IC0, pm.PREC_IC0])
        bst = bt.solve([b, b], [torch.zeros_like(b), torch.zeros_like(b)])
        bt.close()
    finally:
        pm.set_log(None)
    rows = _lines(log)
    assert [r["event"] for r in rows] == ["pcg_solve", "batch_solve", "batch_solve"]
    assert rows[0]["system"] == "pressure" and rows[0]["preconditioner"] == "line"
    assert rows[0]["iters"] == st.iters and rows[0]["status"] == "ok" and rows[0]["rows"] == op.n
    assert rows[0]["rel_residual_true"] == pytest.approx(st.rel_residual_true, rel=1e-5)
    assert rows[0]["pct_of_peak"] == pytest.approx(100 * rows[0]["gbs"] / 6800.0, rel=1e-4)
    assert [r["system"] for r in rows[1:]] == ["velocity_u1", "mass"]
    assert [r["iters"] for r in rows[1:]] == [s.iters for s in bst]
    assert all(r["preconditioner"] == "ic0" for r in rows[1:])
    op.close()


@pytest.fixture
def checked():
    path = build.build(checked=True)
    prev = api.select_library(path)
    try:
        assert pm.build_flags() == pm.PM_BUILD_CHECKED
        yield
    finally:
        api.select_library(prev)


@pytest.mark.parametrize("which,prec", [(pm.OP_VEL_U1, pm.PREC_IC0), (pm.OP_PRESSURE, pm.PREC_LINE),
                                        (pm.OP_MASS, pm.PREC_JACOBI)])
def test_checked_build_solves_clean_and_matches_the_oracle(checked, which, prec):
    b = small_basin()
    op = pm.assemble_operator(b)
    ops = fem.assemble(b)
    rhs = random_vector(op.n, 11 + which)
    if which == pm.OP_VEL_U1:
        rhs[ops.mesh.dirichlet[0]] = 0.0
    x = torch.zeros(op.n, dtype=torch.float64, device="cuda")
    st = op.solve(which, torch.from_numpy(rhs).cuda(), x, pm.Options(rtol=1e-12, prec=prec, max_restarts=5),
                  allow_not_converged=True)
    assert st.status in (pm.PM_OK, pm.PM_NOT_CONVERGED)   # PM_EBOUNDS would raise
    A = {pm.OP_VEL_U1: lambda: ops.A_u(0), pm.OP_PRESSURE: lambda: ops.K_I, pm.OP_MASS: lambda: ops.M}[which]()
    if which == pm.OP_PRESSURE:
        ref = opcg.pressure_solve(A, ops.m, rhs, rtol=1e-12).x
    else:
        ref = opcg.pcg(A, rhs, rtol=1e-13, precond=opcg.jacobi_preconditioner(A)).x
    assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-9 * np.linalg.norm(ref)
    # batched and stepped paths in the checked build too
    bt = pm.Batch([op], [which], pm.Options(rtol=1e-10, prec=prec))
    xb = torch.zeros_like(x)
    bt.solve([torch.from_numpy(rhs).cuda()], [xb])
    bt.close()
    assert np.linalg.norm(xb.cpu().numpy() - ref) <= 1e-8 * np.linalg.norm(ref)
    op.close()


@pytest.mark.parametrize("kernel", [pm.KERNEL_STREAM, pm.KERNEL_RESIDENT])
def test_non_finite_right_hand_side_is_a_breakdown(kernel):
    op = pm.assemble_operator(box_basin())
    rhs = random_vector(op.n, 5)
    rhs[17] = np.nan
    b = torch.from_numpy(rhs).cuda()
    x = torch.zeros_like(b)
    with pytest.raises(pm.PMError) as ei:
        op.solve(pm.OP_VEL_U2, b, x, pm.Options(rtol=1e-10, prec=pm.PREC_IC0, kernel=kernel))
    assert ei.value.status == pm.PM_BREAKDOWN
    bt = pm.Batch([op], [pm.OP_PRESSURE], pm.Options(rtol=1e-10))
    with pytest.raises(pm.PMError) as ei:
        bt.solve([b], [torch.zeros_like(b)])
    assert ei.value.status == pm.PM_BREAKDOWN
    bt.close()
    # the context is still usable
    b2 = torch.from_numpy(random_vector(op.n, 6)).cuda()
    assert op.solve(pm.OP_PRESSURE, b2, torch.zeros_like(b2), pm.Options(rtol=1e-10)).status == pm.PM_OK
    op.close()
