"""Mixed precision (FP32 / BF16 operator values, FP32 inner PCG, FP64 dots, alpha/beta and outer
refinement) against the FP64 oracle.

Bar: every solve reaches the FP64 stopping rule (true residual <= rtol, or the FP64 floor), and
its error against the oracle's FP64 solution stays within the conditioning bound
    |x_mixed - x_oracle| / |x_oracle| <= kappa * (rho_mixed + rho_oracle),
kappa estimated from the Lanczos tridiagonal of an unpreconditioned oracle CG run (its extreme
Ritz values lie inside the spectrum, so the estimate is from below; a factor 4 covers that).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import theta_basin  # noqa: E402
from oracle import fem, pcg as opcg, step as ostep  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, ocean_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu

import paper_1207_0486_gb300 as pm  # noqa: E402

_cache = {}


def case(name):
    if name not in _cache:
        b = {"box16": lambda: theta_basin(box_basin()), "small": small_basin,
             "ocean48": lambda: ocean_basin(nx=48, ny=40, nz=9, dx=1e5),
             "ocean32": lambda: ocean_basin(nx=40, ny=36, nz=32, dx=1e4)}[name]()
        _cache[name] = (b, pm.assemble_operator(b), fem.assemble(b))
    return _cache[name]


def oracle_matrix(ops, which):
    if which == pm.OP_PRESSURE:
        return ops.K_I
    if which in (pm.OP_VEL1_U1, pm.OP_VEL1_U2, pm.OP_VEL1_U3):
        return ops.A_u(which - pm.OP_VEL1_U1, bdf1=True)
    return ops.A_u(which - pm.OP_VEL_U1, bdf1=False)


def lanczos_kappa(A, b, m=None):
    """kappa estimate from the Ritz values of an unpreconditioned CG run."""
    if m is not None:
        b = b - b.sum() / m.sum() * m
        P = (lambda r: r - (m @ r) / m.sum())
    else:
        P = None
    res = opcg.pcg(A, b, rtol=1e-12, precond=P, record=True, max_iter=6000, max_restarts=0)
    al, be = np.array(res.alphas), np.array(res.betas)
    k = len(al)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
    ev = np.linalg.eigvalsh(T)
    return ev.max() / ev.min()


@pytest.mark.parametrize("name", ["box16", "small", "ocean48"])
@pytest.mark.parametrize("which", [pm.OP_VEL_U1, pm.OP_VEL1_U3, pm.OP_PRESSURE])
@pytest.mark.parametrize("precision", [pm.FP32_REFINE, pm.BF16_REFINE])
@pytest.mark.parametrize("prec", [pm.PREC_JACOBI, pm.PREC_LINE, pm.PREC_IC0])
def test_mixed_solve_matches_fp64_oracle(name, which, precision, prec):
    b, op, ops = case(name)
    rhs = random_vector(op.n, 300 + which)
    if which != pm.OP_PRESSURE:
        c = which - (pm.OP_VEL1_U1 if which >= pm.OP_VEL1_U1 else pm.OP_VEL_U1)
        rhs[ops.mesh.dirichlet[c]] = 0.0
    rtol = 1e-8
    bd = torch.from_numpy(rhs).cuda()
    x = torch.zeros_like(bd)
    st = op.solve(which, bd, x, pm.Options(rtol=rtol, prec=prec, precision=precision, max_iter=200000))
    assert st.status == pm.PM_OK
    assert st.rel_residual_true <= max(rtol, st.rel_residual_floor)
    A = oracle_matrix(ops, which)
    if which == pm.OP_PRESSURE:
        ref = opcg.pressure_solve(A, ops.m, rhs, rtol=1e-12 if not name.startswith("ocean") else 2e-9)
    else:
        ref = opcg.pcg(A, rhs, rtol=1e-13, precond=opcg.jacobi_preconditioner(A))
    xg = x.cpu().numpy()
    err = np.linalg.norm(xg - ref.x) / np.linalg.norm(ref.x)
    kappa = lanczos_kappa(A, rhs, ops.m if which == pm.OP_PRESSURE else None)
    bound = 4 * kappa * (max(st.rel_residual_true, st.rel_residual_floor) + ref.rel_res_true)
    assert err <= max(bound, 1e-12), (err, kappa, bound)


@pytest.mark.parametrize("which", [pm.OP_VEL_U1, pm.OP_PRESSURE])
@pytest.mark.parametrize("precision", [pm.FP32_REFINE, pm.BF16_REFINE])
def test_mixed_line_solve_on_32_level_columns(which, precision):
    """32-level columns take the warp-task FP32 line kernel."""
    test_mixed_solve_matches_fp64_oracle("ocean32", which, precision, pm.PREC_LINE)


@pytest.mark.parametrize("precision", [pm.FP32_REFINE, pm.BF16_REFINE])
def test_mixed_projection_step_per_field(precision):
    """Three projection steps on the 16x16x8 box in mixed precision vs the FP64 oracle; the
    per-field relative errors (u, v, w, p) are printed and bounded."""
    b, op, ops = case("box16")
    st = pm.State(op)
    t1 = torch.from_numpy(op.column_field(b.theta[0])).cuda()
    t2 = torch.from_numpy(op.column_field(b.theta[1])).cuda()
    vel = pm.Options(rtol=1e-8, prec=pm.PREC_IC0, precision=precision)
    pres = pm.Options(rtol=1e-8, prec=pm.PREC_LINE, precision=precision)
    ost = ostep.initial_state(ops.n)
    oopt = ostep.StepOptions(vel_rtol=1e-12, pres_rtol=1e-12, pres_prec="line")
    for k in range(3):
        stats = pm.project_step(op, st, t1, t2, vel, pres)
        ostep.project_step(ops, ost, oopt)
        got = [t.cpu().numpy() for t in st.get()]
        errs = {}
        for nm, g, o in zip(("u", "v", "w", "p"), got, (ost.u[0], ost.u[1], ost.u[2], ost.p)):
            scale = np.abs(o).max()
            errs[nm] = 0.0 if scale == 0 else float(np.abs(g - o).max() / scale)
        print(f"precision={precision} step={k} per-field max rel error {errs} "
              f"iters={[s.iters for s in stats[:4]]} outer={[s.outer_iters for s in stats[:4]]}")
        # an FP64 oracle step at rtol 1e-8 itself differs from the 1e-12 one by <= 6e-9 per field
        for nm, e in errs.items():
            assert e <= 1e-6, (k, nm, e)
