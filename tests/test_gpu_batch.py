"""Batched persistent PCG: every system of a batch matches its solo solve and the oracle, results
do not depend on what else is in the batch, and a bounded grid wait reports PM_TIMEOUT."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gpu_util import theta_basin  # noqa: E402
from oracle import fem, pcg as opcg  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, ocean_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu

import paper_1207_0486_gb300 as pm  # noqa: E402

_cache = {}


def case(name):
    if name not in _cache:
        b = {"box16": lambda: theta_basin(box_basin()), "small": small_basin,
             "box24": lambda: box_basin(nh=24, nz=12),
             "ocean48": lambda: ocean_basin(nx=48, ny=40, nz=9, dx=1e5)}[name]()
        _cache[name] = (b, pm.assemble_operator(b), fem.assemble(b))
    return _cache[name]


def rhs_for(name, which, seed):
    b, op, ops = case(name)
    r = random_vector(op.n, seed)
    if which not in (pm.OP_PRESSURE, pm.OP_MASS):
        c = which - (pm.OP_VEL1_U1 if which >= pm.OP_VEL1_U1 else pm.OP_VEL_U1)
        r[ops.mesh.dirichlet[c]] = 0.0
    return r


ENTRIES = [("box16", pm.OP_VEL_U1), ("box16", pm.OP_VEL_U2), ("box16", pm.OP_VEL_U3), ("box16", pm.OP_PRESSURE),
           ("small", pm.OP_VEL1_U1), ("small", pm.OP_PRESSURE), ("box24", pm.OP_VEL_U3), ("box24", pm.OP_PRESSURE)]
# consistent-mass systems (the velocity correction with M instead of its lumped diagonal) and a
# velocity system of the ocean basin (land columns, Dirichlet coasts)
MASS_ENTRIES = [("box16", pm.OP_MASS), ("box24", pm.OP_MASS), ("ocean48", pm.OP_MASS), ("ocean48", pm.OP_VEL_U2)]


def oracle_matrix(ops, which):
    if which == pm.OP_PRESSURE:
        return ops.K_I
    if which == pm.OP_MASS:
        return ops.M
    if which >= pm.OP_VEL1_U1:
        return ops.A_u(which - pm.OP_VEL1_U1, bdf1=True)
    return ops.A_u(which - pm.OP_VEL_U1, bdf1=False)


def oracle_precond(ops, A, prec):
    if prec == pm.PREC_LINE:
        return opcg.line_preconditioner(A, ops.mesh.nz)
    if prec == pm.PREC_IC0:
        return opcg.ic0_preconditioner(A, ops.mesh.colour)[0]
    return opcg.jacobi_preconditioner(A)


def oracle_solve(ops, which, rhs, prec, rtol):
    A = oracle_matrix(ops, which)
    P = oracle_precond(ops, A, prec)
    if which == pm.OP_PRESSURE:
        return opcg.pressure_solve(A, ops.m, rhs, rtol=rtol, precond=P)
    return opcg.pcg(A, rhs, rtol=rtol, precond=P)


def seed_of(entry):
    return 40 + (ENTRIES + MASS_ENTRIES).index(entry)


def run_batch(entries, prec, precision=pm.FP64, rtol=1e-12, autotune=False, per_entry=None):
    opsl = [case(nm)[1] for nm, _ in entries]
    bs = [torch.from_numpy(rhs_for(nm, w, seed_of((nm, w)))).cuda() for nm, w in entries]
    xs = [torch.zeros_like(b) for b in bs]
    batch = pm.Batch(opsl, [w for _, w in entries], pm.Options(rtol=rtol, prec=prec, precision=precision,
                                                               max_iter=200000), autotune=autotune,
                     prec=per_entry)
    stats = batch.solve(bs, xs)
    info = batch.info()
    batch.close()
    return [x.cpu().numpy() for x in xs], stats, info


@pytest.mark.parametrize("prec", [pm.PREC_JACOBI, pm.PREC_LINE, pm.PREC_IC0])
def test_batch_matches_solo_and_oracle(prec):
    entries = ENTRIES + (MASS_ENTRIES if prec == pm.PREC_IC0 else [])
    xs, stats, _ = run_batch(entries, prec)
    for (nm, w), x, st in zip(entries, xs, stats):
        b, op, ops = case(nm)
        rhs = rhs_for(nm, w, seed_of((nm, w)))
        assert st.status == pm.PM_OK, (nm, w)
        assert st.rel_residual_true <= max(1e-12, st.rel_residual_floor)
        # solo solve through the regular entry point
        xd = torch.zeros(op.n, dtype=torch.float64, device="cuda")
        solo = op.solve(w, torch.from_numpy(rhs).cuda(), xd, pm.Options(rtol=1e-12, prec=prec, max_restarts=5),
                        allow_not_converged=True)
        xs_solo = xd.cpu().numpy()
        assert np.linalg.norm(x - xs_solo) <= 1e-9 * np.linalg.norm(xs_solo), (nm, w)
        assert abs(st.first_pass_iters - solo.first_pass_iters) <= max(2, 0.02 * solo.first_pass_iters)
        # the oracle: the same preconditioned recurrence (first-pass iteration count at the same
        # rtol; a different preconditioner still converges, but in a different number of steps)
        # and its solution at a tight tolerance
        same = oracle_solve(ops, w, rhs, prec, 1e-12)
        assert abs(st.first_pass_iters - same.first_pass_iters) <= max(2, 0.02 * same.first_pass_iters), \
            (nm, w, st.first_pass_iters, same.first_pass_iters)
        ref = same if w == pm.OP_PRESSURE else oracle_solve(ops, w, rhs, prec, 1e-13)
        assert np.linalg.norm(x - ref.x) <= 1e-9 * np.linalg.norm(ref.x), (nm, w)


@pytest.mark.parametrize("prec", [pm.PREC_LINE, pm.PREC_IC0])
def test_batch_result_does_not_depend_on_the_mix(prec):
    """A system alone and inside a batch with others gives bit-identical iterates (per-system
    reductions run over that system's tiles in a fixed order; every IC0 row is computed once, after
    the rows it reads, whichever block owns its tile)."""
    alone, st_a, _ = run_batch([ENTRIES[3]], prec, rtol=1e-10)
    mixed, st_m, _ = run_batch(ENTRIES, prec, rtol=1e-10)
    assert np.array_equal(alone[0], mixed[3])
    assert st_a[0].iters == st_m[3].iters


@pytest.mark.parametrize("precision", [pm.FP32_REFINE, pm.BF16_REFINE])
@pytest.mark.parametrize("prec", [pm.PREC_LINE, pm.PREC_IC0])
def test_batch_mixed_precision(prec, precision):
    entries = ENTRIES + (MASS_ENTRIES if prec == pm.PREC_IC0 else [])
    xs, stats, _ = run_batch(entries, prec, precision=precision, rtol=1e-8)
    for (nm, w), x, st in zip(entries, xs, stats):
        b, op, ops = case(nm)
        assert st.status == pm.PM_OK
        assert st.rel_residual_true <= max(1e-8, st.rel_residual_floor)
        rhs = rhs_for(nm, w, seed_of((nm, w)))
        ref = oracle_solve(ops, w, rhs, pm.PREC_JACOBI, 1e-12 if w == pm.OP_PRESSURE else 1e-13)
        assert np.linalg.norm(x - ref.x) <= 1e-5 * np.linalg.norm(ref.x), (nm, w)


def paper_precs(entries):
    """The paper's choice per system: IC0 for the velocity and mass systems; the pressure here
    takes the vertical-line preconditioner."""
    return [pm.PREC_LINE if w == pm.OP_PRESSURE else pm.PREC_IC0 for _, w in entries]


@pytest.mark.parametrize("precision", [pm.FP64, pm.FP32_REFINE])
def test_batch_with_a_preconditioner_per_system(precision):
    """One batch holding IC0 velocity and mass systems next to line-preconditioned pressure
    systems: each system gives the bits it gives in a batch of its own preconditioner, and
    matches its solo solve."""
    entries = ENTRIES + MASS_ENTRIES
    precs = paper_precs(entries)
    rtol = 1e-12 if precision == pm.FP64 else 1e-8
    xs, stats, _ = run_batch(entries, pm.PREC_JACOBI, precision=precision, rtol=rtol, per_entry=precs)
    for p in (pm.PREC_IC0, pm.PREC_LINE):
        sub = [e for e, q in zip(entries, precs) if q == p]
        xs_p, st_p, _ = run_batch(sub, p, precision=precision, rtol=rtol)
        for e, x, st in zip(sub, xs_p, st_p):
            i = entries.index(e)
            assert np.array_equal(xs[i], x), e
            assert stats[i].iters == st.iters, e
    for (nm, w), x, st, p in zip(entries, xs, stats, precs):
        b, op, ops = case(nm)
        assert st.status == pm.PM_OK, (nm, w)
        if precision == pm.FP64:
            rhs = rhs_for(nm, w, seed_of((nm, w)))
            xd = torch.zeros(op.n, dtype=torch.float64, device="cuda")
            solo = op.solve(w, torch.from_numpy(rhs).cuda(), xd, pm.Options(rtol=1e-12, prec=p, max_restarts=5),
                            allow_not_converged=True)
            assert np.linalg.norm(x - xd.cpu().numpy()) <= 1e-9 * np.linalg.norm(xd.cpu().numpy()), (nm, w)
            assert abs(st.first_pass_iters - solo.first_pass_iters) <= max(2, 0.02 * solo.first_pass_iters)


def test_batch_autotune_picks_a_shape():
    xs, stats, info = run_batch(ENTRIES[:4], pm.PREC_LINE, rtol=1e-10, autotune=True)
    assert info["tile_cols"] in (16, 32, 64) and info["block"] in (128, 256)
    assert all(s.status == pm.PM_OK for s in stats)


def test_batch_rejects_bad_options():
    op = case("box16")[1]
    for opts in (pm.Options(prec=7), pm.Options(precision=3), pm.Options(rtol=0.0)):
        with pytest.raises(pm.PMError) as ei:
            pm.Batch([op], [pm.OP_VEL_U1], opts)
        assert ei.value.status == pm.PM_EINVAL
    with pytest.raises(pm.PMError) as ei:
        pm.Batch([op], [pm.OP_GRAD_X], pm.Options(prec=pm.PREC_IC0))
    assert ei.value.status == pm.PM_EINVAL


def test_bounded_grid_wait_reports_timeout_and_gpu_stays_usable():
    assert pm.debug_barrier_timeout() == pm.PM_TIMEOUT
    # the context still works
    xs, stats, _ = run_batch([ENTRIES[0]], pm.PREC_JACOBI, rtol=1e-10)
    assert stats[0].status == pm.PM_OK
