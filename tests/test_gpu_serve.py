"""Continuous-batching server on the GPU: systems admitted between quanta give the same bits as the
one-shot batch, a request served alone and inside a stream of others gives identical results,
solutions match the oracle, and slot / argument errors are reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, pcg as opcg  # noqa: E402
from workloads import Session, Request, box_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu

import paper_1207_0486_gb300 as pm  # noqa: E402
from paper_1207_0486_gb300.serve import GpuBackend, Scheduler, RHS_WHICH  # noqa: E402
from test_gpu_batch import ENTRIES, case, rhs_for, seed_of, run_batch  # noqa: E402


def oracle_solve(ops, which, rhs):
    if which == pm.OP_PRESSURE:
        return opcg.pressure_solve(ops.K_I, ops.m, rhs, rtol=1e-12).x
    A = ops.A_u(which - pm.OP_VEL_U1, bdf1=False)
    return opcg.pcg(A, rhs, rtol=1e-13, precond=opcg.jacobi_preconditioner(A)).x


@pytest.mark.parametrize("precision,prec", [(pm.FP64, pm.PREC_LINE), (pm.FP32_REFINE, pm.PREC_LINE),
                                            (pm.FP64, pm.PREC_IC0), (pm.FP32_REFINE, pm.PREC_IC0),
                                            (pm.BF16_REFINE, pm.PREC_LINE)])
def test_staggered_admission_matches_one_shot_batch(precision, prec):
    """Same tile width and block as the one-shot batch: admitted in three waves between quanta,
    every system reproduces the batch's bits and iteration counts."""
    rtol = 1e-10 if precision == pm.FP64 else 1e-8
    ref_x, ref_st, info = run_batch(ENTRIES, prec, precision=precision, rtol=rtol)
    # the options run_batch uses (its inner_rtol is the Options default)
    srv = pm.Server(slots=8, nz_cap=16, opts=pm.Options(rtol=rtol, prec=prec, precision=precision,
                                                        max_iter=200000),
                    tile_cols=info["tile_cols"], block=info["block"])
    bs, xs, ws, slot_of = [], [], [], {}
    for nm, w in ENTRIES:
        op = case(nm)[1]
        bs.append(torch.from_numpy(rhs_for(nm, w, seed_of((nm, w)))).cuda())
        xs.append(torch.full((op.n,), 7.0, dtype=torch.float64, device="cuda"))  # overwritten: x0 = 0
        ws.append(torch.empty(srv.workspace_bytes(op), dtype=torch.uint8, device="cuda"))
    stats = {}
    waves = [[0, 1, 2], [3, 4], [5, 6, 7]]
    for wave in waves:
        for i in wave:
            nm, w = ENTRIES[i]
            s = srv.admit(case(nm)[1], w, bs[i], xs[i], ws[i])
            assert s is not None
            slot_of[s] = i
        srv.run(3)
        for s, st in srv.poll():
            stats[slot_of.pop(s)] = st
    while slot_of:
        srv.run(16)
        for s, st in srv.poll():
            stats[slot_of.pop(s)] = st
    srv.close()
    for i in range(len(ENTRIES)):
        assert stats[i].status == pm.PM_OK
        assert stats[i].iters == ref_st[i].iters, ENTRIES[i]
        assert np.array_equal(xs[i].cpu().numpy(), ref_x[i]), ENTRIES[i]


def test_server_admission_with_its_own_preconditioner():
    """Systems admitted with their own preconditioners (IC0 velocity and mass, line pressure) give
    the bits of the one-shot batch built with the same per-system list."""
    from test_gpu_batch import MASS_ENTRIES, paper_precs
    entries = ENTRIES + MASS_ENTRIES
    precs = paper_precs(entries)
    ref_x, ref_st, info = run_batch(entries, pm.PREC_JACOBI, rtol=1e-10, per_entry=precs)
    srv = pm.Server(slots=16, nz_cap=16, opts=pm.Options(rtol=1e-10, prec=pm.PREC_JACOBI, max_iter=200000),
                    tile_cols=info["tile_cols"], block=info["block"])
    xs, slot_of, stats = [], {}, {}
    keep = []
    for i, ((nm, w), p) in enumerate(zip(entries, precs)):
        op = case(nm)[1]
        b = torch.from_numpy(rhs_for(nm, w, seed_of((nm, w)))).cuda()
        x = torch.zeros(op.n, dtype=torch.float64, device="cuda")
        ws = torch.empty(srv.workspace_bytes(op), dtype=torch.uint8, device="cuda")
        keep.append((b, ws))
        xs.append(x)
        s = srv.admit(op, w, b, x, ws, prec=p)
        slot_of[s] = i
        if i == 5:       # the rest join while the first ones iterate
            srv.run(4)
            for s2, st in srv.poll():
                stats[slot_of.pop(s2)] = st
    while slot_of:
        srv.run(16)
        for s, st in srv.poll():
            stats[slot_of.pop(s)] = st
    srv.close()
    for i, e in enumerate(entries):
        assert stats[i].status == pm.PM_OK, e
        assert stats[i].iters == ref_st[i].iters, e
        assert np.array_equal(xs[i].cpu().numpy(), ref_x[i]), e
    with pytest.raises(pm.PMError):
        srv2 = pm.Server(slots=2, nz_cap=16)
        try:
            op = case("box16")[1]
            b = torch.zeros(op.n, dtype=torch.float64, device="cuda")
            srv2.admit(op, pm.OP_VEL_U1, b, torch.zeros_like(b),
                       torch.empty(srv2.workspace_bytes(op), dtype=torch.uint8, device="cuda"), prec=9)
        finally:
            srv2.close()


def small_stream():
    sessions = [Session(side=12, nz=8, seed=11), Session(side=16, nz=10, seed=12), Session(side=10, nz=12, seed=13),
                Session(side=14, nz=9, seed=14)]
    reqs = []
    t = 0.0
    for k in range(12):
        t += 0.002
        reqs.append(Request(t_arrival=t, session=k % 4, step=k // 4, nrhs=1 + (k * 3) % 4, rhs_seed=1000 + 17 * k))
    return sessions, reqs


def test_request_alone_and_in_the_mix_give_identical_results():
    sessions, reqs = small_stream()
    target = 9  # session 1, step 2, 4 right-hand sides
    assert reqs[target].nrhs == 4
    keys = [(target, j) for j in range(4)]
    be = GpuBackend(slots=16, nz_cap=16, rhs="host", keep=keys)
    rep = Scheduler(be, sessions, reqs, slots=16, quantum=4).run()
    be.close()
    mixed = {j: be.kept[(target, j)] for j in range(4)}
    rec = rep.records[target]
    assert all(s == pm.PM_OK for r in rep.records for s in r.status)
    # the same request alone (its own session, nothing else resident)
    alone_req = [Request(t_arrival=0.0, session=1, step=0, nrhs=4, rhs_seed=reqs[target].rhs_seed)]
    be2 = GpuBackend(slots=16, nz_cap=16, rhs="host", keep=[(0, j) for j in range(4)])
    rep2 = Scheduler(be2, sessions, alone_req, slots=16, quantum=4).run()
    be2.close()
    for j in range(4):
        assert np.array_equal(be2.kept[(0, j)], mixed[j]), j
    assert rep2.records[0].iters == rec.iters
    # and the oracle's solutions (FP32 inner, FP64 refinement to 1e-8)
    basin = box_basin(nh=16, nz=10, seed=12)
    ops = fem.assemble(basin)
    for j in range(4):
        rhs = random_vector(ops.mesh.n, reqs[target].rhs_seed + j)
        ref = oracle_solve(ops, RHS_WHICH[j], rhs)
        assert np.linalg.norm(mixed[j] - ref) <= 1e-5 * np.linalg.norm(ref), j
    # pressure: zero mean in the M-weighted sense
    assert abs(ops.m @ mixed[3]) <= 1e-12 * np.abs(ops.m).sum() * np.abs(mixed[3]).max()


def test_serial_baseline_agrees():
    sessions, reqs = small_stream()
    keys = [(i, j) for i in range(4) for j in range(reqs[i].nrhs)]
    a = GpuBackend(slots=16, nz_cap=16, rhs="host", keep=keys)
    Scheduler(a, sessions, reqs[:4], slots=16, quantum=4).run()
    a.close()
    b = GpuBackend(slots=16, nz_cap=16, rhs="host", keep=keys)
    rep = Scheduler(b, sessions, reqs[:4], slots=16, mode="serial").run()
    assert all(s == pm.PM_OK for r in rep.records for s in r.status)
    for k in keys:
        assert np.linalg.norm(a.kept[k] - b.kept[k]) <= 1e-5 * np.linalg.norm(b.kept[k]), k


def test_server_slot_and_argument_errors():
    op = case("box16")[1]
    srv = pm.Server(slots=2, nz_cap=8, opts=pm.Options(rtol=1e-8, prec=pm.PREC_JACOBI))
    b = torch.from_numpy(rhs_for("box16", pm.OP_VEL_U1, 1)).cuda()
    xs = [torch.zeros(op.n, dtype=torch.float64, device="cuda") for _ in range(3)]
    ws = [torch.empty(srv.workspace_bytes(op), dtype=torch.uint8, device="cuda") for _ in range(3)]
    assert srv.admit(op, pm.OP_VEL_U1, b, xs[0], ws[0]) is not None
    assert srv.admit(op, pm.OP_VEL_U2, b, xs[1], ws[1]) is not None
    assert srv.admit(op, pm.OP_VEL_U3, b, xs[2], ws[2]) is None  # PM_EBUSY: both slots taken
    with pytest.raises(pm.PMError) as ei:
        srv.admit(op, pm.OP_GRAD_X, b, xs[2], ws[2])
    assert ei.value.status == pm.PM_EINVAL
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(pm.PMError):
        srv.admit(op, pm.OP_VEL_U3, b, xs[2], small)
    done = []
    for _ in range(100):
        srv.run(16)
        done += srv.poll()
        if len(done) == 2:
            break
    assert len(done) == 2 and all(st.status == pm.PM_OK for _, st in done)
    assert srv.admit(op, pm.OP_VEL_U3, b, xs[2], ws[2]) is not None  # a freed slot is reused
    srv.close()
    deep = pm.assemble_operator(box_basin(nh=8, nz=12))
    srv2 = pm.Server(slots=2, nz_cap=8)
    wd = torch.empty(srv2.workspace_bytes(deep), dtype=torch.uint8, device="cuda")
    xd = torch.zeros(deep.n, dtype=torch.float64, device="cuda")
    with pytest.raises(pm.PMError) as ei:
        srv2.admit(deep, pm.OP_PRESSURE, xd, xd, wd)
    assert ei.value.status == pm.PM_EINVAL  # nz 12 > nz_cap 8
    srv2.close()


def test_consistent_mass_correction_is_served_with_ic0():
    """A step with the consistent-mass velocity correction is seven systems: the mass systems
    (j = 4, 5, 6) join the same persistent kernel with IC0 while the others keep the line
    preconditioner. Continuous and serial serving agree, and the mass solutions match the oracle's
    M^{-1} rhs."""
    sessions, reqs = small_stream()
    reqs = [Request(t_arrival=r.t_arrival, session=r.session, step=r.step, nrhs=7, rhs_seed=r.rhs_seed)
            for r in reqs[:4]]
    keys = [(i, j) for i in range(4) for j in range(7)]
    a = GpuBackend(slots=32, nz_cap=16, rhs="host", keep=keys, correction="consistent")
    rep = Scheduler(a, sessions, reqs, slots=32, quantum=4).run()
    a.close()
    assert all(s == pm.PM_OK for r in rep.records for s in r.status)
    assert all(r.iters[j] < 40 for r in rep.records for j in (4, 5, 6)), [r.iters for r in rep.records]
    b = GpuBackend(slots=32, nz_cap=16, rhs="host", keep=keys, correction="consistent")
    Scheduler(b, sessions, reqs, slots=32, mode="serial").run()
    for k in keys:
        assert np.linalg.norm(a.kept[k] - b.kept[k]) <= 1e-5 * np.linalg.norm(b.kept[k]), k
    s0 = sessions[reqs[0].session]
    ops = fem.assemble(box_basin(nh=s0.side, nz=s0.nz, seed=s0.seed))
    for j in (4, 5, 6):
        rhs = random_vector(ops.mesh.n, reqs[0].rhs_seed + j)
        ref = opcg.pcg(ops.M, rhs, rtol=1e-13, precond=opcg.ic0_preconditioner(ops.M, ops.mesh.colour)[0]).x
        assert np.linalg.norm(a.kept[(0, j)] - ref) <= 1e-6 * np.linalg.norm(ref), j
