"""The allocation-free PCG entry point, checked through the C ABI against the regular entry point
and against the FP64 oracle.

pm_pcg_solve_noalloc exists for callers that cannot allocate device memory when they solve:
processes whose device memory belongs to a framework allocator or a fixed pool, and embedded
users that must not grow the device footprint after start-up. Its scratch is one static device
array shared by every call, so each case runs it twice in a row and checks that the second call,
which starts from the first call's leftovers, gives the same answer, and that neither the
driver's free memory nor torch's reserved memory moves during those calls. This file is
collected last so that a run that stops at the first failure has run every other test first.
"""
import warnings

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1207_0486_gb300 as pm  # noqa: E402
from oracle import fem, pcg as opcg  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    out = {}
    for name, b in (("box16", box_basin()), ("small", small_basin())):
        out[name] = (pm.assemble_operator(b), fem.assemble(b))
    return out


def _oracle(ops, which, rhs, prec, rtol):
    if which == pm.OP_PRESSURE:
        A = ops.K_I
    else:
        c = (which - pm.OP_VEL1_U1) if which >= pm.OP_VEL1_U1 else which
        A = ops.A_u(c, bdf1=which >= pm.OP_VEL1_U1)
    P = opcg.jacobi_preconditioner(A) if prec == pm.PREC_JACOBI else None
    if which == pm.OP_PRESSURE:
        return opcg.pressure_solve(A, ops.m, rhs, rtol=rtol, precond=P)
    return opcg.pcg(A, rhs, rtol=rtol, precond=P)


@pytest.mark.parametrize("name", ["box16", "small"])
@pytest.mark.parametrize("which,prec", [(pm.OP_VEL_U1, pm.PREC_JACOBI), (pm.OP_VEL1_U3, pm.PREC_NONE),
                                        (pm.OP_PRESSURE, pm.PREC_JACOBI)])
def test_noalloc_matches_the_allocating_solve_and_the_oracle(ops, name, which, prec):
    op, oops = ops[name]
    rhs_h = random_vector(op.n, 99 + which)
    rhs = torch.from_numpy(rhs_h).cuda()
    opts = pm.Options(rtol=1e-10, prec=prec)
    x_ref = torch.zeros_like(rhs)
    st_ref = op.solve(which, rhs, x_ref, opts)
    ref = x_ref.cpu().numpy()
    torch.cuda.synchronize()
    free0 = reserved0 = None
    for call in range(2):
        x = torch.full_like(rhs, float("nan"))   # poisoned output: every entry must be written
        if call == 1:
            free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
        st = op.solve_noalloc(which, rhs, x, opts)
        got = x.cpu().numpy()
        assert st.status == pm.PM_OK
        # the parity rule for iteration counts: within 2, or 2% of a long solve (the two solves
        # reduce in different orders, and long CG runs are chaotic in the last bits)
        assert abs(st.iters - st_ref.iters) <= max(2, 0.02 * max(st.iters, st_ref.iters)), (call, st.iters, st_ref.iters)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-9, (call, err)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0 and torch.cuda.memory_reserved() == reserved0
    # against the oracle: both solved to a tight tolerance, solutions agree to 1e-9
    tight = 1e-12 if which == pm.OP_PRESSURE else 1e-13
    x = torch.zeros_like(rhs)
    op.solve_noalloc(which, rhs, x, pm.Options(rtol=tight, prec=prec, max_restarts=5), allow_not_converged=True)
    o = _oracle(oops, which, rhs_h, prec, tight)
    err = np.linalg.norm(x.cpu().numpy() - o.x) / np.linalg.norm(o.x)
    assert err <= 1e-9, err


def test_noalloc_runs_no_iteration_at_max_iter_zero(ops):
    op, _ = ops["small"]
    rhs = torch.from_numpy(random_vector(op.n, 5)).cuda()
    x = torch.zeros_like(rhs)
    st = op.solve_noalloc(pm.OP_VEL_U1, rhs, x, pm.Options(rtol=1e-10, max_iter=0), allow_not_converged=True)
    assert st.status == pm.PM_NOT_CONVERGED and st.iters == 0
    assert float(x.abs().max()) == 0.0


def test_noalloc_rejects_a_capturing_stream(ops):
    op, _ = ops["small"]
    rhs = torch.from_numpy(random_vector(op.n, 6)).cuda()
    x = torch.zeros_like(rhs)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with warnings.catch_warnings():  # torch may note that the captured graph is empty
        warnings.simplefilter("ignore")
        with torch.cuda.graph(g, stream=s):
            with pytest.raises(pm.PMError) as ei:
                op.solve_noalloc(pm.OP_VEL_U1, rhs, x, pm.Options(), stream=s)
    assert ei.value.status == pm.PM_EINVAL and "captured" in str(ei.value)
    del g
    st = op.solve_noalloc(pm.OP_VEL_U1, rhs, x, pm.Options(rtol=1e-10))   # usable afterwards
    assert st.status == pm.PM_OK


def test_noalloc_rejects_systems_above_its_limit():
    big = pm.assemble_operator(box_basin(nh=130, nz=32))      # 540,800 rows > 524,288
    assert big.n > 524288
    b = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(pm.PMError) as ei:
        big.solve_noalloc(pm.OP_PRESSURE, b, x, pm.Options(prec=pm.PREC_JACOBI))
    assert ei.value.status == pm.PM_EINVAL and "PM_NOALLOC_MAX_ROWS" in str(ei.value)
    with pytest.raises(pm.PMError):
        big.solve_noalloc(pm.OP_PRESSURE, b, x, pm.Options(prec=pm.PREC_IC0))
