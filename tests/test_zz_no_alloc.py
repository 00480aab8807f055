"""The allocation-free PCG entry point, checked against the regular one through the C ABI.

pm_pcg_solve_noalloc exists for callers that cannot allocate device memory when they solve
(inside a stream capture that must not gain allocation nodes, under a framework-owned or fixed
memory pool, or in embedded use that must not grow after start-up). Its scratch is one static
device array shared by every call, so the test runs it twice in a row and checks that the
second call, which starts from the first call's leftovers, gives the same answer. This file is
collected last so that a run that stops at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1207_0486_gb300 as pm  # noqa: E402
from test_oracle_fem import small_basin  # noqa: E402
from workloads import box_basin, random_vector  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ops():
    return {"box16": pm.assemble_operator(box_basin()), "small": pm.assemble_operator(small_basin())}


@pytest.mark.parametrize("name", ["box16", "small"])
@pytest.mark.parametrize("which,prec", [(pm.OP_VEL_U1, pm.PREC_JACOBI), (pm.OP_VEL1_U3, pm.PREC_NONE),
                                        (pm.OP_PRESSURE, pm.PREC_JACOBI)])
def test_noalloc_matches_the_allocating_solve(ops, name, which, prec):
    op = ops[name]
    rhs = torch.from_numpy(random_vector(op.n, 99 + which)).cuda()
    opts = pm.Options(rtol=1e-10, prec=prec)
    x_ref = torch.zeros_like(rhs)
    st_ref = op.solve(which, rhs, x_ref, opts)
    ref = x_ref.cpu().numpy()
    for call in range(2):
        x = torch.full_like(rhs, float("nan"))   # poisoned output: every entry must be written
        st = op.solve_noalloc(which, rhs, x, opts)
        got = x.cpu().numpy()
        assert st.status == pm.PM_OK
        assert abs(st.iters - st_ref.iters) <= 2, (call, st.iters, st_ref.iters)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 1e-9, (call, err)


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
