"""Parity at the full 512 x 512 x 32 ocean-basin size, in the bench's launch configuration.

The oracle cannot assemble 5.4M-node operators in seconds, so it computes sampled rows one by
one (from the tets that contain each sampled node) and the checks compare those rows, the
SpMV on those rows, and residual rows of the full-size solves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fem, mesh as omesh  # noqa: E402
from workloads import ocean_basin, random_vector  # noqa: E402
from gpu_util import slot_columns  # noqa: E402

pytestmark = pytest.mark.gpu

import paper_1207_0486_gb300 as pm  # noqa: E402

NSAMPLE = 3000


@pytest.fixture(scope="module")
def full():
    b = ocean_basin()
    op = pm.assemble_operator(b)
    mesh = omesh.build_mesh(b)
    rng = np.random.default_rng(7)
    rows = np.unique(np.concatenate([rng.integers(0, mesh.n, NSAMPLE), [0, mesh.n - 1],
                                     np.arange(mesh.nz) + (mesh.ncols // 2) * mesh.nz]))
    sel = np.isin(mesh.tets, rows).any(axis=1)
    tets = mesh.tets[sel]
    vol, grads = fem.tet_geometry(mesh.xyz, tets)
    mats = {
        "M": fem.assemble_matrix(mesh.n, tets, fem.element_mass(vol)),
        "Knu": fem.assemble_matrix(mesh.n, tets, fem.element_stiffness(vol, grads, b.nu)),
        "KI": fem.assemble_matrix(mesh.n, tets, fem.element_stiffness(vol, grads, (1, 1, 1))),
    }
    for c in range(3):
        mats[f"G{c}"] = fem.assemble_matrix(mesh.n, tets, fem.element_gradient(vol, grads, c))
    return b, op, mesh, rows, mats


def _oracle_rows(full, which):
    b, op, mesh, rows, mats = full
    if which == pm.OP_PRESSURE:
        A = mats["KI"]
    elif which == pm.OP_MASS:
        A = mats["M"]
    elif which in (pm.OP_GRAD_X, pm.OP_GRAD_Y, pm.OP_GRAD_Z):
        A = mats[f"G{which - pm.OP_GRAD_X}"]
    else:
        bdf1 = which >= pm.OP_VEL1_U1
        c = which - (pm.OP_VEL1_U1 if bdf1 else pm.OP_VEL_U1)
        alpha = (1.0 if bdf1 else 1.5) / b.dt
        A = (alpha * mats["M"] + mats["Knu"]).tocsr()
        A.sort_indices()
        A = fem.eliminate_dirichlet(A, mesh.dirichlet[c])
    return A[rows].toarray()


@pytest.mark.parametrize("which", [pm.OP_VEL_U1, pm.OP_VEL1_U2, pm.OP_VEL_U3, pm.OP_PRESSURE, pm.OP_MASS,
                                   pm.OP_GRAD_X, pm.OP_GRAD_Z])
def test_fullsize_sampled_rows_and_spmv(full, which):
    b, op, mesh, rows, mats = full
    assert op.n == mesh.n
    vals, nbr, st = op.export(which)
    cols = slot_columns(nbr, op.nz)
    ref = _oracle_rows(full, which)                      # (len(rows), n) dense rows
    for t, r in enumerate(rows):
        g = np.zeros(op.n)
        for s in range(15):
            if cols[s, r] >= 0:
                g[cols[s, r]] += vals[s, r]
        nzc = np.nonzero(ref[t] != 0)[0]
        scale = np.abs(ref[t]).max()
        assert np.abs(g[nzc] - ref[t, nzc]).max() <= 1e-12 * scale
        assert np.abs(np.delete(g, nzc)).max(initial=0.0) <= 1e-12 * scale
    x = random_vector(op.n, 11)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    op.spmv(which, xd, y)
    yo = ref @ x
    err = np.abs(y.cpu().numpy()[rows] - yo).max() / (np.abs(ref) @ np.abs(x)).max()
    assert err <= 1e-14


@pytest.mark.parametrize("which,prec", [(pm.OP_VEL1_U1, pm.PREC_IC0), (pm.OP_PRESSURE, pm.PREC_LINE)])
def test_fullsize_solve_residual_rows(full, which, prec):
    b, op, mesh, rows, mats = full
    rhs = random_vector(op.n, 23)
    if which != pm.OP_PRESSURE:
        rhs[mesh.dirichlet[0]] = 0.0
    rtol = 1e-8
    bd = torch.from_numpy(rhs).cuda()
    x = torch.zeros_like(bd)
    st = op.solve(which, bd, x, pm.Options(rtol=rtol, prec=prec, max_iter=200000))
    assert st.status == pm.PM_OK and st.rel_residual_true <= max(rtol, st.rel_residual_floor)
    rtol = max(rtol, st.rel_residual_floor)
    xg = x.cpu().numpy()
    ref = _oracle_rows(full, which)
    if which == pm.OP_PRESSURE:
        # the solved system is K q = b - lam m, lam = 1'b / 1'm, m = M 1; 1'm is the exact volume
        from test_oracle_fem import sigma_mesh_volume
        m_rows = np.asarray(mats["M"][rows].sum(axis=1)).ravel()
        lam = rhs.sum() / sigma_mesh_volume(b)
        res_rows = (rhs[rows] - lam * m_rows) - ref @ xg
        assert np.abs(res_rows).max() <= 1.01 * rtol * np.linalg.norm(rhs)
    else:
        res_rows = rhs[rows] - ref @ xg
        assert np.abs(res_rows).max() <= rtol * np.linalg.norm(rhs)
