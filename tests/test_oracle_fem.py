"""Pins of the oracle's mesh, element integrals and assembled operators (CPU only)."""
import math

import numpy as np
import pytest

from conftest import read_golden
from oracle import fem, mesh as omesh
from workloads import box_basin, WALL_ALL, WALL_SOUTH, WALL_NORTH, Basin


def small_basin(seed=3, nx=9, ny=8, nz=5, slip=WALL_SOUTH | WALL_NORTH):
    """Irregular little basin: random depths, a land notch, slip south/north walls."""
    rng = np.random.default_rng(seed)
    mask = np.ones((ny, nx), dtype=np.uint8)
    mask[3:5, 0:3] = 0       # land notch on the west side
    mask[ny - 1, nx - 1] = 0
    depth = rng.uniform(200.0, 4000.0, (ny, nx))
    cor = rng.uniform(0.0, 1e-4, (ny, nx))
    theta = rng.standard_normal((2, ny, nx)) * 1e-4
    return Basin(name="small", nx=nx, ny=ny, nz=nz, dx=1e4, dy=1.2e4, mask=mask, depth=depth,
                 slip_walls=slip, nu=(1e8, 2e8, 1e2), dt=2.592e6, coriolis=cor, theta=theta)


@pytest.fixture(scope="module")
def box_ops():
    return fem.assemble(box_basin(nh=6, nz=4))


@pytest.fixture(scope="module")
def basin_ops():
    return fem.assemble(small_basin())


def test_reference_tet_closed_forms():
    g = read_golden("reference_tet_p1.txt")
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    vol, grads = fem.tet_geometry(xyz, np.array([[0, 1, 2, 3]]))
    assert vol[0] == pytest.approx(1.0 / 6.0, abs=1e-15)
    np.testing.assert_allclose(6 * fem.element_stiffness(vol, grads, (1, 1, 1))[0], g["stiffness x6"], atol=1e-14)
    np.testing.assert_allclose(120 * fem.element_mass(vol)[0], g["mass x120"], atol=1e-14)
    np.testing.assert_allclose(24 * fem.element_gradient(vol, grads, 0)[0], g["gradx x24"], atol=1e-14)
    # anisotropic stiffness weights each axis: nu = (2, 3, 5) on the reference tet
    Kn = fem.element_stiffness(vol, grads, (2.0, 3.0, 5.0))[0] * 6
    exp = np.array([[10, -2, -3, -5], [-2, 2, 0, 0], [-3, 0, 3, 0], [-5, 0, 0, 5.0]])
    np.testing.assert_allclose(Kn, exp, atol=1e-14)


def test_kuhn_split_conforms_and_is_positive(basin_ops):
    m = basin_ops.mesh
    assert np.all(basin_ops.vol > 0)
    # every interior triangular face is shared by exactly two tets, boundary faces by one
    faces = np.sort(np.concatenate([m.tets[:, [0, 1, 2]], m.tets[:, [0, 1, 3]], m.tets[:, [0, 2, 3]],
                                    m.tets[:, [1, 2, 3]]]), axis=1)
    _, counts = np.unique(faces, axis=0, return_counts=True)
    assert set(np.unique(counts)) <= {1, 2}


def test_stencil_is_the_15_slot_kuhn_stencil(basin_ops):
    """Every nonzero of the operators joins a node to one of the 14 Kuhn neighbours or itself."""
    m = basin_ops.mesh
    A = basin_ops.K_I.tocoo()
    col = A.row // m.nz
    d = np.stack([m.col_i[A.col // m.nz] - m.col_i[col], m.col_j[A.col // m.nz] - m.col_j[col],
                  (A.col % m.nz) - (A.row % m.nz)], 1)
    allowed = {(0, 0, 0)}
    for v in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]:
        allowed.add(v)
        allowed.add(tuple(-x for x in v))
    assert {tuple(r) for r in d} <= allowed
    assert max(np.diff(basin_ops.K_I.indptr)) <= 15


def test_box_nnz_and_counts():
    ops = fem.assemble(box_basin())
    assert ops.n == 16 * 16 * 8
    assert ops.M.nnz == 26782            # 2048 diagonals + 2 x 12367 Kuhn edges


@pytest.mark.parametrize("which", ["M", "K_nu", "K_I"])
def test_symmetry(basin_ops, which):
    A = getattr(basin_ops, which)
    assert abs(A - A.T).max() <= 1e-14 * abs(A).max()


def test_velocity_operators_symmetric_with_identity_rows(basin_ops):
    for c in range(3):
        for bdf1 in (True, False):
            A = basin_ops.A_u(c, bdf1)
            assert abs(A - A.T).max() <= 1e-14 * abs(A).max()
            D = basin_ops.mesh.dirichlet[c]
            Ad = A[D]
            assert np.allclose(Ad.toarray(), np.eye(basin_ops.n)[D])


def test_nullspace_and_row_sums(basin_ops):
    one = np.ones(basin_ops.n)
    for K in (basin_ops.K_nu, basin_ops.K_I):
        assert abs(K @ one).max() <= 1e-12 * abs(K).max()
    for c in range(3):
        assert abs(basin_ops.G[c] @ one).max() <= 1e-12 * abs(basin_ops.G[c]).max()


def test_gradient_of_coordinates(basin_ops):
    """G_c X_d = delta_cd M 1: the derivative of the coordinate field x_d is delta_cd."""
    m1 = basin_ops.m
    for c in range(3):
        for d in range(3):
            v = basin_ops.G[c] @ basin_ops.mesh.xyz[:, d]
            np.testing.assert_allclose(v, m1 if c == d else 0 * m1, atol=1e-10 * m1.max())


def sigma_mesh_volume(b):
    """Exact volume of the Kuhn-split sigma mesh: each tet's volume is (dx dy / 6) times the
    layer thickness of its single vertical edge; per cell this sums to
    dx dy / 6 (2 h00 + h10 + h01 + 2 h11)."""
    m = b.mask.astype(bool)
    cell = m[:-1, :-1] & m[1:, :-1] & m[:-1, 1:] & m[1:, 1:]
    h = b.depth
    per = (2 * h[:-1, :-1] + h[:-1, 1:] + h[1:, :-1] + 2 * h[1:, 1:]) * b.dx * b.dy / 6.0
    return per[cell].sum()


def test_mass_total_is_domain_volume(box_ops, basin_ops):
    assert box_ops.M.sum() == pytest.approx(0.01, rel=1e-13)
    assert basin_ops.M.sum() == pytest.approx(sigma_mesh_volume(small_basin()), rel=1e-12)


def test_surface_mass(basin_ops):
    m = basin_ops.mesh
    b = small_basin()
    cell = m.cell_active
    area = cell.sum() * b.dx * b.dy
    top = m.surface.astype(float)
    assert (basin_ops.S @ top).sum() == pytest.approx(area, rel=1e-13)
    # linear theta = x: integral = sum over cells of dx dy * (cell centroid x) exactly
    cj, ci = np.nonzero(cell)
    exact = ((ci + 0.5) * b.dx * b.dx * b.dy).sum()
    assert (basin_ops.S @ (top * m.xyz[:, 0])).sum() == pytest.approx(exact, rel=1e-13)


def test_advection_closed_form(basin_ops):
    """Constant velocity U advecting linear fields u_c = a_c . x gives (U . a_c) M 1."""
    rng = np.random.default_rng(5)
    U = rng.standard_normal(3)
    a = rng.standard_normal((3, 3))
    n = basin_ops.n
    xyz = basin_ops.mesh.xyz
    # velocity field: each component c is U_c + a_c . x ; the advected field is u_c itself, so
    # (u . grad) u_c = (U + a x) . a_c -- use a = 0 for the velocity part by splitting fields:
    u = np.stack([np.full(n, U[c]) for c in range(3)])
    out = fem.advection_term(basin_ops, u)
    np.testing.assert_allclose(out, 0.0, atol=1e-12 * basin_ops.m.max())
    # u = U + A x: (u . grad) u_c = sum_d (U_d + (A x)_d) A_cd; integral against phi_i is
    # sum_d A_cd (U_d (M1)_i + (M (A x)_d)_i)
    Ax = xyz @ a.T                                     # (n, 3): (A x)_d
    u = (U[None, :] + Ax).T
    out = fem.advection_term(basin_ops, u)
    M = basin_ops.M
    for c in range(3):
        exp = sum(a[c, d] * (U[d] * basin_ops.m + M @ Ax[:, d]) for d in range(3))
        np.testing.assert_allclose(out[c], exp, rtol=1e-9, atol=1e-9 * abs(exp).max())


def test_advection_against_quadrature():
    """Degree-2 integrand on one tet: compare with the 4-point rule exact for quadratics."""
    rng = np.random.default_rng(11)
    xyz = rng.standard_normal((4, 3))
    tets = np.array([[0, 1, 2, 3]])
    vol, grads = fem.tet_geometry(xyz, tets)
    u = rng.standard_normal((3, 4))

    class O:
        pass
    o = O()
    o.mesh = O()
    o.mesh.tets = tets
    o.vol, o.grads, o.n = vol, grads, 4
    out = fem.advection_term(o, u)
    a, b = 0.5854101966249685, 0.1381966011250105
    pts = [np.array([a, b, b, b]), np.array([b, a, b, b]), np.array([b, b, a, b]), np.array([b, b, b, a])]
    exp = np.zeros((3, 4))
    gu = u @ grads[0]                                  # (c, d)
    for lam in pts:
        uq = u @ lam                                   # (3,) velocity at the point
        for c in range(3):
            exp[c] += vol[0] / 4 * (uq @ gu[c]) * lam
    np.testing.assert_allclose(out, exp, rtol=1e-12, atol=1e-13)


def test_boundary_sets_box():
    b = box_basin(nh=5, nz=4)
    m = omesh.build_mesh(b)
    k = np.tile(np.arange(4), m.ncols)
    i = np.repeat(m.col_i, 4)
    j = np.repeat(m.col_j, 4)
    assert np.array_equal(m.dirichlet[0], (k == 0) | (i == 0) | (i == 4))
    assert np.array_equal(m.dirichlet[1], (k == 0) | (j == 0) | (j == 4))
    assert np.array_equal(m.dirichlet[2], (k == 0) | (k == 3))
    # no-slip walls instead: every lateral wall is Gamma_0
    m2 = omesh.build_mesh(box_basin(nh=5, nz=4, slip_walls=0))
    lat = (i == 0) | (i == 4) | (j == 0) | (j == 4)
    for c in range(2):
        assert np.array_equal(m2.dirichlet[c], (k == 0) | lat)


def test_multicolour_is_proper(basin_ops):
    A = basin_ops.K_I.tocoo()
    col = basin_ops.mesh.colour
    off = A.row != A.col
    assert not np.any(col[A.row[off]] == col[A.col[off]])


# ---------------------------------------------------------------------------------------------
# Manufactured solutions on the thin box (eps = 0.01, nu = (1, 1, 1e-4)): second-order L2.
# ---------------------------------------------------------------------------------------------

EPS = 0.01
NU = (1.0, 1.0, 1e-4)
DT = 0.01


def _mms_velocity(c, xyz, modes, alpha):
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    zeta = (z + EPS) / EPS
    u = np.zeros(len(x))
    f = np.zeros(len(x))
    top = np.zeros(len(x))
    for amp, mm, ll in modes:
        kx, ky = mm * math.pi, ll * math.pi
        if c == 0:     # Dirichlet on x-walls, natural on y-walls, flux theta on top
            X = np.sin(kx * x) * np.cos(ky * y)
            kz = 0.75 * math.pi
            g, dg_top = np.sin(kz * zeta), kz * math.cos(kz)
        elif c == 1:
            X = np.cos(kx * x) * np.sin(ky * y)
            kz = 0.75 * math.pi
            g, dg_top = np.sin(kz * zeta), kz * math.cos(kz)
        else:          # u3 = 0 at bottom and top, natural on all lateral walls
            X = np.cos(kx * x) * np.cos(ky * y)
            kz = math.pi
            g, dg_top = np.sin(kz * zeta), 0.0
        u += amp * X * g
        f += amp * X * g * (alpha + NU[0] * kx ** 2 + NU[1] * ky ** 2 + NU[2] * (kz / EPS) ** 2)
        top += amp * X * NU[2] * dg_top / EPS
    return u, f, top


def _l2(ops, e):
    return math.sqrt(e @ (ops.M @ e))


@pytest.mark.parametrize("c", [0, 1, 2])
def test_mms_velocity_second_order(c):
    from oracle import pcg
    modes = [(1.0, 1, 2), (0.5, 2, 1)]
    errs = []
    for nh, nz in ((8, 4), (16, 8), (32, 16)):
        ops = fem.assemble(box_basin(nh=nh, nz=nz, eps=EPS, nu=NU, dt=DT))
        alpha = ops.alpha(False)
        u, f, top = _mms_velocity(c, ops.mesh.xyz, modes, alpha)
        b = ops.M @ f
        if c < 2:
            b += ops.S @ np.where(ops.mesh.surface, top, 0.0)
        b[ops.mesh.dirichlet[c]] = 0.0
        A = ops.A_u(c, False)
        uh = pcg.pcg(A, b, rtol=1e-13, precond=pcg.jacobi_preconditioner(A)).x
        errs.append(_l2(ops, uh - u) / _l2(ops, u))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r2 < 5.0, errs
    assert r1 > 2.5, errs


def test_mms_pressure_second_order():
    from oracle import pcg
    modes = [(1.0, 1, 2), (0.7, 2, 1)]
    errs = []
    for nh, nz in ((8, 4), (16, 8), (32, 16)):
        ops = fem.assemble(box_basin(nh=nh, nz=nz, eps=EPS, nu=NU, dt=DT))
        x, y, z = ops.mesh.xyz.T
        zeta = (z + EPS) / EPS
        q = np.zeros(ops.n)
        f = np.zeros(ops.n)
        for amp, mm, ll in modes:
            X = np.cos(mm * math.pi * x) * np.cos(ll * math.pi * y)
            k2 = (mm ** 2 + ll ** 2) * math.pi ** 2
            q += amp * X * (1.0 + np.cos(math.pi * zeta))
            f += amp * X * (k2 + (k2 + (math.pi / EPS) ** 2) * np.cos(math.pi * zeta))
        m1 = ops.m
        qh = pcg.pressure_solve(ops.K_I, m1, ops.M @ f, rtol=1e-13).x
        qi = q - (m1 @ q) / m1.sum()
        errs.append(_l2(ops, qh - qi) / _l2(ops, qi))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.2 < r2 < 5.0, errs
    assert r1 > 2.5, errs
