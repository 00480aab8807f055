"""Pins of the Q2 velocity / Q1 pressure oracle (Section 5: the spaces V_h and P_h on bricks;
Eqs. fofa_velo_pred_h, fofa_q_cor_h, fofa_velo_cor_h) against facts fixed by the mathematics:

- the bases are nodal (Kronecker delta at their nodes), sum to one, and reproduce every
  polynomial of degree <= 2 (Q2) or <= 1 (Q1) in each variable;
- 1'M2 1 = 1'M1 1 = the exact volume of a sigma mesh with varying depth and a land mask;
- on a flat box the mass, stiffness and coupling integrals of quadratic fields equal their closed
  forms (the 3-point rule is exact there), and D_c and B_c satisfy integration by parts;
- manufactured solutions converge at third order in L2 for Q2 and second order for Q1;
- one projection removes a pure gradient (the correction's sign; a flipped sign returns about
  twice the field).
A dropped term, a wrong sign or index, or a transposed operand in any of the element integrals
fails one of these.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import q2q1
from workloads import box_basin


def _rng_points(n, seed=0):
    return np.random.default_rng(seed).random((n, 3))


def test_reference_bases_are_nodal_and_reproduce_polynomials():
    nodes2 = q2q1.Q2_OFF / 2.0
    phi, grad = q2q1.tensor_basis(nodes2, 2)
    assert np.allclose(phi, np.eye(27), atol=1e-14)
    P = _rng_points(50)
    phi, grad = q2q1.tensor_basis(P, 2)
    assert np.allclose(phi.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(grad.sum(axis=1), 0.0, atol=1e-12)
    # a member of Q2: degree <= 2 in each variable (and its gradient)
    f = lambda x, y, z: 1 + x - 2 * y * z + 3 * x * x * y * y * z * z - y * y * z  # noqa: E731
    fx = lambda x, y, z: 1 + 6 * x * y * y * z * z  # noqa: E731
    fz = lambda x, y, z: -2 * y + 6 * x * x * y * y * z - y * y  # noqa: E731
    fv = f(*nodes2.T)
    assert np.allclose(phi @ fv, f(*P.T), atol=1e-12)
    assert np.allclose(grad[:, :, 0] @ fv, fx(*P.T), atol=1e-11)
    assert np.allclose(grad[:, :, 2] @ fv, fz(*P.T), atol=1e-11)
    nodes1 = q2q1.Q1_OFF.astype(float)
    phi1, g1 = q2q1.tensor_basis(nodes1, 1)
    assert np.allclose(phi1, np.eye(8), atol=1e-15)
    phi1, g1 = q2q1.tensor_basis(P, 1)
    t = lambda x, y, z: 2 - x + 4 * x * y * z - 3 * y * z  # noqa: E731
    assert np.allclose(phi1 @ t(*nodes1.T), t(*P.T), atol=1e-13)
    assert np.allclose(g1[:, :, 1] @ t(*nodes1.T), (4 * P[:, 0] * P[:, 2] - 3 * P[:, 2]), atol=1e-13)


def _sloped_basin():
    """A 7 x 6 x 4 basin with a bilinear-in-each-cell depth that varies from cell to cell and a
    land corner."""
    b = box_basin(nh=7, nz=4, eps=0.05, nhy=6)
    X, Y = np.meshgrid(np.arange(b.nx), np.arange(b.ny))
    b.depth = 0.05 * (1.0 + 0.3 * np.sin(X) + 0.2 * Y * Y / 25.0)
    b.mask[:2, :2] = 0
    return b


def test_volume_of_a_sigma_mesh_with_land():
    b = _sloped_basin()
    ops = q2q1.assemble_q2q1(b)
    cell = ops.mesh.base.cell_active
    d = b.depth
    vol = b.dx * b.dy * 0.25 * (d[:-1, :-1] + d[1:, :-1] + d[:-1, 1:] + d[1:, 1:])
    exact = float(vol[cell].sum())
    assert ops.M2.sum() == pytest.approx(exact, rel=1e-13, abs=0)
    assert ops.M1.sum() == pytest.approx(exact, rel=1e-13, abs=0)
    # symmetric positive mass, stiffness without constants in its range
    assert abs(ops.M2 - ops.M2.T).max() < 1e-15 * abs(ops.M2).max()
    assert np.abs(ops.K2 @ np.ones(ops.mesh.n2)).max() < 1e-12 * abs(ops.K2).max()
    assert np.abs(ops.K1 @ np.ones(ops.mesh.n1)).max() < 1e-12 * abs(ops.K1).max()
    assert np.all(ops.m2 > 0)   # row-sum lumping is positive on bricks


def test_linear_fields_on_skewed_bricks():
    """On the sloped mesh the bricks are skewed (d z / d xi != 0), so the gradient transform
    J^{-T} matters. Physical linear fields lie in both spaces (the geometry map is trilinear), their
    gradients are exact at every point, and the integrands reduce to constants times det J:
    f = g . x gives f' K2 f = (g . nu g) |Omega|, and 1' D_c x_d = 1' B_c x_d = delta_cd |Omega|."""
    b = _sloped_basin()
    ops = q2q1.assemble_q2q1(b)
    vol = ops.M1.sum()
    g = np.array([0.3, -1.1, 2.0])
    nu = np.array(b.nu)
    f2 = ops.mesh.xyz2 @ g
    f1 = ops.mesh.base.xyz @ g
    assert f2 @ (ops.K2 @ f2) == pytest.approx(float(g @ (nu * g)) * vol, rel=1e-12, abs=0)
    assert f1 @ (ops.K1 @ f1) == pytest.approx(float(g @ g) * vol, rel=1e-12, abs=0)
    one1 = np.ones(ops.mesh.n1)
    one2 = np.ones(ops.mesh.n2)
    for c in range(3):
        for d in range(3):
            want = vol if c == d else 0.0
            assert one1 @ (ops.D[c] @ ops.mesh.xyz2[:, d]) == pytest.approx(want, rel=1e-12, abs=1e-14 * vol)
            assert one2 @ (ops.B[c] @ ops.mesh.base.xyz[:, d]) == pytest.approx(want, rel=1e-12, abs=1e-14 * vol)


@pytest.fixture(scope="module")
def flat():
    """Unit square x [-eps, 0], eps = 0.3, 5 x 5 x 3 vertices, anisotropic nu."""
    b = box_basin(nh=5, nz=3, eps=0.3, nu=(1.3, 0.7, 0.2))
    return b, q2q1.assemble_q2q1(b)


def test_flat_box_mass_and_stiffness_closed_forms(flat):
    b, ops = flat
    x, y, z = ops.mesh.xyz2.T
    e = 0.3
    f = x * x
    g = y * z
    # int x^2 y z = (1/3)(1/2)(-e^2/2)
    assert f @ (ops.M2 @ g) == pytest.approx((1 / 3) * 0.5 * (-e * e / 2), rel=1e-13, abs=0)
    # int (x^2)^2 = (1/5) e
    assert f @ (ops.M2 @ f) == pytest.approx(e / 5, rel=1e-13, abs=0)
    h = x * x + 3 * y * z                      # grad = (2x, 3z, 3y)
    nu = b.nu
    exact = nu[0] * 4 * (1 / 3) * e + nu[1] * 9 * (e ** 3 / 3) + nu[2] * 9 * (1 / 3) * e
    assert h @ (ops.K2 @ h) == pytest.approx(exact, rel=1e-13, abs=0)
    # Q1: grad(xy) . grad(xz) = (y, x, 0) . (z, 0, x) = y z, and int y z = (1/2)(-e^2/2)
    X, Y, Z = ops.mesh.base.xyz.T
    assert (X * Y) @ (ops.K1 @ (X * Z)) == pytest.approx(0.5 * (-e * e / 2), rel=1e-13, abs=0)
    assert (X * Y) @ (ops.M1 @ Z) == pytest.approx(0.25 * (-e * e / 2), rel=1e-13, abs=0)


def test_flat_box_coupling_and_integration_by_parts(flat):
    b, ops = flat
    x, y, z = ops.mesh.xyz2.T
    X, Y, Z = ops.mesh.base.xyz.T
    e = 0.3
    # p' D_1 u = int y * d_x(x^2) = int 2 x y = (1)(1/2) e
    assert Y @ (ops.D[0] @ (x * x)) == pytest.approx(0.5 * e, rel=1e-13, abs=0)
    # p' D_3 u = int x * d_z(z^2) = (1/2) * (-e^2)
    assert X @ (ops.D[2] @ (z * z)) == pytest.approx(0.5 * (-e * e), rel=1e-13, abs=0)
    # u' B_2 q with u = x z (Q2) and q = y z (Q1, d_y q = z): int x z^2 = (1/2)(e^3/3)
    assert (x * z) @ (ops.B[1] @ (Y * Z)) == pytest.approx(0.5 * e ** 3 / 3, rel=1e-13, abs=0)
    # integration by parts: q' D_c u + u' B_c q = int_boundary q u n_c
    u = x * x + y * z
    q = 1.0 + X * Y
    # c = 1: faces x = 1 (n = +1) and x = 0 (n = -1): int_{x=1} (1 + y)(1 + y z) - int_{x=0} (1)(y z)
    bnd = (1.0 * e + 0.5 * e) + (0.5 * (-e * e / 2) + (1 / 3) * (-e * e / 2)) - 0.5 * (-e * e / 2)
    assert q @ (ops.D[0] @ u) + u @ (ops.B[0] @ q) == pytest.approx(bnd, rel=1e-13, abs=0)
    # c = 3: faces z = 0 (n = +1, u = x^2) and z = -e (n = -1, u = x^2 - e y)
    top = (1 / 3) + (1 / 3) * 0.5
    bot = ((1 / 3) - e * 0.5) + 0.5 * ((1 / 3) - e * (1 / 3))
    assert q @ (ops.D[2] @ u) + u @ (ops.B[2] @ q) == pytest.approx(top - bot, rel=1e-13, abs=0)


def _interior(mesh_xyz, L=(1.0, 1.0), D=1.0):
    x, y, z = mesh_xyz.T
    tol = 1e-12
    return (x > tol) & (x < L[0] - tol) & (y > tol) & (y < L[1] - tol) & (z > -D + tol) & (z < -tol)


def _mms_q2(nh):
    b = box_basin(nh=nh, nz=nh, eps=1.0, nu=(1.0, 1.0, 1.0))
    ops = q2q1.assemble_q2q1(b)
    hi = q2q1.element_quadrature(ops.mesh, 6)
    pts = np.einsum("qv,evi->eqi", q2q1.tensor_basis(q2q1.cube_rule(6)[0], 1)[0], ops.mesh.corners)
    us = lambda p: np.sin(np.pi * p[..., 0]) * np.sin(np.pi * p[..., 1]) * np.sin(np.pi * (p[..., 2] + 1))  # noqa
    f = (1.0 + 3 * np.pi ** 2) * us(pts)                       # (M + K) u* with nu = I
    load = np.zeros(ops.mesh.n2)
    np.add.at(load, ops.mesh.e2.ravel(), np.einsum("eq,eq,qb->eb", hi.dV, f, hi.phi2).ravel())
    A = (ops.M2 + ops.K2).tocsr()
    inner = _interior(ops.mesh.xyz2)
    u = np.zeros(ops.mesh.n2)
    u[inner] = spla.spsolve(A[inner][:, inner].tocsc(), load[inner])
    uh = np.einsum("qb,eb->eq", hi.phi2, u[ops.mesh.e2])
    return float(np.sqrt(np.sum(hi.dV * (uh - us(pts)) ** 2)))


def _mms_q1(nh):
    b = box_basin(nh=nh, nz=nh, eps=1.0, nu=(1.0, 1.0, 1.0))
    ops = q2q1.assemble_q2q1(b)
    hi = q2q1.element_quadrature(ops.mesh, 6)
    pts = np.einsum("qv,evi->eqi", q2q1.tensor_basis(q2q1.cube_rule(6)[0], 1)[0], ops.mesh.corners)
    us = lambda p: np.sin(np.pi * p[..., 0]) * np.sin(np.pi * p[..., 1]) * np.sin(np.pi * (p[..., 2] + 1))  # noqa
    f = (1.0 + 3 * np.pi ** 2) * us(pts)
    load = np.zeros(ops.mesh.n1)
    np.add.at(load, ops.mesh.e1.ravel(), np.einsum("eq,eq,qb->eb", hi.dV, f, hi.phi1).ravel())
    A = (ops.M1 + ops.K1).tocsr()
    inner = _interior(ops.mesh.base.xyz)
    p = np.zeros(ops.mesh.n1)
    p[inner] = spla.spsolve(A[inner][:, inner].tocsc(), load[inner])
    ph = np.einsum("qb,eb->eq", hi.phi1, p[ops.mesh.e1])
    return float(np.sqrt(np.sum(hi.dV * (ph - us(pts)) ** 2)))


def test_manufactured_solutions_converge_at_the_expected_orders():
    """(M + K) u = f on the unit cube, u* = sin(pi x) sin(pi y) sin(pi (z + 1)), u = 0 on the
    boundary: halving h divides the L2 error by about 8 for Q2 and 4 for Q1."""
    e2 = [_mms_q2(nh) for nh in (4, 7)]
    e1 = [_mms_q1(nh) for nh in (5, 9)]
    assert e2[0] / e2[1] > 6.5, e2
    assert 3.5 < e1[0] / e1[1] < 4.6, e1


def _gradient_field(nh):
    b = box_basin(nh=nh, nz=nh, eps=1.0, nu=(1.0, 1.0, 1.0))
    ops = q2q1.assemble_q2q1(b)
    x, y, z = ops.mesh.xyz2.T
    zz = z + 1.0
    pi = np.pi
    ut = np.stack([-pi * np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * zz),
                   -pi * np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * zz),
                   -pi * np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * zz)])
    return ops, ut


def _m_norm(ops, v):
    return float(np.sqrt(sum(v[c] @ (ops.M2 @ v[c]) for c in range(3))))


@pytest.mark.parametrize("lumped", [False, True])
def test_projection_removes_a_pure_gradient(lumped):
    """u~ = grad(phi), d phi / dn = 0: q ~ alpha phi and u = u~ - (1/alpha) grad q ~ 0, better
    under refinement; with the sign flipped, u would be about 2 u~."""
    ratios = []
    for nh in (4, 7):
        ops, ut = _gradient_field(nh)
        a = ops.alpha(False)
        _, res = q2q1.pressure_increment(ops, ut, False)
        u = q2q1.correct_velocity(ops, ut, res.x, a, lumped=lumped)
        ratios.append(_m_norm(ops, u) / _m_norm(ops, ut))
        flipped = q2q1.correct_velocity(ops, ut, -res.x, a, lumped=lumped)
        assert _m_norm(ops, flipped) / _m_norm(ops, ut) > 1.8
    # measured: 0.27 / 0.11 (consistent), 0.24 / 0.08 (lumped) on 3 and 6 bricks per side
    assert ratios[0] < 0.35 and ratios[1] < 0.15, ratios
    assert ratios[0] / ratios[1] > 2.2, ratios


def test_wind_driven_step_lowers_the_discrete_divergence():
    b = box_basin(nh=6, nz=4)
    th = np.zeros((2, b.ny, b.nx))
    Y = np.linspace(0.0, 1.0, b.ny)[:, None] * np.ones((1, b.nx))
    th[0] = -1e-4 * np.cos(np.pi * Y)
    b.theta = th
    ops = q2q1.assemble_q2q1(b)
    st = q2q1.initial_state(ops)
    for _ in range(2):
        rep = q2q1.project_step(ops, st)
        d_pred = np.linalg.norm(q2q1.discrete_divergence(ops, rep["u_tilde"]))
        d_corr = np.linalg.norm(q2q1.discrete_divergence(ops, st.u))
        assert d_corr < 0.6 * d_pred, (d_corr, d_pred)
        assert all(r.converged for r in rep["vel"]) and rep["pres"].converged
    assert abs(ops.m1 @ st.p) <= 1e-10 * np.abs(st.p).max() * ops.m1.sum()
    assert np.all(np.isfinite(st.u))
