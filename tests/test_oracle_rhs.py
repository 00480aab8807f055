"""Closed-form pins of the oracle's right-hand sides: the velocity prediction's (Eq.
fofa_velo_pred_h) term by term, and the pressure increment's (Eq. fofa_q_cor_h). Each term is
isolated on a uniform box where it has a closed form, so that a wrong BDF coefficient, a flipped
Coriolis sign, G in place of G^T or a wrong alpha fails here."""
import copy

import numpy as np
import pytest

from oracle import fem
from workloads import box_basin


@pytest.fixture(scope="module")
def ops():
    return fem.assemble(box_basin(nh=7, nz=6))


def interior(ops):
    """Nodes whose basis function vanishes on the whole boundary of the box."""
    m = ops.mesh
    k = np.arange(m.n) % m.nz
    col = np.arange(m.n) // m.nz
    i, j = m.col_i[col], m.col_j[col]
    return (k > 0) & (k < m.nz - 1) & (i > 0) & (i < m.nx - 1) & (j > 0) & (j < m.ny - 1)


def rhs(ops, uk=None, um=None, p=None, bdf1=False):
    z = np.zeros((3, ops.n))
    return fem.velocity_rhs(ops, z if uk is None else uk, z if um is None else um,
                            np.zeros(ops.n) if p is None else p, bdf1)


@pytest.mark.parametrize("case", ["bdf2_current", "bdf2_previous", "bdf1"])
def test_time_derivative_coefficients(ops, case):
    """Constant states: advection vanishes and b_c = coef * U * (M 1) / dt on the free rows, with
    coef = 2 (u^k) and -1/2 (u^{k-1}) for BDF2 and 1 for the BDF1 start."""
    U = 0.7
    one = np.full((3, ops.n), U)
    uk, um, bdf1, coef = {"bdf2_current": (one, None, False, 2.0), "bdf2_previous": (None, one, False, -0.5),
                          "bdf1": (one, 3.0 * one, True, 1.0)}[case]
    b = rhs(ops, uk, um, bdf1=bdf1)
    m1 = ops.m
    for c in range(3):
        free = ~ops.mesh.dirichlet[c]
        np.testing.assert_allclose(b[c][free], coef * U * m1[free] / ops.dt, rtol=1e-10)
        assert np.all(b[c][ops.mesh.dirichlet[c]] == 0.0)


def test_coriolis_deflects_to_the_right(ops):
    """-(2 Omega ^ u) with 2 Omega = f e3: (f u2, -f u1, 0). A uniform eastward flow in the
    northern hemisphere (f > 0) is pushed south."""
    f0, U1, U2 = 1e-4, 0.3, -0.2
    o = copy.copy(ops)
    o.coriolis = np.full(ops.n, f0)
    u = np.zeros((3, ops.n))
    u[0], u[1] = U1, U2
    b = rhs(o, u, bdf1=True)
    m1 = ops.m
    hist = u / ops.dt
    expect = [hist[0] + f0 * U2, hist[1] - f0 * U1, hist[2]]
    for c in range(3):
        free = ~ops.mesh.dirichlet[c]
        np.testing.assert_allclose(b[c][free], expect[c][free] * m1[free], rtol=1e-10, atol=1e-18)
    # the Coriolis part alone, for u = (U1, 0, 0)
    u[1] = 0.0
    b0 = rhs(ops, u, bdf1=True)
    b1 = rhs(o, u, bdf1=True)
    free = ~ops.mesh.dirichlet[1]
    d = (b1[1] - b0[1])[free]
    assert np.all(d < 0.0)
    np.testing.assert_allclose(d, -f0 * U1 * m1[free], rtol=1e-10)


@pytest.mark.parametrize("c", [0, 1, 2])
def test_pressure_term_is_g_transpose(ops, c):
    """(G_c^T p)_i = int p d_c phi_i. For p = x_c this is -int phi_i = -(M 1)_i at interior nodes
    (the boundary term vanishes there); G_c p would give +(M 1)_i. Other components see 0."""
    inner = interior(ops)
    assert inner.sum() > 10
    p = ops.mesh.xyz[:, c].copy()
    b = rhs(ops, p=p)
    m1 = ops.m
    for d in range(3):
        want = -m1[inner] if d == c else np.zeros(inner.sum())
        np.testing.assert_allclose(b[d][inner], want, rtol=1e-10, atol=1e-12 * m1.max())
    # a constant pressure exerts no force on interior nodes
    b = rhs(ops, p=np.ones(ops.n))
    for d in range(3):
        np.testing.assert_allclose(b[d][inner], 0.0, atol=1e-12 * m1.max())


def test_wind_tension_on_the_surface(ops):
    """int_{Gamma_s} theta phi_i = theta dx dy at interior surface nodes of a uniform grid (each
    such node is a vertex of six surface triangles of area dx dy / 2); u3 gets no tension, and
    nodes below the surface get none."""
    m = ops.mesh
    o = copy.copy(ops)
    t1, t2 = 2e-5, -3e-5
    o.theta = np.stack([np.full(ops.n, t1), np.full(ops.n, t2)])
    b = rhs(o)
    k = np.arange(m.n) % m.nz
    col = np.arange(m.n) // m.nz
    i, j = m.col_i[col], m.col_j[col]
    top_inner = (k == m.nz - 1) & (i > 0) & (i < m.nx - 1) & (j > 0) & (j < m.ny - 1)
    np.testing.assert_allclose(b[0][top_inner], t1 * m.dx * m.dy, rtol=1e-12)
    np.testing.assert_allclose(b[1][top_inner], t2 * m.dx * m.dy, rtol=1e-12)
    assert np.all(b[2] == 0.0)
    assert np.all(b[0][k < m.nz - 1] == 0.0) and np.all(b[1][k < m.nz - 1] == 0.0)


@pytest.mark.parametrize("bdf1", [False, True])
def test_divergence_rhs(ops, bdf1):
    """b_p = -alpha sum_c G_c u~_c, alpha = 3/(2 dt) (BDF2) or 1/dt (BDF1). For u~ = x_c e_c the
    divergence is 1 everywhere, so b_p = -alpha M 1 on every node; u~ = x_d e_c (d != c) is
    divergence-free and gives 0."""
    alpha = 1.0 / ops.dt if bdf1 else 1.5 / ops.dt
    m1 = ops.m
    for c in range(3):
        u = np.zeros((3, ops.n))
        u[c] = ops.mesh.xyz[:, c]
        np.testing.assert_allclose(fem.divergence_rhs(ops, u, bdf1), -alpha * m1, rtol=1e-10)
        u[c] = ops.mesh.xyz[:, (c + 1) % 3]
        np.testing.assert_allclose(fem.divergence_rhs(ops, u, bdf1), 0.0, atol=1e-10 * alpha * m1.max())
