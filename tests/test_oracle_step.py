"""Pins of the oracle's projection (Section 3, Eqs. correc_velo_u, press_cor; Section 5, Eqs.
fofa_q_cor_h, fofa_velo_cor_h): the sign of the velocity correction and what the correction is
for, removing the gradient part of the prediction.

Continuous fact used: for u~ = grad(phi) with d phi / dn = 0 on the boundary, Eq. press_cor gives
q = (3 / (2 dt)) phi and Eq. correc_velo_u gives u = u~ - (2 dt / 3) grad q = 0. The discrete
projection removes grad(phi) up to the discretisation error, which falls as the mesh is refined.
A correction with the opposite sign returns about 2 grad(phi) instead.
"""
import numpy as np
import pytest

from oracle import fem, step
from workloads import box_basin


def _cube_gradient_field(nh):
    """P1 interpolant of grad(phi), phi = cos(pi x) cos(pi y) cos(pi (z + 1)) on [0,1]^2 x [-1,0]."""
    ops = fem.assemble(box_basin(nh=nh, nz=nh, eps=1.0))
    x, y, z = ops.mesh.xyz.T
    zz = z + 1.0
    pi = np.pi
    ut = np.stack([-pi * np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * zz),
                   -pi * np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * zz),
                   -pi * np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * zz)])
    return ops, ut


def _m_norm(ops, v):
    return float(np.sqrt(sum(v[c] @ (ops.M @ v[c]) for c in range(3))))


def _project(ops, ut, lumped, bdf1=False):
    o = step.StepOptions(vel_rtol=1e-12, pres_rtol=1e-12, lumped_correction=lumped)
    _, res = step.pressure_increment(ops, ut, bdf1, None, o)
    u, _ = step.correct_velocity(ops, ut, res.x, ops.alpha(bdf1), o)
    return u, res.x


@pytest.mark.parametrize("lumped", [False, True])
def test_projection_removes_a_pure_gradient(lumped):
    """||u||_M / ||u~||_M after one projection of grad(phi): small, and falling under refinement
    (it would be close to 2 with the correction's sign flipped)."""
    ratios = []
    for nh in (9, 17):
        ops, ut = _cube_gradient_field(nh)
        u, _ = _project(ops, ut, lumped)
        ratios.append(_m_norm(ops, u) / _m_norm(ops, ut))
    bound = (0.2, 0.07) if lumped else (0.12, 0.04)
    assert ratios[0] < bound[0] and ratios[1] < bound[1], ratios
    assert ratios[0] / ratios[1] > 2.5, ratios


@pytest.mark.parametrize("bdf1", [True, False])
def test_pressure_increment_is_alpha_phi(bdf1):
    """q approximates alpha * (phi - its mean) (Eq. press_cor with u~ = grad phi); alpha = 1/dt on
    the BDF1 start step and 3/(2 dt) after."""
    ops, ut = _cube_gradient_field(17)
    _, q = _project(ops, ut, lumped=False, bdf1=bdf1)
    x, y, z = ops.mesh.xyz.T
    phi = np.cos(np.pi * x) * np.cos(np.pi * y) * np.cos(np.pi * (z + 1.0))
    m = ops.m
    phi0 = phi - (m @ phi) / m.sum()
    a = ops.alpha(bdf1)
    assert np.linalg.norm(q - a * phi0) <= 0.03 * np.linalg.norm(a * phi0)


@pytest.mark.parametrize("lumped", [False, True])
def test_correction_lowers_the_discrete_divergence(lumped):
    """sum_c G_c u_c (the integral of div u against each basis function) is smaller after the
    correction than for the prediction: on the cube for the pure gradient, and after a
    wind-driven step of the 16 x 16 x 8 box, Dirichlet sets included."""
    ops, ut = _cube_gradient_field(9)
    u, _ = _project(ops, ut, lumped)
    d0 = np.linalg.norm(step.discrete_divergence(ops, ut))
    d1 = np.linalg.norm(step.discrete_divergence(ops, u))
    assert d1 < 0.35 * d0, (d1, d0)

    b = box_basin()
    th = np.zeros((2, b.ny, b.nx))
    Y = np.linspace(0.0, 1.0, b.ny)[:, None] * np.ones((1, b.nx))
    th[0] = -1e-4 * np.cos(np.pi * Y)
    b.theta = th
    ops = fem.assemble(b)
    st = step.initial_state(ops.n)
    rep = step.project_step(ops, st, step.StepOptions(vel_rtol=1e-12, pres_rtol=1e-12,
                                                      lumped_correction=lumped))
    d_pred = np.linalg.norm(step.discrete_divergence(ops, rep.u_tilde))
    d_corr = np.linalg.norm(step.discrete_divergence(ops, st.u))
    assert d_corr < 0.6 * d_pred, (d_corr, d_pred)


def test_diagnostics_closed_forms():
    """Kinetic energy of a uniform flow is |U|^2 |Omega| / 2 (|Omega| = 1 x 1 x eps for the box);
    a linear field (x, y, -2z) is divergence free and G_c X_d = delta_cd M 1 makes its discrete
    divergence vanish; (x, 0, 0) has sum_c G_c u_c = M 1; a constant pressure is its own mean."""
    b = box_basin(nh=7, nz=5, eps=0.01)
    ops = fem.assemble(b)
    st = step.initial_state(ops.n)
    st.u[0], st.u[1], st.u[2] = 0.3, -0.4, 1.2
    st.p[:] = 2.5
    d = step.diagnostics(ops, st)
    assert d["kinetic_energy"] == pytest.approx(0.5 * (0.09 + 0.16 + 1.44) * 0.01, rel=1e-12, abs=0)
    assert d["p_mean"] == pytest.approx(2.5, rel=1e-14, abs=0)
    x, y, z = ops.mesh.xyz.T
    st.u = np.stack([x, y, -2.0 * z])
    d = step.diagnostics(ops, st, u_tilde=np.stack([x, 0 * x, 0 * x]))
    assert d["div_u"] <= 1e-13 * np.linalg.norm(ops.m)
    assert d["div_u_tilde"] == pytest.approx(np.linalg.norm(ops.m), rel=1e-12, abs=0)
