"""Pins of the oracle's PCG, preconditioners and projection step (CPU only)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fem, pcg, step
from workloads import box_basin, random_vector
from test_oracle_fem import small_basin


@pytest.fixture(scope="module")
def tiny():
    return fem.assemble(box_basin(nh=4, nz=4))


@pytest.fixture(scope="module")
def basin():
    return fem.assemble(small_basin())


def _rhs(ops, c, seed):
    b = random_vector(ops.n, seed)
    if c is not None:
        b[ops.mesh.dirichlet[c]] = 0.0
    return b


@pytest.mark.parametrize("prec", ["jacobi", "ic0", "ic0_natural", "none"])
@pytest.mark.parametrize("which", ["tiny", "basin"])
def test_pcg_matches_dense_cholesky(prec, which, tiny, basin):
    ops = tiny if which == "tiny" else basin
    for c in range(3):
        A = ops.A_u(c, bdf1=(c == 1))
        b = _rhs(ops, c, 10 + c)
        P = {"jacobi": lambda: pcg.jacobi_preconditioner(A),
             "ic0": lambda: pcg.ic0_preconditioner(A, ops.mesh.colour)[0],
             "ic0_natural": lambda: pcg.ic0_preconditioner(A)[0],
             "none": lambda: None}[prec]()
        res = pcg.pcg(A, b, rtol=1e-14, precond=P, max_iter=20000)
        x = pcg.dense_cholesky_solve(A, b)
        assert np.linalg.norm(res.x - x) <= 1e-11 * np.linalg.norm(x), (prec, c)


@pytest.mark.parametrize("which", ["tiny", "basin"])
def test_pressure_matches_dense_augmented_system(which, tiny, basin):
    ops = tiny if which == "tiny" else basin
    b = _rhs(ops, None, 7)          # inconsistent on purpose: the multiplier absorbs 1'b
    res = pcg.pressure_solve(ops.K_I, ops.m, b, rtol=1e-12, max_iter=50000)
    x = pcg.dense_augmented_solve(ops.K_I, ops.m, b)
    assert abs(ops.m @ res.x) <= 1e-12 * np.linalg.norm(x) * ops.m.sum()
    assert np.linalg.norm(res.x - x) <= 1e-10 * np.linalg.norm(x)


def _pattern_check(A, f):
    """(L L^T)_ij == A_ij on the pattern of lower(P A P^T)."""
    LLt = (f.factor_matrix() @ f.factor_matrix().T).tocsr()
    low = f.lower.tocoo()
    got = np.asarray(LLt[low.row, low.col]).ravel()
    return np.max(np.abs(got - low.data)) / np.abs(low.data).max()


def test_ic0_defining_property(basin):
    for c in range(3):
        A = basin.A_u(c)
        for colour in (basin.mesh.colour, None):
            _, f = pcg.ic0_preconditioner(A, colour)
            assert f.shift == 0.0
            assert _pattern_check(A, f) <= 1e-13


def test_ic0_mmatrix_no_breakdown():
    """Pure stiffness of a cube-cell mesh (non-obtuse Kuhn tets: an M-matrix) with a Dirichlet face."""
    b = box_basin(nh=6, nz=6, eps=1.0)         # dx = dy = 0.2, dz = 0.2: cubes
    b.depth[:] = 1.0
    ops = fem.assemble(b)
    K = fem.eliminate_dirichlet(ops.K_I, ops.mesh.gamma0)
    off = K - sp.diags(K.diagonal())
    assert off.max() <= 1e-15                  # M-matrix: non-positive off-diagonals
    for colour in (ops.mesh.colour, None):
        _, f = pcg.ic0_preconditioner(K, colour)
        assert f.shift == 0.0
        assert _pattern_check(K, f) <= 1e-13
        Lm = f.factor_matrix().toarray()
        assert np.all(np.diag(Lm) > 0)


def test_ic0_is_exact_on_a_tridiagonal_matrix():
    """IC(0) of a tridiagonal SPD matrix has no dropped fill: it is the exact Cholesky factor."""
    n = 50
    A = sp.diags([-np.ones(n - 1), 2.5 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")
    _, f = pcg.ic0_preconditioner(A, None)
    L = np.linalg.cholesky(A.toarray())
    np.testing.assert_allclose(f.factor_matrix().toarray(), L, atol=1e-14)
    r = np.random.default_rng(1).standard_normal(n)
    np.testing.assert_allclose(f.apply(r), np.linalg.solve(A.toarray(), r), rtol=1e-12)


def _scipy_cg_iters(A, b, Pfun, rtol):
    count = [0]

    def cb(xk):
        count[0] += 1
    Mop = spla.LinearOperator(A.shape, matvec=Pfun) if Pfun is not None else None
    try:
        spla.cg(A, b, rtol=rtol, atol=0.0, M=Mop, maxiter=100000, callback=cb)
    except TypeError:  # older scipy
        spla.cg(A, b, tol=rtol, atol=0.0, M=Mop, maxiter=100000, callback=cb)
    return count[0]


@pytest.mark.parametrize("prec", ["jacobi", "ic0"])
def test_iteration_counts_match_scipy_cg(prec):
    ops = fem.assemble(box_basin())
    for c in range(3):
        A = ops.A_u(c, bdf1=True)
        b = _rhs(ops, c, 100 + c)
        P = pcg.jacobi_preconditioner(A) if prec == "jacobi" else pcg.ic0_preconditioner(A, ops.mesh.colour)[0]
        res = pcg.pcg(A, b, rtol=1e-10, precond=P)
        assert res.restarts == 0
        it = _scipy_cg_iters(A, b, P, 1e-10)
        assert abs(res.iters - it) <= 1, (c, res.iters, it)


def test_lanczos_spectrum_bounds():
    """CG's alpha/beta define a Lanczos tridiagonal whose extreme eigenvalues lie inside the
    spectrum of the (Jacobi-preconditioned) operator and approach its ends."""
    ops = fem.assemble(box_basin(nh=6, nz=4))
    A = ops.A_u(0, bdf1=True)
    b = _rhs(ops, 0, 3)
    P = pcg.jacobi_preconditioner(A)
    res = pcg.pcg(A, b, rtol=1e-12, precond=P, record=True)
    al, be = np.array(res.alphas), np.array(res.betas)
    k = len(al)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
    ev = np.linalg.eigvalsh(T)
    d = A.diagonal()
    S = A.toarray() / np.sqrt(np.outer(d, d))
    keep = ~ops.mesh.dirichlet[0]
    evA = np.linalg.eigvalsh(S[np.ix_(keep, keep)])
    assert ev.min() >= evA.min() * (1 - 1e-8) and ev.max() <= evA.max() * (1 + 1e-8)
    assert ev.max() >= 0.99 * evA.max()


def test_step_rest_stays_at_rest():
    b = box_basin()
    ops = fem.assemble(b)
    st = step.initial_state(ops.n)
    for _ in range(2):
        rep = step.project_step(ops, st)
        assert np.all(st.u == 0) and np.all(st.p == 0)
        assert all(r.iters == 0 for r in rep.vel)


def test_step_wind_driven_box():
    """One wind-driven step: solves converge, q has zero mean, boundary sets hold."""
    b = box_basin()
    th = np.zeros((2, b.ny, b.nx))
    X, Y = np.meshgrid(np.linspace(0, 1, b.nx), np.linspace(0, 1, b.ny))
    th[0] = -np.cos(np.pi * Y) * 1e-4
    b.theta = th
    ops = fem.assemble(b)
    st = step.initial_state(ops.n)
    for k in range(3):
        rep = step.project_step(ops, st, step.StepOptions(vel_rtol=1e-10, pres_rtol=1e-10))
        for r in rep.vel:
            assert r.converged
        assert rep.pres.converged
        assert abs(ops.m @ st.q) <= 1e-12 * np.abs(st.q).max() * ops.m.sum()
        for c in range(3):
            assert np.all(st.u[c][ops.mesh.dirichlet[c]] == 0.0)
    assert np.abs(st.u[0]).max() > 0


def test_step_consistent_vs_lumped_correction():
    b = small_basin()
    ops = fem.assemble(b)
    s1, s2 = step.initial_state(ops.n), step.initial_state(ops.n)
    step.project_step(ops, s1, step.StepOptions(vel_rtol=1e-12, pres_rtol=1e-12))
    step.project_step(ops, s2, step.StepOptions(vel_rtol=1e-12, pres_rtol=1e-12, lumped_correction=False))
    # same prediction and pressure; the corrections differ by the mass-lumping error only
    np.testing.assert_allclose(s1.p, s2.p, rtol=1e-9, atol=1e-12 * np.abs(s1.p).max())
    d = np.linalg.norm(s1.u - s2.u) / np.linalg.norm(s2.u)
    assert d < 0.5


def _line_block_matrix(A, nz):
    """The block diagonal of A made of each column's entries with |dk| <= 1 (scipy, no Thomas)."""
    C = A.tocoo()
    keep = (C.row // nz == C.col // nz) & (np.abs(C.row - C.col) <= 1)
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)


@pytest.mark.parametrize("which", ["vel", "pres"])
def test_line_preconditioner_solves_the_column_blocks(which, basin):
    nz = basin.mesh.nz
    A = basin.A_u(0) if which == "vel" else basin.K_I
    P = _line_block_matrix(A, nz)
    apply = pcg.line_preconditioner(A, nz)
    r = random_vector(basin.n, 8)
    z = apply(r)
    assert np.linalg.norm(P @ z - r) <= 1e-12 * np.linalg.norm(r)
    z2 = spla.spsolve(P.tocsc(), r)
    assert np.linalg.norm(z - z2) <= 1e-10 * np.linalg.norm(z2)


def test_line_preconditioner_is_exact_on_a_block_diagonal_matrix(basin):
    """If A has no coupling between columns, line-preconditioned CG converges in one step."""
    P = _line_block_matrix(basin.A_u(2), basin.mesh.nz)
    b = _rhs(basin, 2, 9)
    res = pcg.pcg(P, b, rtol=1e-12, precond=pcg.line_preconditioner(P, basin.mesh.nz))
    assert res.iters == 1


def test_line_iteration_counts_match_scipy_cg():
    ops = fem.assemble(box_basin())
    for A, c in ((ops.A_u(0, True), 0), (ops.K_I, None)):
        b = _rhs(ops, c, 41)
        if c is None:
            b = b - b.sum() / ops.m.sum() * ops.m
        P = pcg.line_preconditioner(A, ops.mesh.nz)
        res = pcg.pcg(A, b, rtol=1e-9, precond=P, max_restarts=0)
        it = _scipy_cg_iters(A, b, P, 1e-9)
        assert abs(res.first_pass_iters - it) <= 1, (res.first_pass_iters, it)


def test_manufactured_right_hand_sides_recover_their_field():
    """The small-case benchmark's manufactured solves (b = A u* for the seeded sinusoid field of
    workloads.manufactured_field): on the 16 x 16 x 8 box the oracle's PCG to 1e-10 returns u*
    for the velocity system (Dirichlet rows are identity rows, so u* is the exact solution) and
    u* minus its M-weighted mean for the pure-Neumann pressure system."""
    from oracle import fem, pcg as opcg
    from workloads import box_basin, manufactured_field, mms_modes
    b = box_basin()
    ops = fem.assemble(b)
    us = manufactured_field(b, ops.mesh.col_i, ops.mesh.col_j, mms_modes())
    assert us.shape == (ops.n,) and np.abs(us).max() > 0.1
    # the field at one node, by hand: column (i, j) = (3, 5), level k = 2
    i, j, k = 3, 5, 2
    s = 1.0 - k / (b.nz - 1)
    want = sum(a * np.sin(m * np.pi * i / 15) * np.sin(l * np.pi * j / 15) for a, m, l in mms_modes())
    assert us[(j * 16 + i) * b.nz + k] == pytest.approx(want * np.cos(0.5 * np.pi * s), rel=1e-13)
    A = ops.A_u(0)
    x = opcg.pcg(A, A @ us, rtol=1e-10, precond=opcg.jacobi_preconditioner(A)).x
    assert np.linalg.norm(x - us) <= 1e-7 * np.linalg.norm(us)
    K = ops.K_I
    m = ops.m
    q = opcg.pressure_solve(K, m, K @ us, rtol=1e-10, precond=opcg.jacobi_preconditioner(K)).x
    u0 = us - (m @ us) / m.sum()
    assert np.linalg.norm(q - u0) <= 1e-6 * np.linalg.norm(u0)
