"""Pins of the oracle's compensated residual and of its FP64 acceptance floor, against exact
rational arithmetic (fractions.Fraction: every float is a rational, and sums and products of
rationals are exact).

- TwoSum and TwoProduct are error-free: s + e == a + b and p + e == a * b exactly.
- residual_dot2 (Dot2 of Ogita, Rump and Oishi, applied per row) equals b - A x computed exactly,
  to about one rounding of the result, on rows built so that the plain FP64 residual is mostly
  rounding noise.
- The floor u (|A||x| + |b|) bounds, row by row, the exact residual of the correctly rounded
  solution of a small ill-conditioned system; the oracle's PCG, asked for a residual below that
  floor, stops once restarts stall and reports the exact residual it reached.
"""
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import fem, pcg
from workloads import box_basin

U = 2.0 ** -53


def _fr(v):
    return [Fraction(float(t)) for t in np.ravel(v)]


def _wide_floats(rng, n, emin=-300, emax=300):
    return rng.standard_normal(n) * np.exp2(rng.integers(emin, emax, n).astype(float))


def test_two_sum_is_error_free():
    rng = np.random.default_rng(1)
    a = _wide_floats(rng, 4000, -60, 60)
    b = _wide_floats(rng, 4000, -60, 60)
    s, e = pcg.two_sum(a, b)
    for ai, bi, si, ei in zip(_fr(a), _fr(b), _fr(s), _fr(e)):
        assert si + ei == ai + bi
    # e is the rounding error of s: at most half an ulp of s
    assert np.all(np.abs(e) <= np.spacing(np.abs(s)) / 2)


def test_two_product_is_error_free():
    rng = np.random.default_rng(2)
    a = _wide_floats(rng, 4000, -200, 200)
    b = _wide_floats(rng, 4000, -200, 200)
    p, e = pcg.two_product(a, b)
    for ai, bi, pi, ei in zip(_fr(a), _fr(b), _fr(p), _fr(e)):
        assert pi + ei == ai * bi
    assert np.all(np.abs(e) <= np.spacing(np.abs(p)) / 2)


def _exact_residual(A, x, b):
    A = A.tocsr()
    xs = _fr(x)
    out = []
    for i in range(A.shape[0]):
        acc = Fraction(float(b[i]))
        for k in range(A.indptr[i], A.indptr[i + 1]):
            acc -= Fraction(float(A.data[k])) * xs[A.indices[k]]
        out.append(acc)
    return out


def test_residual_dot2_is_exact_to_one_rounding():
    """Rows whose terms cancel to 1e-12 of their size: b_i is the exactly rounded value of
    sum_j a_ij x_j plus a tiny offset, so the true residual is tiny and the plain FP64 residual is
    mostly rounding noise, while Dot2 gets it to about one rounding."""
    rng = np.random.default_rng(3)
    n = 60
    A = sp.random(n, n, density=0.2, random_state=4, format="csr") + sp.eye(n) * 3.0
    A.data *= np.exp2(rng.integers(-20, 20, A.nnz).astype(float))
    x = rng.standard_normal(n) * 1e3
    exact_ax = _exact_residual(A, x, np.zeros(n))          # -(A x) exactly
    b = np.array([-float(v) for v in exact_ax])            # correctly rounded A x
    b *= 1.0 + 1e-12 * rng.standard_normal(n)              # leave a small true residual
    r_exact = _exact_residual(A, x, b)
    r2 = pcg.residual_dot2(A, x, b)
    r_plain = b - A @ x
    ax_abs = abs(A) @ np.abs(x)
    err2 = [abs(Fraction(float(r2[i])) - r_exact[i]) for i in range(n)]
    for i in range(n):
        # one rounding of the result plus a second-order term of the cancelled size
        assert err2[i] <= Fraction(2 * U) * abs(r_exact[i]) + Fraction(1e-30) * Fraction(float(ax_abs[i])), i
    err_plain = max(float(abs(Fraction(float(r_plain[i])) - r_exact[i]) / abs(r_exact[i])) for i in range(n))
    assert err_plain > 1e-3            # the plain residual is not even the right order in some row


def test_floor_on_a_hand_computed_example():
    """A = [[4, -1], [-1, 4]], x = (1, -2), b = (1, 1): |A||x| + |b| = (4 + 2 + 1, 1 + 8 + 1) =
    (7, 10), so the floor is 2^-53 sqrt(49 + 100) / sqrt(2) = 2^-53 sqrt(74.5)."""
    A = sp.csr_matrix(np.array([[4.0, -1.0], [-1.0, 4.0]]))
    got = pcg.residual_floor(A, np.array([1.0, -2.0]), np.array([1.0, 1.0]))
    assert got / 2.0 ** -53 == pytest.approx(8.631338250816034, rel=1e-15)


def _exact_solve(A, b):
    """x = A^{-1} b by Gaussian elimination in rationals (small dense SPD A)."""
    n = A.shape[0]
    M = [[Fraction(float(v)) for v in row] + [Fraction(float(b[i]))] for i, row in enumerate(A.toarray())]
    for k in range(n):
        piv = M[k][k]
        for i in range(k + 1, n):
            f = M[i][k] / piv
            if f:
                for j in range(k, n + 1):
                    M[i][j] -= f * M[k][j]
    x = [Fraction(0)] * n
    for i in range(n - 1, -1, -1):
        acc = M[i][n] - sum(M[i][j] * x[j] for j in range(i + 1, n))
        x[i] = acc / M[i][i]
    return x


@pytest.fixture(scope="module")
def thin_system():
    """The u1 prediction operator of a 4 x 4 x 4 box 1e-3 deep (nu = (1, 1, 1e-6)): a small SPD
    system whose couplings differ by six orders of magnitude."""
    ops = fem.assemble(box_basin(nh=4, nz=4, eps=1e-3, nu=(1.0, 1.0, 1e-6)))
    A = ops.A_u(0)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(ops.n)
    b[ops.mesh.dirichlet[0]] = 0.0
    return A, b, _exact_solve(A, b)


def test_floor_bounds_the_residual_of_the_rounded_solution(thin_system):
    A, b, xs = thin_system
    x = np.array([float(v) for v in xs])                   # correctly rounded x*
    r = _exact_residual(A, x, b)
    bound = U * (abs(A) @ np.abs(x))
    for i in range(len(b)):
        assert abs(r[i]) <= Fraction(float(bound[i])) * (1 + Fraction(4 * U)), i
    floor = U * np.linalg.norm(abs(A) @ np.abs(x) + np.abs(b)) / np.linalg.norm(b)
    rel = float(np.sqrt(float(sum(v * v for v in r)))) / np.linalg.norm(b)
    assert rel <= floor


def test_pcg_stops_at_the_floor_and_reports_the_exact_residual(thin_system):
    A, b, xs = thin_system
    res = pcg.pcg(A, b, rtol=1e-18, precond=pcg.jacobi_preconditioner(A), max_restarts=6)
    assert res.converged and res.rel_res_true > 1e-18 and res.rel_res_true <= res.rel_res_floor
    r = _exact_residual(A, res.x, b)
    rel_exact = float(np.sqrt(float(sum(v * v for v in r)))) / np.linalg.norm(b)
    assert res.rel_res_true == pytest.approx(rel_exact, rel=1e-6)
    # and it is within a small factor of the best any FP64 vector does (the rounded x*)
    x_best = np.array([float(v) for v in xs])
    rb = _exact_residual(A, x_best, b)
    rel_best = float(np.sqrt(float(sum(v * v for v in rb)))) / np.linalg.norm(b)
    # restarts carry on while they halve it: the first pass alone stops about 3x higher here
    assert rel_exact <= 1.5 * rel_best
    err = max(abs(float(Fraction(float(res.x[i])) - xs[i])) for i in range(len(b))) / max(abs(float(v)) for v in xs)
    assert err <= 1e-6
