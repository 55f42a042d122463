"""Pins of the oracle's DOP853 integrator (the paper's DOP 8 / DOP 8(5) solvers,
Sec. Functionalities) to facts fixed outside the oracle:

- the Butcher order conditions, enumerated here from rooted trees and evaluated
  in exact rational arithmetic on the oracle's own (double) tableau: order 8 for
  the propagated weights, order 5 and 3 for the two embedded weight sets;
- the closed-form nodes of the DOP853 construction;
- the stability polynomial on the harmonic oscillator (one step is an exact
  multiplication in the complex plane) and on the inverted oscillator's
  Lyapunov spectrum;
- 8th-order convergence under step halving on Henon-Heiles;
- SciPy's independent DOP853 implementation, run at a forced fixed step, and
  run adaptively step by step against the oracle's controller.
"""
from fractions import Fraction
from functools import lru_cache

import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import uniform_vectors


# --------------------------------------------------------------------------
# rooted trees and order conditions
# --------------------------------------------------------------------------

@lru_cache(None)
def _trees(n):
    """All rooted trees with n vertices; a tree is the sorted tuple of its
    root's subtrees."""
    if n == 1:
        return ((),)
    out = set()

    def forests(rem, largest):
        # multisets of subtrees with rem vertices in total, in non-increasing order
        if rem == 0:
            yield ()
            return
        for m in range(rem, 0, -1):
            for t in _trees(m):
                key = (m, t)
                if largest is not None and key > largest:
                    continue
                for rest in forests(rem - m, key):
                    yield (t,) + rest

    for f in forests(n - 1, None):
        out.add(tuple(sorted(f)))
    return tuple(sorted(out))


def _order(t):
    return 1 + sum(_order(s) for s in t)


def _gamma(t):
    g = _order(t)
    for s in t:
        g *= _gamma(s)
    return g


def _worst_residuals(a, b, max_order):
    """max over trees of each order of |sum_i b_i Phi_i(t) - 1/gamma(t)|, exact
    in rationals on the given (double) coefficients."""
    s = len(b)
    A = [[Fraction(float(a[i, j])) for j in range(s)] for i in range(s)]
    B = [Fraction(float(x)) for x in b]

    @lru_cache(None)
    def phi(t):
        v = [Fraction(1)] * s
        for sub in t:
            ps = phi(sub)
            av = [sum(A[i][j] * ps[j] for j in range(i)) for i in range(s)]
            v = [v[i] * av[i] for i in range(s)]
        return tuple(v)

    worst = {}
    for n in range(1, max_order + 1):
        worst[n] = max(abs(float(sum(B[i] * p for i, p in enumerate(phi(t))) - Fraction(1, _gamma(t))))
                       for t in _trees(n))
    return worst


def test_tree_enumeration_counts():
    # number of rooted trees with n vertices (Cayley; OEIS A000081)
    assert [len(_trees(n)) for n in range(1, 10)] == [1, 1, 2, 4, 9, 20, 48, 115, 286]
    assert _gamma(((), ())) == 3 and _gamma((((),),)) == 6


def test_dop853_order_conditions():
    a, b, e5, b3 = O.dop853_tableau()
    assert np.all(np.triu(a) == 0)
    w = _worst_residuals(a, b, 9)
    for n in range(1, 9):          # all 200 conditions of orders 1..8
        assert w[n] < 2e-15, (n, w[n])
    assert w[9] > 1e-6             # and not order 9
    w5 = _worst_residuals(a, b - e5, 6)
    for n in range(1, 6):
        assert w5[n] < 2e-15, (n, w5[n])
    assert w5[6] > 1e-5
    w3 = _worst_residuals(a, b3, 4)
    for n in range(1, 4):
        assert w3[n] < 2e-15, (n, w3[n])
    assert w3[4] > 1e-3
    # the 3rd-order weights use stages 1, 9 and 12 only
    assert set(np.nonzero(b3)[0]) == {0, 8, 11}
    assert set(np.nonzero(b)[0]) == {0, 5, 6, 7, 8, 9, 10, 11}


def test_dop853_nodes_closed_forms():
    """Nodes of the DOP853 construction: c4, c5 = (6 -+ sqrt 6)/30,
    c3 = 2 c4 / 3, c2 = 4 c4 / 9, then 1/3, 1/4, 4/13, 127/195, 3/5, 6/7, 1."""
    a, _, _, _ = O.dop853_tableau()
    c = a.sum(axis=1)
    r6 = np.sqrt(6.0)
    c4 = (6 - r6) / 30
    want = [0, 4 * c4 / 9, 2 * c4 / 3, c4, (6 + r6) / 30, 1 / 3, 1 / 4, 4 / 13, 127 / 195,
            3 / 5, 6 / 7, 1]
    np.testing.assert_allclose(c, want, rtol=0, atol=2e-15)


def _stability_poly(h):
    """R(w) = 1 + sum_q w^q b^T A^(q-1) 1 of the oracle's tableau (A nilpotent)."""
    a, b, _, _ = O.dop853_tableau()
    coef, v = [1.0], np.ones(12)
    for _ in range(12):
        coef.append(float(b @ v))
        v = a @ v
    return lambda w: sum(cq * w**q for q, cq in enumerate(coef)), coef


def test_dop853_stability_polynomial_on_harmonic_oscillator():
    R, coef = _stability_poly(0.0)
    from math import factorial
    np.testing.assert_allclose(coef[:9], [1 / factorial(q) for q in range(9)], rtol=0, atol=1e-15)
    S = O.system(O.HARMONIC, 1)
    h, n = 0.25, 400
    prm = O.params(h, n, n_dev=1, renorm=False, sample_every=0, integrator=O.DOP853)
    ens = O.Ensemble(S, prm, np.array([[0.3], [-0.7]]), w_in=np.array([[1.0], [0.5]]))
    ens.integrate(prm)
    g = R(-1j * h) ** n
    zx, zw = g * (0.3 - 0.7j), g * (1.0 + 0.5j)
    assert abs(complex(ens.x[0, 0], ens.x[1, 0]) - zx) < 1e-13
    assert abs(complex(ens.w[0, 0], ens.w[1, 0]) - zw) < 1e-13
    # and 8th order against the exact rotation
    ex = (0.3 - 0.7j) * np.exp(-1j * h * n)
    assert abs(zx - ex) < 2e-7


def test_dop853_lyapunov_inverted_oscillator_closed_form():
    """The inverted-oscillator spectrum (see the RK4 pin) with the DOP853
    stability polynomial in place of RK4's."""
    R, _ = _stability_poly(0.0)
    S = O.system(O.INVERTED, 2)
    h, n = 0.05, 400
    T = n * h
    lam, st = O.lyapunov(S, O.params(h, n, qr_every=10, integrator=O.DOP853),
                         np.array([[0.1], [0.2], [0.3], [-0.1]]))
    a, b = R(h), R(-h)
    rho = abs(R(1j * h))
    l1 = (2 * n * np.log(a) + np.log1p((b / a) ** (2 * n)) - np.log(2.0)) / (2 * T)
    l3 = n * np.log(a * b) / T - l1
    l2 = np.log(rho) / h
    np.testing.assert_allclose(lam[:, 0], [l1, l2, l3, l2], rtol=0, atol=1e-12)
    assert st[0] == O.OK


def _hh_ic(y, py, E):
    rad = 2 * E - py * py - y * y + 2 * y**3 / 3
    return np.array([[0.0], [y], [np.sqrt(rad)], [py]])


def test_dop853_eighth_order_under_step_halving():
    S = O.henon_heiles()
    x0 = _hh_ic(0.12, 0.05, 1 / 8)
    w = uniform_vectors(7, 1, 2, 4)
    out = {}
    for h in (0.8, 0.4, 0.05):
        prm = O.params(h, int(round(9.6 / h)), n_dev=2, renorm=False, sample_every=0,
                       integrator=O.DOP853)
        e = O.Ensemble(S, prm, x0, w_in=w)
        e.integrate(prm)
        out[h] = np.concatenate([e.x[:, 0], e.w[:, 0]])
    e1 = np.abs(out[0.8] - out[0.05]).max()
    e2 = np.abs(out[0.4] - out[0.05]).max()
    assert 1e-12 < e2 < e1 < 1e-4
    assert 7.0 < np.log2(e1 / e2) < 9.0


# --------------------------------------------------------------------------
# SciPy's DOP853 as an independent implementation
# --------------------------------------------------------------------------

def _hh_joint_rhs(k, ld_p):
    """Henon-Heiles (x, y, px, py) with k tangent vectors and the LD integrand,
    written out here from the Hamiltonian H = (px^2 + py^2 + x^2 + y^2)/2 + x^2 y - y^3/3."""

    def f(t, z):
        x, y, px, py = z[:4]
        fx = np.array([px, py, -x - 2 * x * y, -y - x * x + y * y])
        out = [fx]
        for j in range(k):
            dx, dy, dpx, dpy = z[4 + 4 * j: 8 + 4 * j]
            out.append(np.array([dpx, dpy, -(1 + 2 * y) * dx - 2 * x * dy,
                                 -2 * x * dx - (1 - 2 * y) * dy]))
        if ld_p:
            out.append(np.array([np.sum(np.abs(fx) ** ld_p)]))
        return np.concatenate(out)

    return f


def test_dop853_fixed_step_matches_scipy():
    si = pytest.importorskip("scipy.integrate")
    S = O.henon_heiles()
    k, h, n = 2, 1 / 16, 160
    x0 = _hh_ic(0.25, -0.1, 1 / 8)
    w = uniform_vectors(3, 1, k, 4)
    prm = O.params(h, n, n_dev=k, renorm=False, sample_every=0, ld_p=0.5, integrator=O.DOP853)
    e = O.Ensemble(S, prm, x0, w_in=w)
    e.integrate(prm)
    z0 = np.concatenate([x0[:, 0], w[:, 0], [0.0]])
    # huge atol: every error estimate is tiny, so SciPy takes exactly max_step each time
    sol = si.solve_ivp(_hh_joint_rhs(k, 0.5), (0.0, n * h), z0, method="DOP853",
                       first_step=h, max_step=h, rtol=1e-3, atol=1e10)
    assert sol.success and len(sol.t) == n + 1
    np.testing.assert_allclose(np.diff(sol.t), h, rtol=0, atol=1e-15)
    zo = np.concatenate([e.x[:, 0], e.w[:, 0], e.ld])
    assert np.abs(zo - sol.y[:, -1]).max() < 1e-13


@pytest.mark.parametrize("ic,first", [((0.25, -0.1), 0.01), ((0.29094, -0.28125), 1.5)])
def test_dop853_adaptive_matches_scipy_step_by_step(ic, first):
    """The oracle's adaptive DOP 8(5) follows SciPy's DOP853 step for step (the
    same error norm and controller), including rejected first attempts."""
    si = pytest.importorskip("scipy.integrate")
    S = O.henon_heiles()
    x0 = _hh_ic(ic[0], ic[1], 1 / 8)
    rtol, atol, T = 1e-9, 1e-12, 30.0
    prm = O.params(first, 1, n_dev=0, renorm=False, sample_every=0, integrator=O.DOP853)
    e = O.Ensemble(S, prm, x0)
    ts = []
    while e.t[0] < T if hasattr(e, "t") else True:
        e.integrate_adaptive(prm, T, rtol, atol)
        ts.append(e.t[0])
        assert e.err_last[0] < 1.0
        assert len(ts) < 100000
    sv = si.DOP853(_hh_joint_rhs(0, 0), 0.0, x0[:, 0], T, rtol=rtol, atol=atol, first_step=first)
    st = []
    while sv.status == "running":
        sv.step()
        st.append(sv.t)
    assert sv.status == "finished"
    assert len(ts) == len(st)
    # the error estimates are differences of nearly equal stage sums, so their
    # summation order (SciPy: BLAS dot products) moves them by ~1e-8 relative,
    # and the step sizes with them
    np.testing.assert_allclose(ts, st, rtol=1e-6, atol=0)
    assert np.abs(e.x[:, 0] - sv.y).max() < 1e-11
    assert e.n_exec[0] == len(ts)
    assert e.err_max[0] >= e.err_last[0]
    if first > 1.0:
        assert e.n_rej[0] >= 1
    # one call with a large step budget takes the same steps
    e2 = O.Ensemble(S, O.params(first, 10**6, n_dev=0, renorm=False, sample_every=0,
                                integrator=O.DOP853), x0)
    e2.integrate_adaptive(O.params(first, 10**6, n_dev=0, renorm=False, sample_every=0,
                                   integrator=O.DOP853), T, rtol, atol)
    assert e2.n_exec[0] == len(ts) and e2.t[0] == T
    np.testing.assert_array_equal(e2.x, e.x)


def test_dop853_adaptive_tolerance_proportionality():
    """Global error at t = 20 falls roughly in proportion to the tolerance, and
    the step count grows like tol^(-1/8)."""
    S = O.henon_heiles()
    x0 = _hh_ic(0.12, 0.05, 1 / 8)
    ref = O.Ensemble(S, O.params(0.01, 2000, n_dev=0, renorm=False, sample_every=0,
                                 integrator=O.DOP853), x0)
    ref.integrate(O.params(0.01, 2000, n_dev=0, renorm=False, sample_every=0, integrator=O.DOP853))
    errs, steps = [], []
    for tol in (1e-6, 1e-9):
        prm = O.params(0.01, 10**6, n_dev=0, renorm=False, sample_every=0, integrator=O.DOP853)
        e = O.Ensemble(S, prm, x0)
        e.integrate_adaptive(prm, 20.0, tol, tol)
        assert e.status[0] == O.OK and e.t[0] == 20.0
        errs.append(np.abs(e.x[:, 0] - ref.x[:, 0]).max())
        steps.append(e.n_exec[0])
    assert errs[1] < errs[0] / 30
    assert 1.5 < steps[1] / steps[0] < 4.0


def test_dop853_adaptive_step_fail():
    """At t = 1e20 the smallest allowed step (10 ulp(t) = 163840) is far too long:
    the attempt is rejected (its error is not even finite), the shrunk step falls
    below the limit and the orbit freezes as STEP_FAIL with its state untouched.
    With rtol = atol = 0 no error norm is below 1: the step shrinks until it
    fails the same way."""
    S = O.henon_heiles()
    x0 = _hh_ic(0.12, 0.05, 1 / 8)
    prm = O.params(0.1, 100, n_dev=0, renorm=False, sample_every=0, integrator=O.DOP853)
    e = O.Ensemble(S, prm, x0)
    e.integrate_adaptive(prm, 0.0, 1e-9, 1e-9)        # allocates t, h; nothing to do
    e.t[0] = 1e20
    e.integrate_adaptive(prm, 2e20, 1e-9, 1e-9)
    assert e.status[0] == O.STEP_FAIL
    assert e.n_exec[0] == 0 and e.t[0] == 1e20 and e.n_rej[0] == 1
    np.testing.assert_array_equal(e.x, x0)
    e = O.Ensemble(S, prm, x0)
    e.integrate_adaptive(prm, 10.0, 0.0, 0.0)
    assert e.status[0] == O.STEP_FAIL
    assert e.n_exec[0] == 0 and e.t[0] == 0.0 and e.n_rej[0] > 400
    np.testing.assert_array_equal(e.x, x0)


def test_dop853_lyapunov_sum_vanishes_to_eighth_order():
    """For a Hamiltonian flow the exponents sum to 0 (Liouville).  A one-step map
    with stability function R has determinant prod R(h mu) R(-h mu) over the
    eigenvalue pairs, 1 + O(h^9) for DOP853 (R(z) = e^z + O(z^9)) against
    1 + O(h^5) for RK4: on FPUT chains at h = 0.05 the DOP853 sum is at the
    rounding level while RK4's is ~1e-6."""
    from paper_2507_00622_gb300.inputs import normal_mode_draws
    N, n = 8, 3
    Q, P = normal_mode_draws(3, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    sums = {}
    for integ in (O.RK4, O.DOP853):
        lam, st = O.lyapunov(O.fput(N), O.params(0.05, 400, integrator=integ, qr_every=10), ics)
        assert np.all(st == O.OK)
        sums[integ] = np.abs(lam.sum(axis=0)).max()
    assert sums[O.DOP853] < 1e-11
    assert sums[O.RK4] > 1e-7


# --------------------------------------------------------------------------
# Lyapunov spectrum with adaptive DOP 8(5)
# --------------------------------------------------------------------------

def test_adaptive_lyapunov_inverted_oscillator_flow_spectrum():
    """With a tight tolerance the spectrum is that of the exact flow: for
    H = (p1^2 - q1^2)/2 + (p2^2 + q2^2)/2 and W(T) = exp(A T), the QR of W gives
    R_11 = sqrt(cosh 2T) = 1 / R_33 and R_22 = R_44 = 1, so
    lambda = (ln cosh 2T / 2T, 0, -ln cosh 2T / 2T, 0) in column order."""
    S = O.system(O.INVERTED, 2)
    T = 20.0
    lam, st, acc, rej = O.lyapunov_adaptive(S, O.params(0.01, 10**6, qr_every=10),
                                            np.array([[0.1], [0.2], [0.3], [-0.1]]), T, 1e-12, 1e-12)
    l1 = (2 * T + np.log1p(np.exp(-4 * T)) - np.log(2.0)) / (2 * T)
    np.testing.assert_allclose(lam[:, 0], [l1, 0.0, -l1, 0.0], rtol=0, atol=1e-9)
    assert st[0] == O.OK and acc[0] > 10


def test_adaptive_lyapunov_fput_liouville_and_fixed_step_agreement():
    from paper_2507_00622_gb300.inputs import normal_mode_draws
    N, n = 8, 3
    Q, P = normal_mode_draws(3, N, n)
    ics = O.fput_mode_ics(O.fput(N), Q, P, np.full(n, 0.1 * N))
    lam, st, acc, rej = O.lyapunov_adaptive(O.fput(N), O.params(0.05, 10**6, qr_every=10), ics,
                                            20.0, 1e-10, 1e-10)
    assert np.all(st == O.OK)
    assert np.abs(lam.sum(axis=0)).max() < 1e-8
    lf, _ = O.lyapunov(O.fput(N), O.params(0.02, 1000, qr_every=10, integrator=O.DOP853), ics)
    assert np.abs(lam - lf).max() < 1e-8
    # a step budget shorter than the run freezes the orbit
    lam, st, acc, rej = O.lyapunov_adaptive(O.fput(N), O.params(0.05, 5, qr_every=10), ics,
                                            20.0, 1e-10, 1e-10)
    assert np.all(st == O.STEP_FAIL) and np.all(np.isnan(lam)) and np.all(acc == 5)
