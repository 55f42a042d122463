"""Pins of the CPU oracle to facts fixed outside the oracle itself.

Each test checks the oracle against a closed form, an invariant, a published
test vector, a library routine on a special case, or an independent
derivation (sympy differentiation of the Hamiltonians the paper prints),
chosen so that a dropped term, a wrong sign or index, or a transposed operand
anywhere in the oracle fails at least one of them.
"""
import numpy as np
import pytest

import oracle as O
from paper_2507_00622_gb300.inputs import hh_section_box, normal_mode_draws, uniform_vectors

sympy = pytest.importorskip("sympy")


def _R(z):
    """Stability polynomial of classic RK4."""
    return 1 + z + z**2 / 2 + z**3 / 6 + z**4 / 24


def _hh_ic(y, py, E):
    rad = 2 * E - py * py - y * y + 2 * y**3 / 3
    return np.array([[0.0], [y], [np.sqrt(rad)], [py]])


# --------------------------------------------------------------------------
# RK4 core
# --------------------------------------------------------------------------

def test_rk4_harmonic_equals_stability_polynomial_power():
    """For H = (p^2 + q^2)/2, zeta = q + i p obeys zeta' = -i zeta, and one RK4
    step multiplies zeta by R(-ih) exactly."""
    S = O.system(O.HARMONIC, 1)
    h, n = 0.1, 500
    prm = O.params(h, n, n_dev=0, renorm=False, sample_every=0)
    ens = O.Ensemble(S, prm, np.array([[0.3], [-0.7]]))
    ens.integrate(prm)
    zn = _R(-1j * h) ** n * (0.3 - 0.7j)
    assert abs(ens.x[0, 0] - zn.real) < 1e-13
    assert abs(ens.x[1, 0] - zn.imag) < 1e-13
    # and it stays within O(t h^4) of the exact rotation
    ex = (0.3 - 0.7j) * np.exp(-1j * h * n)
    assert abs(complex(ens.x[0, 0], ens.x[1, 0]) - ex) < 50 * h**4


def test_rk4_fourth_order_under_step_halving():
    S = O.henon_heiles()
    x0 = _hh_ic(0.12, 0.05, 1 / 8)
    w = uniform_vectors(7, 1, 2, 4)
    out = []
    for h in (0.1, 0.05, 0.025):
        prm = O.params(h, int(round(10 / h)), n_dev=2, renorm=False, sample_every=0)
        e = O.Ensemble(S, prm, x0, w_in=w)
        e.integrate(prm)
        out.append(np.concatenate([e.x[:, 0], e.w[:, 0]]))
    r = np.abs(out[0] - out[1]).max() / np.abs(out[1] - out[2]).max()
    assert 16 * 0.9 < r < 16 * 1.1


def test_yoshida_and_rk4_agree_to_fourth_order():
    """Two independent 4th-order integrators (RK4 on the joint system; Yoshida
    composition with its tangent map) converge to the same flow."""
    S = O.henon_heiles()
    x0 = _hh_ic(0.1, 0.1, 1 / 8)
    w = uniform_vectors(0, 1, 2, 4)
    diffs = []
    for h in (0.01, 0.005):
        n = int(round(10 / h))
        a = O.Ensemble(S, O.params(h, n, n_dev=2, renorm=False, sample_every=0), x0, w_in=w)
        a.integrate(O.params(h, n, n_dev=2, renorm=False, sample_every=0))
        pb = O.params(h, n, n_dev=2, renorm=False, sample_every=0, integrator=O.YOSHIDA4)
        b = O.Ensemble(S, pb, x0, w_in=w)
        b.integrate(pb)
        diffs.append(max(np.abs(a.x - b.x).max(), np.abs(a.w - b.w).max()))
    assert diffs[0] < 1e-7
    assert 12 < diffs[0] / diffs[1] < 20


# --------------------------------------------------------------------------
# Hamiltonians, equations of motion, Hessians (independent sympy derivation)
# --------------------------------------------------------------------------

def _sym_check(sysd, Hexpr, qs, ps, rng, npts=5, scale=0.4):
    N = len(qs)
    grad = [sympy.diff(Hexpr, v) for v in qs + ps]
    hess = [[sympy.diff(Hexpr, a, b) for b in qs] for a in qs]
    fH = sympy.lambdify(qs + ps, Hexpr, "numpy")
    fg = sympy.lambdify(qs + ps, grad, "numpy")
    fh = sympy.lambdify(qs + ps, hess, "numpy")
    for _ in range(npts):
        x = rng.uniform(-scale, scale, 2 * N)
        f = O.rhs(sysd, x)
        g = np.array(fg(*x), dtype=float)
        # Hamilton's equations: q' = dH/dp, p' = -dH/dq
        np.testing.assert_allclose(f[:N], g[N:], rtol=0, atol=1e-14)
        np.testing.assert_allclose(f[N:], -g[:N], rtol=0, atol=1e-13)
        np.testing.assert_allclose(O.hessian(sysd, x[:N]), np.array(fh(*x), dtype=float),
                                   rtol=0, atol=1e-13)
        assert abs(O.energy(sysd, x) - float(fH(*x))) < 1e-14


def test_henon_heiles_equations_from_hamiltonian():
    x, y, px, py = sympy.symbols("x y p_x p_y")
    H = px**2 / 2 + py**2 / 2 + (x**2 + y**2) / 2 + x**2 * y - y**3 / 3  # Eq. Ham_HH
    # the printed equations of motion (Eq. ham_eqs_HH) follow from it
    assert sympy.simplify(-sympy.diff(H, x) - (-x - 2 * x * y)) == 0
    assert sympy.simplify(-sympy.diff(H, y) - (-y - x**2 + y**2)) == 0
    _sym_check(O.henon_heiles(), H, [x, y], [px, py], np.random.default_rng(1))


@pytest.mark.parametrize("N", [1, 2, 5])
def test_fput_equations_from_hamiltonian(N):
    """FPUT chain with fixed ends q_0 = q_{N+1} = 0.  The Hamiltonian summed
    over the N+1 bonds D_i = q_i - q_{i-1}, i = 1..N+1, reproduces the
    printed equations of motion (Eq. ham_eqs_FPU) for every i, including the
    bond to the wall at i = 1."""
    k, a, b = 0.8, 0.3, 1.2
    qs = list(sympy.symbols(f"q1:{N + 1}"))
    ps = list(sympy.symbols(f"p1:{N + 1}"))
    qq = [0] + qs + [0]
    D = [qq[i] - qq[i - 1] for i in range(1, N + 2)]  # D[0] = D_1 ... D[N] = D_{N+1}
    H = sum(p**2 / 2 for p in ps) + sum(k / 2 * r**2 + a / 3 * r**3 + b / 4 * r**4 for r in D)
    for i in range(1, N + 1):
        Di, Dn = D[i - 1], D[i]
        printed = -k * (Di - Dn) - a * (Di**2 - Dn**2) - b * (Di**3 - Dn**3)
        assert sympy.expand(-sympy.diff(H, qs[i - 1]) - printed) == 0
    _sym_check(O.fput(N, beta=b, alpha=a, kk=k), H, qs, ps, np.random.default_rng(N))


def test_quartic_and_test_oscillators_from_hamiltonian():
    q = list(sympy.symbols("q1:4"))
    p = list(sympy.symbols("p1:4"))
    eps = 0.1
    H = sum(v**2 for v in p) / 2 + sum(v**2 for v in q) / 2 + eps * (
        q[0]**2 * q[1]**2 + q[1]**2 * q[2]**2 + q[0]**2 * q[2]**2)
    _sym_check(O.system(O.QUARTIC3, 3, eps=eps), H, q, p, np.random.default_rng(3), scale=1.5)
    q2, p2 = list(sympy.symbols("a1:3")), list(sympy.symbols("b1:3"))
    Hi = (p2[0]**2 - q2[0]**2) / 2 + (p2[1]**2 + q2[1]**2) / 2
    _sym_check(O.system(O.INVERTED, 2), Hi, q2, p2, np.random.default_rng(4))
    Hh = sum(v**2 for v in p2) / 2 + sum(v**2 for v in q2) / 2
    _sym_check(O.system(O.HARMONIC, 2), Hh, q2, p2, np.random.default_rng(5))


# --------------------------------------------------------------------------
# Variational equations
# --------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["hh", "fput", "quartic", "inverted", "harmonic"])
def test_deviation_vectors_equal_derivative_of_numerical_flow(case):
    """RK4 applied to the joint system (x, w) yields exactly the tangent map
    of the RK4 step, so w(T) equals the central difference of the numerical
    flow along w(0) up to O(eps^2)."""
    rng = np.random.default_rng(11)
    if case == "hh":
        S, x0 = O.henon_heiles(), _hh_ic(0.2, -0.1, 1 / 8)[:, 0]
    elif case == "fput":
        S, x0 = O.fput(5, beta=1.2, alpha=0.3, kk=0.8), rng.uniform(-0.4, 0.4, 10)
    elif case == "quartic":
        S, x0 = O.system(O.QUARTIC3, 3, eps=0.1), rng.uniform(-1.2, 1.2, 6)
    elif case == "inverted":
        S, x0 = O.system(O.INVERTED, 2), rng.uniform(-0.5, 0.5, 4)
    else:
        S, x0 = O.system(O.HARMONIC, 3), rng.uniform(-0.5, 0.5, 6)
    d = 2 * S.n_dof
    w0 = rng.uniform(-1, 1, d)
    h, n, eps = 0.01, 500, 1e-6
    prm = O.params(h, n, n_dev=1, renorm=False, sample_every=0)
    e = O.Ensemble(S, prm, x0[:, None], w_in=w0[:, None])
    e.integrate(prm)
    p0 = O.params(h, n, n_dev=0, sample_every=0)
    plus = O.Ensemble(S, p0, (x0 + eps * w0)[:, None]).integrate(p0).x[:, 0]
    minus = O.Ensemble(S, p0, (x0 - eps * w0)[:, None]).integrate(p0).x[:, 0]
    fd = (plus - minus) / (2 * eps)
    assert np.abs(e.w[:, 0] - fd).max() < 1e-7 * max(1.0, np.abs(fd).max())


# --------------------------------------------------------------------------
# Energy and health
# --------------------------------------------------------------------------

def test_energy_drift_bounds_and_order():
    S = O.henon_heiles()
    y0, y1, p0, p1 = hh_section_box(1 / 8)
    ics, st = O.grid_ics(1 / 8, y0, y1, 8, p0, p1, 8)
    prm = O.params(0.01, 20000, n_dev=0, sample_every=10)
    e = O.Ensemble(S, prm, ics, st)
    e.integrate(prm)
    assert np.nanmax(e.dh_max[st == 0]) < 1e-9
    # FPUT: RK4 drift shrinks at least ~h^4 under step halving
    F = O.fput(8)
    Q, P = normal_mode_draws(3, 8, 4)
    ics = O.fput_mode_ics(F, Q, P, np.full(4, 0.8))
    drift = []
    for h in (0.05, 0.025):
        p = O.params(h, int(round(100 / h)), n_dev=0, sample_every=int(round(1 / h)))
        drift.append(O.Ensemble(F, p, ics).integrate(p).dh_max.max())
    assert drift[0] < 1e-4 and drift[0] / drift[1] > 14


def test_escape_freezes_orbit_and_labels_it():
    S = O.henon_heiles()
    ic = np.array([[0.0], [0.3], [0.2], [0.55]])
    prm = O.params(0.01, 20000, n_dev=2, ld_p=0.5, escape_r2=4.0)
    e = O.Ensemble(S, prm, ic)
    assert O.energy(S, ic[:, 0]) > 1 / 6
    e.integrate(prm)
    assert e.status[0] == O.ESCAPED
    assert e.x[0, 0] ** 2 + e.x[1, 0] ** 2 > 4.0
    assert 0 < e.n_exec[0] < 20000
    _, _, lab = e.indicators()
    assert lab[0] == 2


def test_nonfinite_and_forbidden_status():
    S = O.henon_heiles()
    ics = np.array([[0.0, np.nan, 0.0], [0.1, 0.0, 0.1], [0.3, 0.0, 0.3], [0.1, 0.0, 0.1]])
    ic_st = np.array([0, 0, O.FORBIDDEN], dtype=np.int32)
    prm = O.params(0.01, 200, n_dev=2, ld_p=0.5, dh_limit=1e-30, sample_every=100)
    e = O.Ensemble(S, prm, ics, ic_st)
    assert list(e.status) == [O.OK, O.NONFINITE, O.FORBIDDEN]
    e.integrate(prm)
    # a drift limit of 1e-30 trips at the first health check (step 100)
    assert e.status[0] == O.ENERGY_DRIFT and e.n_exec[0] == 100
    sali, gali, lab = e.indicators()
    assert list(lab) == [-1, -1, -1]
    assert np.isnan(sali[2]) and np.isnan(gali[:, 2]).all()


def test_chunked_integration_is_bit_identical():
    S = O.henon_heiles()
    y0, y1, p0, p1 = hh_section_box(1 / 6)
    ics, st = O.grid_ics(1 / 6, y0, y1, 6, p0, p1, 6)
    full = O.params(0.01, 3000, n_dev=3, ld_p=0.5, escape_r2=4.0)
    a = O.Ensemble(S, full, ics, st, seed=5)
    a.integrate(full)
    b = O.Ensemble(S, full, ics, st, seed=5)
    for s0 in (0, 1000, 2000):
        b.integrate(O.params(0.01, 1000, step0=s0, n_dev=3, ld_p=0.5, escape_r2=4.0))
    for name in ("x", "w", "ld", "dh_max", "n_exec", "status"):
        np.testing.assert_array_equal(getattr(a, name), getattr(b, name))


# --------------------------------------------------------------------------
# Initial conditions and seeding
# --------------------------------------------------------------------------

def test_grid_ics_lie_on_energy_shell():
    for E in (1 / 8, 1 / 6):
        y0, y1, p0, p1 = hh_section_box(E)
        ics, st = O.grid_ics(E, y0, y1, 32, p0, p1, 32)
        S = O.henon_heiles()
        assert (st == 0).sum() > 600
        for o in range(ics.shape[1]):
            y = y0 + (o // 32 + 0.5) * (y1 - y0) / 32
            py = p0 + (o % 32 + 0.5) * (p1 - p0) / 32
            if st[o] == 0:
                assert ics[0, o] == 0.0 and ics[2, o] >= 0.0
                assert abs(ics[1, o] - y) < 1e-15 and abs(ics[3, o] - py) < 1e-15
                assert abs(O.energy(S, ics[:, o]) - E) < 1e-15
            else:
                # no real p_x: the point with p_x = 0 already lies above the shell
                assert O.energy(S, np.array([0.0, y, 0.0, py])) > E
                assert np.isnan(ics[:, o]).all()


def test_splitmix64_published_test_vector():
    """First outputs of SplitMix64 seeded with 1234567, as published with the
    reference implementation of the generator (Vigna, splitmix64.c)."""
    ref = [6457827717110365317, 3203168211198807973, 9817491932198370423,
           4593380528125082431, 16408922859458223821]
    assert O.splitmix64_stream(1234567, 5) == ref
    # seeded vectors: orbit 0, vector 0, components 0..3 use outputs 1..4
    w = O.seed_vectors(1234567, 1, 1, 4)[:, 0]
    u = np.array([2.0 * ((z >> 11) * 2.0**-53) - 1.0 for z in ref[:4]])
    np.testing.assert_allclose(w, u / np.linalg.norm(u), rtol=0, atol=1e-16)


def test_fput_mode_ics_energy_and_sine_transform():
    from scipy.fft import dst
    N, n = 8, 6
    F = O.fput(N)
    Q, P = normal_mode_draws(9, N, n)
    E = np.full(n, 0.1 * N)
    ics = O.fput_mode_ics(F, Q, P, E)
    for o in range(n):
        assert abs(O.energy(F, ics[:, o]) - E[o]) < 1e-13
        # unscaled q = sqrt(2/(N+1)) * DST-I(Q); scipy's DST-I carries a factor 2
        q = np.sqrt(2.0 / (N + 1)) * dst(Q[:, o], type=1) / 2
        p = np.sqrt(2.0 / (N + 1)) * dst(P[:, o], type=1) / 2
        s = ics[0, o] / q[0]
        np.testing.assert_allclose(ics[:N, o], s * q, rtol=1e-12)
        np.testing.assert_allclose(ics[N:, o], s * p, rtol=1e-12)
        # the transform is orthogonal: sum q^2 = s^2 sum Q^2
        assert abs((ics[:N, o] ** 2).sum() - s * s * (Q[:, o] ** 2).sum()) < 1e-12


# --------------------------------------------------------------------------
# SALI and GALI
# --------------------------------------------------------------------------

def _sali(a, b):
    a, b = a / np.linalg.norm(a), b / np.linalg.norm(b)
    return min(np.linalg.norm(a + b), np.linalg.norm(a - b))


def test_jacobi_singular_values_match_lapack():
    rng = np.random.default_rng(2)
    for d, k in ((4, 2), (4, 4), (6, 6), (8, 3), (16, 5)):
        A = rng.standard_normal((d, k))
        sv = np.sort(O.jacobi_sv(A))[::-1]
        np.testing.assert_allclose(sv, np.linalg.svd(A, compute_uv=False), rtol=1e-13)


def test_gali_closed_forms():
    S = O.system(O.HARMONIC, 2)
    th = np.array([1.0, 1e-3, 1e-7, 1e-10])
    # w1 = e1, w2 = cos(th) e1 + sin(th) e2: GALI_2 = sin(th); SALI = |w1 - w2| = 2 sin(th/2)
    w = np.zeros((8, th.size))
    w[0] = 1.0
    w[4] = np.cos(th)
    w[5] = np.sin(th)
    st = np.zeros(th.size, dtype=np.int32)
    sali, gali = np.empty(th.size), np.empty((1, th.size))
    lab = np.empty(th.size, dtype=np.int8)
    import ctypes as C
    O.lib().o_indicators(C.byref(S), th.size, 2, O._p(w), O._p(st), 1e-8, O._p(sali),
                         O._p(gali), O._p(lab))
    np.testing.assert_allclose(gali[0], np.sin(th), rtol=1e-12)
    np.testing.assert_allclose(sali, 2 * np.sin(th / 2), rtol=1e-6)
    # GALI_2 = |w1 + w2| |w1 - w2| / 2 for unit vectors, on random pairs
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = rng.standard_normal(4), rng.standard_normal(4)
        a, b = a / np.linalg.norm(a), b / np.linalg.norm(b)
        g2 = np.prod(O.jacobi_sv(np.stack([a, b], 1)))
        assert abs(g2 - np.linalg.norm(a + b) * np.linalg.norm(a - b) / 2) < 1e-14


def test_sali_gali_constant_under_harmonic_flow():
    """The RK4 map of the harmonic oscillator is a uniform scaling times a
    rotation, so angles between deviation vectors (SALI, GALI_k) are exactly
    preserved."""
    S = O.system(O.HARMONIC, 2)
    rng = np.random.default_rng(8)
    ics = rng.uniform(-1, 1, (4, 5))
    prm = O.params(0.01, 5000, n_dev=4, ld_p=0.5)
    e = O.Ensemble(S, prm, ics, seed=3)
    w0 = e.w.copy()
    e.integrate(prm)
    sali, gali, _ = e.indicators()
    for o in range(5):
        W = w0[:, o].reshape(4, 4).T  # columns = vectors
        assert abs(sali[o] - _sali(W[:, 0], W[:, 1])) < 1e-11
        for m in range(2, 5):
            ref = np.prod(np.linalg.svd(W[:, :m], compute_uv=False))
            assert abs(gali[m - 2, o] - ref) < 1e-11 * max(ref, 1e-3)


@pytest.fixture(scope="module")
def hh_reference_orbits():
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hh_reference_orbits.json")
    with open(path) as f:
        return json.load(f)


def test_sali_regular_orbit_stays_and_gali_power_laws(hh_reference_orbits):
    """Regular orbit of a 2-DOF system: SALI fluctuates about a positive value,
    GALI_3 ~ t^-2 and GALI_4 ~ t^-4 (Skokos et al. 2008, GALI for N = 2)."""
    S = O.henon_heiles()
    r = hh_reference_orbits["regular"]
    ic = _hh_ic(r["y"], r["py"], r["E"])
    e = O.Ensemble(S, O.params(0.01, 1, n_dev=4), ic, seed=1)
    ts, g3, g4, sa = [], [], [], []
    step = 0
    for t_target in (250, 500, 1000, 2000):
        n = int(round(t_target / 0.01)) - step
        e.integrate(O.params(0.01, n, step0=step, n_dev=4))
        step += n
        sali, gali, _ = e.indicators()
        ts.append(t_target)
        sa.append(sali[0])
        g3.append(gali[1, 0])
        g4.append(gali[2, 0])
    assert min(sa) > 5e-4
    s3 = np.polyfit(np.log(ts), np.log(g3), 1)[0]
    s4 = np.polyfit(np.log(ts), np.log(g4), 1)[0]
    assert -2.6 < s3 < -1.4
    assert -4.8 < s4 < -3.2


def test_sali_decay_rate_matches_lyapunov_exponents(hh_reference_orbits):
    """Chaotic orbit: SALI ~ exp(-(lambda_1 - lambda_2) t) (Skokos 2001); for a
    2-DOF Hamiltonian lambda_2 = 0, and lambda_1 comes from the independent
    QR computation of the spectrum."""
    S = O.henon_heiles()
    c = hh_reference_orbits["chaotic"]
    ic = _hh_ic(c["y"], c["py"], c["E"])
    e = O.Ensemble(S, O.params(0.01, 1, n_dev=2), ic, seed=1)
    ts, ls = [], []
    step = 0
    for i in range(1, 41):
        n = 2500
        e.integrate(O.params(0.01, n, step0=step, n_dev=2))
        step += n
        sali, _, _ = e.indicators()
        if 1e-13 < sali[0] < 1e-3:
            ts.append(step * 0.01)
            ls.append(np.log(sali[0]))
    assert len(ts) >= 4
    slope = np.polyfit(ts, ls, 1)[0]
    lam, st = O.lyapunov(S, O.params(0.01, step, qr_every=10), ic)
    lam1 = lam[0, 0]
    assert lam1 > 0.01
    assert abs(-slope - lam1) < 0.35 * lam1
    # pairing and vanishing sum for the Hamiltonian spectrum
    srt = np.sort(lam[:, 0])[::-1]
    assert abs(srt.sum()) < 1e-6
    assert abs(srt[0] + srt[3]) < 0.05 * lam1 + 2.0 / (step * 0.01)


# --------------------------------------------------------------------------
# Lyapunov spectrum
# --------------------------------------------------------------------------

def test_lyapunov_inverted_oscillator_closed_form():
    """H = (p1^2 - q1^2)/2 + (p2^2 + q2^2)/2 is linear, so W evolves by
    M = R(hA) and the accumulated QR diagonal equals that of M^n.  In column
    order (q1, q2, p1, p2), with a = R(h), b = R(-h) and rho = |R(ih)|:
      lambda_1 = ln((a^2n + b^2n)/2) / (2T),  lambda_3 = n ln(ab)/T - lambda_1,
      lambda_2 = lambda_4 = ln(rho)/h."""
    S = O.system(O.INVERTED, 2)
    h, n = 0.01, 2000
    T = n * h
    lam, st = O.lyapunov(S, O.params(h, n, qr_every=10),
                         np.array([[0.1], [0.2], [0.3], [-0.1]]))
    a, b = _R(h), _R(-h)
    rho = abs(_R(1j * h))
    l1 = (2 * n * np.log(a) + np.log1p((b / a) ** (2 * n)) - np.log(2.0)) / (2 * T)
    l3 = n * np.log(a * b) / T - l1
    l2 = np.log(rho) / h
    np.testing.assert_allclose(lam[:, 0], [l1, l2, l3, l2], rtol=0, atol=1e-12)
    assert st[0] == O.OK


def test_lyapunov_harmonic_chain_limit():
    """beta -> 0: the FPUT chain is linear with purely rotating normal modes,
    so every exponent vanishes up to the RK4 damping ln|R(i w h)|/h and the
    O(1/T) transient."""
    N = 4
    F = O.fput(N, beta=0.0)
    Q, P = normal_mode_draws(1, N, 2)
    ics = O.fput_mode_ics(F, Q, P, np.full(2, 0.4))
    lam, st = O.lyapunov(F, O.params(0.05, 4000, qr_every=10), ics)
    assert np.abs(lam).max() < 0.05
    assert abs(lam[:, 0].sum()) < 1e-6


def test_fput_linear_chain_ensemble_follows_matrix_exponential():
    """alpha = beta = 0: the chain is linear, x' = A x with A = [[0, I], [-K, 0]]
    and K the fixed-end Laplacian (Eq. ham_eqs_FPU at k = 1), and the deviation
    vectors obey the same equation.  After time t the ensemble's state is
    expm(A t) x0 and each renormalised vector the unit vector along
    expm(A t) w0, up to RK4's O(h^4) error; GALI_2 and SALI follow from those
    unit vectors.  An independent check (scipy's expm) of the FPUT ensemble
    path: Hessian, stage loop, renormalisation and indicators together."""
    from scipy.linalg import expm
    N, k, n, h, steps = 6, 3, 5, 0.005, 2000
    F = O.fput(N, beta=0.0)
    K = 2.0 * np.eye(N) - np.eye(N, k=1) - np.eye(N, k=-1)
    A = np.block([[np.zeros((N, N)), np.eye(N)], [-K, np.zeros((N, N))]])
    Q, P = normal_mode_draws(17, N, n)
    ics = O.fput_mode_ics(F, Q, P, np.full(n, 0.3))
    e = O.Ensemble(F, O.params(h, 1, n_dev=k), ics, seed=21)
    w0 = e.w.copy()
    e.integrate(O.params(h, steps, n_dev=k))
    Phi = expm(A * h * steps)
    d = 2 * N
    np.testing.assert_allclose(e.x, Phi @ ics, atol=1e-9)
    U = np.empty((k, d, n))
    for j in range(k):
        v = Phi @ w0[j * d:(j + 1) * d]
        U[j] = v / np.linalg.norm(v, axis=0)
        np.testing.assert_allclose(e.w[j * d:(j + 1) * d], U[j], atol=1e-9)
    sali, gali, _ = e.indicators()
    for o in range(n):
        for m in range(2, k + 1):  # GALI_m from the first m unit vectors
            sv = np.linalg.svd(U[:m, :, o].T, compute_uv=False)
            np.testing.assert_allclose(gali[m - 2, o], np.prod(sv), rtol=1e-7)
        a, b = U[0, :, o], U[1, :, o]
        np.testing.assert_allclose(sali[o], min(np.linalg.norm(a + b), np.linalg.norm(a - b)),
                                   rtol=1e-7)


# --------------------------------------------------------------------------
# Lagrangian descriptors
# --------------------------------------------------------------------------

def test_ld_harmonic_closed_form_and_convergence():
    """q = A cos t, p = -A sin t: int_0^{2pi} (|q'|^1/2 + |p'|^1/2) dt
    = 8 sqrt(A) int_0^{pi/2} sin^{1/2}, and the integral equals
    sqrt(pi)/2 Gamma(3/4)/Gamma(5/4).  The integrand is only Holder-1/2 at its
    zeros, so RK4 converges like h^1.5 here."""
    from scipy.special import gamma
    I = np.sqrt(np.pi) / 2 * gamma(0.75) / gamma(1.25)
    A = 2.0
    exact = 8 * I * np.sqrt(A)
    S = O.system(O.HARMONIC, 1)
    errs = []
    for n in (4000, 16000):
        prm = O.params(2 * np.pi / n, n, n_dev=0, ld_p=0.5, sample_every=0)
        e = O.Ensemble(S, prm, np.array([[A], [0.0]]))
        e.integrate(prm)
        errs.append(abs(e.ld[0] - exact))
    assert errs[1] < 5e-6
    assert 6.0 < errs[0] / errs[1] < 10.0


def test_backward_ld_retraces_the_orbit():
    """A backward run (h < 0) integrates the same integrand over |t|: from
    q = A cos t at t = 0 back to t = -2 pi the LD is the same closed form, and
    running forward to T then backward to 0 returns to the initial state with
    twice the forward LD (the orbit retraces itself to O(T h^4); the two LD
    quadratures agree to the RK4 error of the non-smooth integrand)."""
    from scipy.special import gamma
    I = np.sqrt(np.pi) / 2 * gamma(0.75) / gamma(1.25)
    A = 2.0
    S = O.system(O.HARMONIC, 1)
    n = 16000
    prm = O.params(-2 * np.pi / n, n, n_dev=0, ld_p=0.5, sample_every=0)
    e = O.Ensemble(S, prm, np.array([[A], [0.0]]))
    e.integrate(prm)
    assert abs(e.ld[0] - 8 * I * np.sqrt(A)) < 5e-6
    H = O.henon_heiles()
    x0 = np.array([[0.0], [0.1], [np.sqrt(0.25 - 0.01 - 0.01 + 2 * 0.001 / 3)], [0.1]])
    f = O.Ensemble(H, O.params(0.01, 1, n_dev=1, ld_p=0.5), x0)
    f.integrate(O.params(0.01, 2000, n_dev=1, ld_p=0.5))
    ld_f = f.ld[0]
    f.integrate(O.params(-0.01, 2000, n_dev=1, ld_p=0.5))
    assert np.abs(f.x - x0).max() < 1e-9
    assert abs(f.ld[0] - 2 * ld_f) < 1e-6 * ld_f


def test_ld_indicators_on_synthetic_fields():
    ny, npy = 7, 9
    iy, ip = np.meshgrid(np.arange(ny), np.arange(npy), indexing="ij")
    st = np.zeros(ny * npy, dtype=np.int32)
    const = np.full(ny * npy, 3.0)
    dl, sl = O.ld_indicators(ny, npy, const, st)
    inner = ((iy > 0) & (iy < ny - 1) & (ip > 0) & (ip < npy - 1)).ravel()
    assert np.all(dl[inner] == 0) and np.all(sl[inner] == 0)
    assert np.isnan(dl[~inner]).all() and np.isnan(sl[~inner]).all()
    lin = (5.0 + 0.5 * iy + 0.25 * ip).ravel()
    dl, sl = O.ld_indicators(ny, npy, lin, st)
    np.testing.assert_allclose(sl[inner], 0.0, atol=1e-15)
    np.testing.assert_allclose(dl[inner], (2 * 0.5 + 2 * 0.25) / (4 * lin[inner]), rtol=1e-14)
    quad = (10.0 + iy**2 + 2.0 * ip**2).astype(float).ravel()
    dl, sl = O.ld_indicators(ny, npy, quad, st)
    # second differences 2 and 4: S_L = (2/LD + 4/LD)/2
    np.testing.assert_allclose(sl[inner], 3.0 / quad[inner], rtol=1e-13)
    np.testing.assert_allclose(
        dl[inner], (np.abs(4.0 * iy.ravel()[inner]) + np.abs(8.0 * ip.ravel()[inner]))
        / (4 * quad[inner]), rtol=1e-13)
    st2 = st.copy()
    st2[3 * npy + 4] = O.FORBIDDEN
    dl, sl = O.ld_indicators(ny, npy, quad, st2)
    for o in (3 * npy + 4, 2 * npy + 4, 4 * npy + 4, 3 * npy + 3, 3 * npy + 5):
        assert np.isnan(dl[o]) and np.isnan(sl[o])
    assert np.isfinite(dl[2 * npy + 2])


# --------------------------------------------------------------------------
# early exit, per-orbit end steps, quartic shell initial conditions
# --------------------------------------------------------------------------

def test_early_exit_stops_at_first_health_check_below_threshold(hh_reference_orbits):
    S = O.henon_heiles()
    c, r = hh_reference_orbits["chaotic"], hh_reference_orbits["regular"]
    ics = np.concatenate([_hh_ic(c["y"], c["py"], c["E"]), _hh_ic(r["y"], r["py"], r["E"])], axis=1)
    kw = dict(n_dev=2, sample_every=100, sali_threshold=1e-8)
    e = O.Ensemble(S, O.params(0.01, 1, **kw), ics, seed=4)
    e.integrate(O.params(0.01, 100000, early_exit=True, **kw))
    assert list(e.status) == [O.EARLY_CHAOTIC, O.OK]
    m = int(e.n_exec[0])
    assert m % 100 == 0 and 0 < m < 100000 and e.n_exec[1] == 100000
    sali, _, lab = e.indicators(1e-8)
    assert sali[0] < 1e-8 and list(lab) == [1, 0]
    # the same orbit without early exit is above the threshold one check earlier
    f = O.Ensemble(S, O.params(0.01, 1, **kw), ics[:, :1], seed=4)
    f.integrate(O.params(0.01, m - 100, **kw))
    assert f.indicators(1e-8)[0][0] >= 1e-8
    f.integrate(O.params(0.01, 100, step0=m - 100, **kw))
    np.testing.assert_array_equal(f.x[:, 0], e.x[:, 0])


def test_per_orbit_end_steps():
    S = O.henon_heiles()
    y0, y1, p0, p1 = hh_section_box(1 / 8)
    ics, st = O.grid_ics(1 / 8, y0, y1, 3, p0, p1, 3)
    t_end = np.array([0, 150, 300, 450, 600, 750, 900, 1050, 1200], dtype=np.int64)
    kw = dict(n_dev=2, ld_p=0.5)
    e = O.Ensemble(S, O.params(0.01, 1, **kw), ics, st, seed=2)
    for s0 in (0, 500):
        e.integrate(O.params(0.01, 500, step0=s0, **kw), t_end=t_end)
    ok = st == 0
    np.testing.assert_array_equal(e.n_exec[ok], np.minimum(t_end, 1000)[ok])
    for o in np.where(ok)[0]:
        f = O.Ensemble(S, O.params(0.01, 1, **kw), ics[:, o:o + 1], seed=2,
                       w_in=O.seed_vectors(2, ics.shape[1], 2, 4)[:, o:o + 1])
        f.integrate(O.params(0.01, int(min(t_end[o], 1000)), **kw))
        np.testing.assert_array_equal(f.x[:, 0], e.x[:, o])


def test_quartic_shell_ics():
    S = O.system(O.QUARTIC3, 3, eps=0.1)
    rng = np.random.default_rng(12)
    dirs = rng.standard_normal((6, 50))
    E = rng.uniform(1.0, 10.0, 50)
    ics = O.shell_ics(S, dirs, E)
    for o in range(50):
        assert abs(O.energy(S, ics[:, o]) - E[o]) < 1e-12 * E[o]
        u = dirs[:, o] / np.linalg.norm(dirs[:, o])
        np.testing.assert_allclose(ics[:, o] / np.linalg.norm(ics[:, o]), u, atol=1e-14)
