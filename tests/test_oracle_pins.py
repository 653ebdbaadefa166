"""Pins of the FP64 oracle to facts other than itself (no GPU).

Each test cites what fixes the expected value: a hand-computed example, a
closed form, a numerical quadrature, a finite-difference derivative of an
independent expression, an invariance of the exact sum, or convergence to the
direct sum.  Mutation tests at the end plant plausible mistakes in (copies of)
the oracle's steps and check that a pin catches each one.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate, special

import workloads as W
from oracle import direct, greens, params, se

GOLD = os.path.join(os.path.dirname(__file__), "golden")
KNAMES = ["stokeslet", "stresslet", "rotlet"]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


# ---------------------------------------------------------------- direct sum (O1)

def test_two_point_golden():
    """Hand-computed two-point sums (Section 2, eqs. def_stokeslet/def_stresslet/def_rotlet)."""
    g = json.load(open(os.path.join(GOLD, "two_point.json")))
    x, f, q = np.array(g["x"]), np.array(g["f"]), np.array(g["q"])
    for k, name in enumerate(KNAMES):
        want = np.array([[float(Fraction(v)) for v in row] for row in g["u"][name]])
        got = direct.direct(k, x, f, q if k == 1 else None)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-15)


def _num_grad(fun, x, h=1e-3):
    """4th-order central difference gradient of a scalar function of a 3-vector."""
    g = np.zeros(3)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        g[a] = (-fun(x + 2 * e) + 8 * fun(x + e) - 8 * fun(x - e) + fun(x - 2 * e)) / (12 * h)
    return g


def _num_hess(fun, x, h=1e-3):
    return np.array([_num_grad(lambda y, a=a: _num_grad(fun, y, h)[a], x, h) for a in range(3)])


def _num_third(fun, x, h=2e-3):
    return np.array([_num_hess(lambda y, a=a: _num_grad(fun, y, h)[a], x, h) for a in range(3)])


R_TEST = np.array([0.3, -0.5, 0.7])


def _operator_form(phi, r, kernel):
    """Apply the operator of eqs. stokeslet_op / stresslet_op to the radial
    function phi (by finite differences), or -eps_jlm d_m of phi for the rotlet."""
    d3 = _num_third(phi, r)  # d3[a][b][c] = d_a d_b d_c phi
    lap_grad = np.array([d3[m, 0, 0] + d3[m, 1, 1] + d3[m, 2, 2] for m in range(3)])
    hess = _num_hess(phi, r)
    G = np.zeros((3, 3, 3))
    I = np.eye(3)
    if kernel == 0:
        lap = np.trace(hess)
        G[:, :, 0] = I * lap - hess
    elif kernel == 1:
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    G[j, l, m] = (I[j, l] * lap_grad[m] + I[l, m] * lap_grad[j] +
                                  I[m, j] * lap_grad[l]) - 2 * d3[j, l, m]
    else:
        grad = _num_grad(phi, r)
        for j in range(3):
            for l in range(3):
                for m in range(3):
                    e = se._eps(j, l, m)
                    G[j, l, 0] += -e * grad[m]
    return G


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_kernels_match_operator_forms(kernel):
    """S = (delta lap - dd) r, T = [(delta d + ..) lap - 2 ddd] r (eqs. stokeslet_op,
    stresslet_op) and Omega = -eps d(1/r) (definition; the paper's rotlet_op has 2x)."""
    if kernel == 2:
        phi = lambda y: 1.0 / np.linalg.norm(y)  # noqa: E731
    else:
        phi = lambda y: np.linalg.norm(y)  # noqa: E731
    want = _operator_form(phi, R_TEST, kernel)
    got = direct.kernel_full(kernel, R_TEST)[0]
    if kernel != 1:
        got = got.copy()
        got[:, :, 1:] = 0
    np.testing.assert_allclose(got, want, atol=2e-6 * np.abs(want).max())


def test_direct_invariances():
    """Exact-sum invariances: translation, rotation covariance, homogeneity of
    degree -1 (S) and -2 (T, Omega) (Section 2 definitions)."""
    x, f = W.stokeslet_uniform(60, 11)
    q = W.unit_vectors(60, 11)
    th = 0.7
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    Rm = Rz @ Rx
    for k in range(3):
        qq = q if k == 1 else None
        u = direct.direct(k, x, f, qq)
        np.testing.assert_allclose(direct.direct(k, x + np.array([3.0, -1.0, 0.5]), f, qq), u,
                                   rtol=1e-12, atol=1e-12 * np.abs(u).max())
        ur = direct.direct(k, x @ Rm.T, f @ Rm.T, None if qq is None else qq @ Rm.T)
        np.testing.assert_allclose(ur, u @ Rm.T, atol=1e-11 * np.abs(u).max())
        s = 2.5
        deg = 1 if k == 0 else 2
        np.testing.assert_allclose(direct.direct(k, s * x, f, qq), u / s**deg, rtol=1e-12,
                                   atol=1e-13 * np.abs(u).max())


@pytest.mark.parametrize("kernel", [0, 2])
def test_direct_reciprocity(kernel):
    """The stokeslet matrix is symmetric and even, the rotlet antisymmetric and odd,
    so sum g.u(f) = sum f.u(g) for both."""
    x, f = W.stokeslet_uniform(80, 12)
    g = W.normal_vectors(80, 13)
    a = np.sum(g * direct.direct(kernel, x, f))
    b = np.sum(f * direct.direct(kernel, x, g))
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_direct_gradients_fd(kernel):
    """O1 position/strength gradients of L = sum g.u against central differences."""
    x, f = W.stokeslet_uniform(25, 14)
    q = W.unit_vectors(25, 14) if kernel == 1 else None
    g = W.normal_vectors(25, 15)
    gx = direct.grad_x(kernel, x, f, g, q)
    hh = 1e-6
    for p in (0, 7, 19):
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[p, a] += hh
            xm[p, a] -= hh
            fd = (np.sum(g * direct.direct(kernel, xp, f, q)) -
                  np.sum(g * direct.direct(kernel, xm, f, q))) / (2 * hh)
            assert abs(fd - gx[p, a]) <= 1e-6 * max(1.0, abs(fd))
    if kernel != 1:
        gf = direct.grad_f(kernel, x, g)
        for p in (2, 11):
            for a in range(3):
                fp = f.copy()
                fp[p, a] += 1.0
                fd = np.sum(g * direct.direct(kernel, x, fp)) - np.sum(g * direct.direct(kernel, x, f))
                assert abs(fd - gf[p, a]) <= 1e-10 * max(1.0, abs(fd))


def test_direct_stresslet_strength_gradients():
    """O1 stresslet gradients in f and q: L is linear in each f_p and each q_p, so a
    unit step gives the derivative exactly, and Euler's relation for the
    bilinear L gives sum f.dL/df = sum q.dL/dq = L."""
    x, f = W.stokeslet_uniform(30, 16)
    q = W.unit_vectors(30, 16)
    g = W.normal_vectors(30, 17)
    L0 = np.sum(g * direct.direct(1, x, f, q))
    gf, gq = direct.grad_fq(x, f, q, g)
    for p in (0, 13, 29):
        for a in range(3):
            fp = f.copy()
            fp[p, a] += 1.0
            qp = q.copy()
            qp[p, a] += 1.0
            dfd = np.sum(g * direct.direct(1, x, fp, q)) - L0
            dqd = np.sum(g * direct.direct(1, x, f, qp)) - L0
            assert abs(dfd - gf[p, a]) <= 1e-10 * max(1.0, abs(dfd))
            assert abs(dqd - gq[p, a]) <= 1e-10 * max(1.0, abs(dqd))
    assert abs(np.sum(f * gf) - L0) <= 1e-10 * abs(L0)
    assert abs(np.sum(q * gq) - L0) <= 1e-10 * abs(L0)
    sub = direct.grad_fq(x, f, q, g, targets=[4, 9])
    np.testing.assert_allclose(sub[0], gf[[4, 9]], rtol=1e-14, atol=0)


# ------------------------------------------------------ Ewald split (Section 3)

def _phi_hasimoto(xi):
    """r - Phi^H(r) with Phi^H from Table 1 (Hasimoto row)."""
    def phi(y):
        r = np.linalg.norm(y)
        return r - (r * special.erf(xi * r) + math.exp(-xi**2 * r**2) / (math.sqrt(math.pi) * xi))
    return phi


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_real_space_kernels_from_splitting(kernel):
    """K^R = K [r - Phi^H] (stokeslet, stresslet) and -eps d[erfc(xi r)/r] (rotlet),
    differentiated numerically; pins eqs. SR_Op, TR_Op (with the factor r in the
    delta-term) and RR_Op (halved for the definition normalisation)."""
    xi = 2.3
    r = R_TEST * 0.6
    if kernel == 2:
        phi = lambda y: special.erfc(xi * np.linalg.norm(y)) / np.linalg.norm(y)  # noqa: E731
    else:
        phi = _phi_hasimoto(xi)
    want = _operator_form(phi, r, kernel)
    got = direct.kernel_real(kernel, r, xi)[0].copy()
    if kernel != 1:
        got[:, :, 1:] = 0
    np.testing.assert_allclose(got, want, atol=3e-6 * np.abs(want).max())


def test_stresslet_printed_delta_term_fails_the_splitting_pin():
    """The printed TR_Op delta coefficient (4 xi^3/sqrt(pi)) e^{-xi^2 r^2} (no r) does
    not match the splitting function's derivatives; the oracle's does."""
    xi = 2.3
    r = R_TEST * 0.6
    rn = np.linalg.norm(r)
    want = _operator_form(_phi_hasimoto(xi), r, 1)
    got = direct.kernel_real(1, r, xi)[0]
    rh = r / rn
    I = np.eye(3)
    sym = np.einsum("jl,m->jlm", I, rh) + np.einsum("lm,j->jlm", I, rh) + np.einsum("mj,l->jlm", I, rh)
    ex = math.exp(-xi**2 * rn**2)
    printed = got - (4 * xi**3 * rn / math.sqrt(math.pi) * ex) * sym + (4 * xi**3 / math.sqrt(math.pi) * ex) * sym
    assert np.abs(printed - want).max() > 100 * np.abs(got - want).max()


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_real_space_limits(kernel):
    """xi -> 0 gives K^R -> K; r -> 0 gives K^R - K -> -4 xi/sqrt(pi) I (S, eq. Slimit), 0 (T, Omega)."""
    r = R_TEST
    np.testing.assert_allclose(direct.kernel_real(kernel, r, 1e-7)[0],
                               direct.kernel_full(kernel, r)[0], rtol=1e-6, atol=1e-9)
    xi = 1.7
    want = np.zeros((3, 3, 3))
    if kernel == 0:
        want[:, :, 0] = greens.self_coefficient(0, xi) * np.eye(3)
    # the remainder is O(r^2) for S and O(r) for T and Omega: shrinking r by 10
    # shrinks it by 100 and 10 (to within 10 %)
    d = []
    for s in (1e-2, 1e-3):
        rs = R_TEST * s
        d.append(np.abs(direct.kernel_real(kernel, rs, xi)[0] - direct.kernel_full(kernel, rs)[0]
                        - want).max())
    order = 2 if kernel == 0 else 1
    assert d[1] < 1.1 * d[0] / 10**order


@pytest.mark.parametrize("kernel", [0, 2])
def test_real_space_gradient_fd(kernel):
    xi = 3.1
    r = R_TEST * 0.4
    got = direct.kernel_real_grad(kernel, r, xi)[0]
    for j in range(3):
        for l in range(3):
            fd = _num_grad(lambda y: direct.kernel_real(kernel, y, xi)[0][j, l, 0], r, 1e-4)
            np.testing.assert_allclose(got[:, j, l], fd, atol=1e-7 * max(1, np.abs(fd).max()))


# ---------------------------------------- truncated Green's functions (Section 4)

@pytest.mark.parametrize("k", [0.0, 0.3, 1.7, 5.0, 23.0])
def test_truncated_transforms_vs_quadrature(k):
    """eqs. HhatR, BhatR: (4 pi / k) int_0^R r G(r) sin(kr) dr for G = 1/r, r; limits
    2 pi R^2 and pi R^4 at k = 0."""
    R = 1.3
    if k == 0.0:
        hq = 4 * math.pi * integrate.quad(lambda r: r, 0, R)[0]
        bq = 4 * math.pi * integrate.quad(lambda r: r**3, 0, R)[0]
        assert abs(hq - 2 * math.pi * R**2) < 1e-12
        assert abs(bq - math.pi * R**4) < 1e-12
    else:
        hq = 4 * math.pi / k * integrate.quad(lambda r: math.sin(k * r), 0, R, limit=200)[0]
        bq = 4 * math.pi / k * integrate.quad(lambda r: r**2 * math.sin(k * r), 0, R, limit=200)[0]
    assert greens.hhat_trunc(np.array([k]), R)[0] == pytest.approx(hq, rel=1e-10, abs=1e-12)
    assert greens.bhat_trunc(np.array([k]), R)[0] == pytest.approx(bq, rel=1e-10, abs=1e-12)


def test_truncated_biharmonic_series_branch_is_continuous():
    R = 2.0
    ks = np.array([0.3, 0.5, 0.7]) / R  # R k around the switch point
    series = greens.bhat_trunc(ks, R, series_below=10.0)
    closed = greens.bhat_trunc(ks, R, series_below=0.0)
    np.testing.assert_allclose(series, closed, rtol=1e-12)


def test_untruncated_limits():
    """For large R the truncated kernels approach 4 pi / k^2 and -8 pi / k^4 on average
    (eq. def_harm_biharm): average over an oscillation period of cos(Rk)."""
    k = 3.0
    R = np.linspace(200.0, 200.0 + 2 * math.pi / k, 4001)[:-1]
    h = np.mean([greens.hhat_trunc(np.array([k]), r)[0] for r in R])
    assert h == pytest.approx(greens.hhat(k), rel=1e-6)


def _gaussian_solve(kind, Mt=48, sigma=0.08):
    """Free-space solve of Section 4.1/4.3 with a Gaussian density centred in the box."""
    p = se.SEParams(L=1.0, M=Mt - 8, P=8, xi=5.0, rc=0.1)
    assert p.Mt == Mt
    h = p.h
    y = np.arange(Mt) * h
    c = y[Mt // 2]
    Z, Y, X = np.meshgrid(y, y, y, indexing="ij")
    r2 = (X - c) ** 2 + (Y - c) ** 2 + (Z - c) ** 2
    rho = np.exp(-r2 / (2 * sigma**2)) / (2 * math.pi * sigma**2) ** 1.5
    Gh = se.precompute_ghat(kind, p)
    import scipy.fft as sfft
    phi = sfft.ifftn(Gh * sfft.fftn(rho, s=(p.Mf,) * 3)).real[:Mt, :Mt, :Mt]
    return phi, np.sqrt(r2), sigma


def test_precompute_harmonic_solve_gaussian():
    """Section 4.3 mollified harmonic kernel: int rho(y)/|x-y| dy = erf(r/(sigma sqrt2))/r."""
    phi, r, s = _gaussian_solve("H")
    rr = np.where(r == 0, 1.0, r)
    exact = np.where(r == 0, math.sqrt(2 / math.pi) / s, special.erf(rr / (s * math.sqrt(2))) / rr)
    assert np.abs(phi - exact).max() < 1e-9 * np.abs(exact).max()


def test_precompute_biharmonic_solve_gaussian():
    """Section 4.3 mollified biharmonic kernel: int rho(y)|x-y| dy =
    sigma sqrt(2/pi) e^{-r^2/2 sigma^2} + (r + sigma^2/r) erf(r/(sigma sqrt2))."""
    phi, r, s = _gaussian_solve("B")
    rr = np.where(r == 0, 1.0, r)
    exact = s * math.sqrt(2 / math.pi) * np.exp(-r**2 / (2 * s**2)) + np.where(
        r == 0, s * math.sqrt(2 / math.pi), (rr + s**2 / rr) * special.erf(rr / (s * math.sqrt(2))))
    assert np.abs(phi - exact).max() < 1e-9 * np.abs(exact).max()


def test_precompute_is_real_and_even():
    p = se.SEParams(L=1.0, M=12, P=8, xi=5.0, rc=0.1)
    Gh = se.precompute_ghat("B", p)
    assert np.abs(Gh.imag).max() < 1e-10 * np.abs(Gh.real).max()
    g = Gh.real
    np.testing.assert_allclose(g, g[::-1, :, :][np.r_[-1, 0:p.Mf - 1]], rtol=1e-10,
                               atol=1e-12 * np.abs(g).max())


# ------------------------------------------------ Spectral Ewald steps (Section 5)

def test_spread_gather_adjoint_and_mass():
    """<gather(w), v> = h^3 <w, spread(v)> to roundoff; h^3 sum_i Gauss(y_i - x) = 1
    to the truncation level e^{-m^2/2} for an interior point."""
    p = se.SEParams(L=1.0, M=20, P=16, xi=8.0, rc=0.3)
    x = W.uniform_points(40, 21)
    v = W.normal_vectors(40, 22)
    w = W.normal_vectors(p.Mt**3, 23).T.reshape(3, p.Mt, p.Mt, p.Mt).copy()
    lhs = np.sum(se.gather(w, x, p) * v)
    rhs = p.h**3 * np.sum(w * se.spread(x, v, p))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    one = se.spread(np.array([[0.5, 0.5, 0.5]]), np.ones((1, 1)), p)
    assert abs(p.h**3 * one.sum() - 1.0) < 1e-6


def _fourier_brute(kernel, x, src9, q, xi):
    """u^F(x_m) = sum_{n != m} (K - K^R)(x_m - x_n) . s_n + lim_{r->0}(K - K^R) s_m."""
    N = len(x)
    u = np.zeros((N, 3))
    for m in range(N):
        r = x[m] - np.delete(x, m, axis=0)
        KF = direct.kernel_full(kernel, r) - direct.kernel_real(kernel, r, xi)
        fs = np.delete(src9, m, axis=0)
        if kernel == 1:
            qs = np.delete(q, m, axis=0)
            u[m] = np.einsum("njlm,nl,nm->j", KF, fs, qs)
        else:
            u[m] = np.einsum("njl,nl->j", KF[..., 0], fs)
    if kernel == 0:
        u += -greens.self_coefficient(0, xi) * src9
    return u


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_fourier_part_matches_closed_form_sum(kernel):
    """Steps 1-5 alone equal the closed-form Fourier-space sum with K^F = K - K^R
    (all pairs, plus the r -> 0 limit for the self image) to the P-controlled
    approximation level (P = 24: about 12 digits, Section 8.2)."""
    x, f = W.stokeslet_uniform(120, 31)
    q = W.unit_vectors(120, 31) if kernel == 1 else None
    xi = 5.0
    want = _fourier_brute(kernel, x, f, q, xi)
    parts = se.se_eval(kernel, x, f, q, M=24, P=24, xi=xi, rc=0.2, parts=True,
                       deltaL_policy="strict")
    assert rel(parts["F"], want) < 2e-12


@pytest.mark.parametrize("kernel", [0, 1])
def test_deltaL_condition_decouples_errors(kernel):
    """Section 5.3 / Fig. P_errors: with delta_L = d the approximation error grows when
    M is larger than xi needs (eta << 1); eq. deltaL_cond keeps it at the P level."""
    x, f = W.stokeslet_uniform(120, 31)
    q = W.unit_vectors(120, 31) if kernel == 1 else None
    xi = 5.0
    want = _fourier_brute(kernel, x, f, q, xi)
    kw = dict(M=32, P=24, xi=xi, rc=0.2, parts=True)
    e_d = rel(se.se_eval(kernel, x, f, q, **kw)["F"], want)
    e_strict = rel(se.se_eval(kernel, x, f, q, deltaL_policy="strict", **kw)["F"], want)
    assert e_strict < 2e-12 and e_d > 1e4 * e_strict


@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_se_matches_direct(kernel):
    """The whole method (Section 8) converges to the direct sum: relative L2 1e-9 at P=24."""
    x, f = W.stokeslet_uniform(250, 41)
    q = W.unit_vectors(250, 41) if kernel == 1 else None
    u = se.se_eval(kernel, x, f, q, M=28, P=24, xi=7.5, rc=0.7)
    assert rel(u, direct.direct(kernel, x, f, q)) < 1e-9


def test_se_xi_independence():
    """xi only balances work between real and Fourier space (Section 5.3)."""
    x, f = W.stokeslet_uniform(200, 42)
    q = W.unit_vectors(200, 42)
    for k in range(3):
        qq = q if k == 1 else None
        u1 = se.se_eval(k, x, f, qq, M=24, P=24, xi=6.0, rc=0.85)
        u2 = se.se_eval(k, x, f, qq, M=36, P=24, xi=9.0, rc=0.57)
        assert rel(u1, u2) < 2e-9


def test_se_p_convergence():
    """Approximation error decays exponentially in P (Section 5.3; P = 16 ~ 8 digits)."""
    x, f = W.stokeslet_uniform(200, 43)
    ref = direct.direct(0, x, f)
    errs = [rel(se.se_eval(0, x, f, M=32, P=P, xi=8.0, rc=0.7, deltaL_policy="strict"), ref)
            for P in (6, 10, 16)]
    assert errs[0] > 50 * errs[1] > 2500 * errs[2]
    assert errs[2] < 1e-8


def test_se_translation_by_grid_multiple_is_exact():
    """Shifting points and box by a multiple of h shifts the grid identically."""
    x, f = W.stokeslet_uniform(150, 44)
    M = 20
    h = 1.0 / M
    s = np.array([3 * h, -5 * h, 2 * h])
    u1 = se.se_eval(0, x, f, M=M, P=16, xi=6.0, rc=0.6)
    u2 = se.se_eval(0, x + s, f, x0=tuple(s), M=M, P=16, xi=6.0, rc=0.6)
    assert rel(u2, u1) < 1e-13


@pytest.mark.parametrize("kernel", [0, 2])
def test_se_operator_reciprocity(kernel):
    """The discrete SE operator is symmetric for S and Omega (spread = gather^T,
    symmetric multiplier, symmetric cutoff): sum g.SE(f) = sum f.SE(g) to roundoff,
    far below the approximation error (P = 8)."""
    x, f = W.stokeslet_uniform(150, 45)
    g = W.normal_vectors(150, 46)
    a = np.sum(g * se.se_eval(kernel, x, f, M=16, P=8, xi=5.0, rc=0.3))
    b = np.sum(f * se.se_eval(kernel, x, g, M=16, P=8, xi=5.0, rc=0.3))
    assert abs(a - b) < 1e-12 * (abs(a) + abs(b))


def test_strict_deltaL_policy():
    """eq. deltaL_cond extends the grid when eta < 1 and stays accurate."""
    p = se.SEParams(L=1.0, M=24, P=8, xi=6.0, rc=0.6, deltaL_policy="strict")
    assert p.eta < 1 and p.n_ext > p.P
    x, f = W.stokeslet_uniform(120, 47)
    ref = direct.direct(0, x, f)
    e_strict = rel(se.se_eval(0, x, f, M=24, P=8, xi=6.0, rc=0.6, deltaL_policy="strict"), ref)
    e_d = rel(se.se_eval(0, x, f, M=24, P=8, xi=6.0, rc=0.6), ref)
    assert e_strict < 1e-4 and e_strict < e_d / 10


# ------------------------------------------------------- estimates (Section 7)

@pytest.mark.parametrize("kernel", [0, 1, 2])
def test_error_estimates_track_measured_errors(kernel):
    """Tables 2 and 3 estimate the truncation errors within a small factor."""
    N, L = 400, 1.0
    x, f = W.stokeslet_uniform(N, 51)
    q = W.unit_vectors(N, 51) if kernel == 1 else None
    Q = params.q_sum(kernel, f, q)
    ref = direct.direct(kernel, x, f, q)
    xi = 8.0
    # real-space truncation with a very fine Fourier part
    rc = 0.25
    u = se.se_eval(kernel, x, f, q, M=48, P=24, xi=xi, rc=rc)
    meas = np.sqrt(np.mean(np.sum((u - ref) ** 2, axis=1)))
    est = params.real_error(kernel, Q, xi, L, rc)
    assert est / 10 < meas < est * 10
    # Fourier truncation with a long real-space cutoff
    M = 14 if kernel != 1 else 18
    parts = se.se_eval(kernel, x, f, q, M=M, P=24, xi=xi, rc=0.9, parts=True)
    u = parts["F"] + parts["R"] + parts["self"]
    meas = np.sqrt(np.mean(np.sum((u - ref) ** 2, axis=1)))
    est = params.fourier_error(kernel, Q, xi, L, M, parts["params"].R)
    assert est / 30 < meas < est * 30


# ------------------------------------------------------------ gradients

@pytest.mark.parametrize("kernel", [0, 2])
def test_se_gradients(kernel):
    """SE gradients (adjoint grid + Gaussian-derivative quadrature + real-space
    derivative) match the exact direct-sum gradients and central differences of
    the SE value itself."""
    x, f = W.stokeslet_uniform(60, 61)
    g = W.normal_vectors(60, 62)
    kw = dict(M=24, P=20, xi=6.5, rc=0.7)
    gf, gx = se.se_grad(kernel, x, f, g, **kw)
    assert rel(gf, direct.grad_f(kernel, x, g)) < 1e-8
    assert rel(gx, direct.grad_x(kernel, x, f, g)) < 1e-7
    hh = 1e-5
    for p_, a in ((3, 0), (40, 2)):
        xp, xm = x.copy(), x.copy()
        xp[p_, a] += hh
        xm[p_, a] -= hh
        fd = (np.sum(g * se.se_eval(kernel, xp, f, **kw)) - np.sum(g * se.se_eval(kernel, xm, f, **kw))) / (2 * hh)
        assert abs(fd - gx[p_, a]) < 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------------------ mutation checks

def test_mutations_are_caught(monkeypatch):
    """Plausible mistakes planted in copies of the oracle's steps fail a pin."""
    x, f = W.stokeslet_uniform(120, 71)
    ref = direct.direct(0, x, f)
    kw = dict(M=24, P=24, xi=6.8, rc=0.73)
    assert rel(se.se_eval(0, x, f, **kw), ref) < 1e-9
    orig_scale = se.scale
    orig_gather = se.gather

    # (a) dropped Hasimoto factor (1 + k^2 / 4 xi^2)
    def scale_no_hasimoto(kernel, Ghat, G, p, transpose=False):
        kx, ky, kz = se._kgrid(p)
        k2 = kx**2 + ky**2 + kz**2
        return orig_scale(kernel, Ghat / (1.0 + k2 / (4 * p.xi**2)), G, p, transpose)
    monkeypatch.setattr(se, "scale", scale_no_hasimoto)
    assert rel(se.se_eval(0, x, f, **kw), ref) > 1e-4
    monkeypatch.setattr(se, "scale", orig_scale)

    # (b) missing h^3 quadrature weight
    monkeypatch.setattr(se, "gather", lambda w, xt, p: orig_gather(w, xt, p) / p.h**3)
    assert rel(se.se_eval(0, x, f, **kw), ref) > 1e-2
    monkeypatch.setattr(se, "gather", orig_gather)

    # (c) eta factor applied twice in the middle Gaussian (e^{-k^2/4xi^2} instead of (1-eta))
    def scale_wrong_eta(kernel, Ghat, G, p, transpose=False):
        kx, ky, kz = se._kgrid(p)
        k2 = kx**2 + ky**2 + kz**2
        return orig_scale(kernel, Ghat * np.exp(-p.eta * k2 / (4 * p.xi**2)), G, p, transpose)
    monkeypatch.setattr(se, "scale", scale_wrong_eta)
    assert rel(se.se_eval(0, x, f, **kw), ref) > 1e-4
    monkeypatch.setattr(se, "scale", orig_scale)

    # (d) rotlet in the operator normalisation (x2) fails against the definition
    u2 = se.se_eval(2, x, f, **kw)
    assert rel(2 * u2, direct.direct(2, x, f)) > 0.5
