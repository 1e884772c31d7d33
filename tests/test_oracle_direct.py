"""Pins of the oracle's direct solver and of its App. A.4 spectral toolkit.

``direct_solve`` is the result definition at full size: the exact discrete
solution the V-cycle converges to.  It is pinned here against routes that do
not share its arithmetic: the dense LU solve of the Kronecker-assembled
operator (every boundary mix, anisotropic boxes, non-zero faces), the closed
forms of the sinusoidal eigenvectors (Dirichlet and periodic), and the
oracle's own multigrid driven to 1e-13.

``m_eff`` (Eqs. minimum_iteration, sopt_theory), ``first_zero_s`` and
``s_opt_global`` (App. A.4, the two-step search) are pinned against an
eigendecomposition of the RKL1 iteration matrix built from the 1D matrix of
Eq. M_matrix, against brute-force searches with numpy's Legendre series, and
against the two numbers the paper prints for the m_eff curve of Fig.
spectral_iteration (the curve decreases up to s = 35 and has its global
minimum at s = 56).  The paper does not state the N of that figure; N = 64 is
the size at which the oracle's curve shows both printed facts, and the test
records that reading.

The last tests plant mistakes in the oracle and check that the pins catch them.
"""

import json
import math
import os

import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

import oracle
import oracle.sg_oracle as S
import workloads as W

O = oracle
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def P(s, x):
    """Legendre P_s by numpy's series evaluation (independent of the oracle)."""
    c = np.zeros(s + 1)
    c[s] = 1.0
    return npleg.legval(x, c)


def rel_max(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


# ---------------------------------------------------------------------------
# direct_solve
# ---------------------------------------------------------------------------

DENSE_CASES = [((8, 8, 8), (0, 0, 0), (1.0, 1.0, 1.0)),
               ((8, 8, 8), (1, 1, 1), (1.0, 1.0, 1.0)),
               ((6, 4, 8), (1, 0, 0), (1.5, 2.0, 1.0)),
               ((4, 6, 8), (0, 1, 1), (1.0, 0.5, 2.0)),
               ((5, 7, 3), (0, 0, 0), (0.7, 1.3, 1.1))]


@pytest.mark.parametrize("shape,bc,box", DENSE_CASES)
def test_direct_solve_matches_dense_lu(shape, bc, box):
    rho = W.random_field(shape, 11) + 0.3
    faces = W.random_faces(shape, 12)
    lo = (0.0, -0.5, 0.25)
    hi = tuple(l + b for l, b in zip(lo, box))
    a = O.direct_solve(rho, lo, hi, bc, faces, 2.5)
    b = O.dense_solve(rho, lo, hi, bc, faces, 2.5)
    assert rel_max(a, b) < 1e-12


def test_direct_solve_dirichlet_sinusoid_closed_form():
    # sin(pi x) sin(pi y) sin(pi z) at cell centres of [0, 1]^3 is an exact
    # eigenvector of the cell-centred operator with phi = 0 faces:
    # lambda = -(12 / h^2) sin^2(pi h / 2)
    n = 32
    p = W.sinusoid(n)
    h = 1.0 / n
    lam = -(12.0 / h ** 2) * math.sin(math.pi * h / 2) ** 2
    phi = O.direct_solve(p.rho, p.lo, p.hi, p.bc, None, 1.0)
    assert rel_max(phi, p.rho / lam) < 1e-13


def test_direct_solve_periodic_mode_closed_form():
    # cos(2 pi x) cos(4 pi y) sin(2 pi z) on the periodic unit cube (12 x 16 x 8
    # cells): lambda = -(4/hx^2) sin^2(pi hx) - (4/hy^2) sin^2(2 pi hy) - (4/hz^2) sin^2(pi hz)
    nz, ny, nx = 12, 16, 8
    X, Y, Z = W.mesh((nz, ny, nx), (0, 0, 0), (1, 1, 1))
    rho = np.cos(2 * np.pi * X) * np.cos(4 * np.pi * Y) * np.sin(2 * np.pi * Z)
    hx, hy, hz = 1.0 / nx, 1.0 / ny, 1.0 / nz
    lam = (-(4 / hx ** 2) * math.sin(math.pi * hx) ** 2 - (4 / hy ** 2) * math.sin(2 * math.pi * hy) ** 2
           - (4 / hz ** 2) * math.sin(math.pi * hz) ** 2)
    phi = O.direct_solve(rho + 3.0, (0, 0, 0), (1, 1, 1), (1, 1, 1), None, 1.0)   # the mean is removed
    assert rel_max(phi, rho / lam) < 1e-13
    assert abs(phi.mean()) < 1e-15


@pytest.mark.parametrize("shape,bc", [((32, 32, 32), (0, 0, 0)), ((16, 32, 24), (1, 0, 0))])
def test_multigrid_converges_to_direct_solve(shape, bc):
    rho = W.random_field(shape, 21)
    faces = W.random_faces(shape, 22)
    lo, hi = (0.0, 0.0, 0.0), (1.5, 2.0, 1.0)
    ref = O.direct_solve(rho, lo, hi, bc, faces, 2.0)
    phi, info = O.solve(rho, lo, hi, bc, faces, 2.0, tol=1e-13)
    assert info.rel_residual <= 1e-13
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-11


def test_direct_solve_residual_of_the_sphere_benchmark_at_64():
    p = W.sphere(64)
    phi = O.direct_solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0)
    h = O.spacing(p.shape, p.lo, p.hi)
    f = O.source(p.rho, 1.0, p.bc)
    r0 = O.l2norm(O.residual(np.zeros(p.shape), f, h, p.bc, p.faces))
    assert O.l2norm(O.residual(phi, f, h, p.bc, p.faces)) / r0 < 1e-13


def lambda_min(shape, h, bc):
    """Smallest |eigenvalue| of L_h with homogeneous ghosts: the lowest mode
    of every Dirichlet axis plus the zero mode of every periodic axis; with
    every axis periodic, the lowest non-zero mode (the mean-free subspace)."""
    if all(b == O.PERIODIC for b in bc):
        return min((4.0 / h[d] ** 2) * math.sin(math.pi / shape[2 - d]) ** 2 for d in range(3))
    return sum((4.0 / h[d] ** 2) * math.sin(math.pi / (2 * shape[2 - d])) ** 2
               for d in range(3) if bc[d] != O.PERIODIC)


def error_bound_factor(p, ref):
    """K with ||phi - ref|| / ||ref|| <= K ||L phi - f|| / ||L 0 - f|| for any
    phi: the error e = phi - ref solves L_0 e = r (homogeneous ghosts, L_0
    symmetric), so ||e|| <= ||r|| / lambda_min, and ||L 0 - f|| is the norm of
    the right-hand side of L_0 ref = f - b."""
    h = O.spacing(p.shape, p.lo, p.hi)
    f = O.source(p.rho, p.four_pi_G, p.bc)
    rhs0 = O.laplacian(np.zeros(p.shape), h, p.bc, p.faces) - f
    return float(np.linalg.norm(rhs0) / (lambda_min(p.shape, h, p.bc) * np.linalg.norm(ref)))


def test_error_bound_factor_holds_on_a_multigrid_iterate():
    # the bound the full-size GPU tests use, checked against the direct
    # solution on partly converged oracle solves (Dirichlet and periodic)
    for p in (W.sphere(32), W.grf(32, seed=3)):
        h = O.spacing(p.shape, p.lo, p.hi)
        f = O.source(p.rho, p.four_pi_G, p.bc)
        ref = O.direct_solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G)
        phi, info = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, cycles=2)
        K = error_bound_factor(p, ref)
        err = np.linalg.norm(phi - ref) / np.linalg.norm(ref)
        rel_r = info.rel_residual
        assert err <= K * rel_r * (1 + 1e-9)
        assert err > 1e-3 * K * rel_r          # the bound is not vacuous


# ---------------------------------------------------------------------------
# App. A.4: m_eff, first zero, global s_opt, Fig. sk_opt
# ---------------------------------------------------------------------------

def rkl1_iteration_matrix(N, s):
    """R = Y_s of one RKL1 super-step at tau_max on the 1D matrix of Eq.
    M_matrix (dx = 1), built by running the stage recursion on matrices."""
    M = np.diag(-2.0 * np.ones(N - 1)) + np.diag(np.ones(N - 2), 1) + np.diag(np.ones(N - 2), -1)
    w1 = 2.0 / (s * s + s)
    tau = 1.0 / (2.0 * w1)            # tau_max = dx^2 / (2 w1)
    I = np.eye(N - 1)
    y_prev, y = I, I + w1 * tau * M
    for j in range(2, s + 1):
        y_prev, y = y, (2.0 * j - 1.0) / j * (y + w1 * tau * M @ y) - (j - 1.0) / j * y_prev
    return y


@pytest.mark.parametrize("N,s", [(16, 5), (32, 12), (64, 20), (64, 56)])
def test_m_eff_against_iteration_matrix_eigenvalues(N, s):
    rho = float(np.max(np.abs(np.linalg.eigvalsh(rkl1_iteration_matrix(N, s)))))
    d = 2.0
    expect = s * d / -math.log10(rho)
    assert abs(O.m_eff(s, N, d, kmax=N // 2) - expect) <= 1e-8 * expect


def test_m_eff_counts_super_steps_that_gain_d_decades():
    # m_RKL = m_eff / s super-steps shrink the slowest mode by 10^d: one fewer
    # (rounded up) does not
    N, s, d = 64, 20, 2.0
    R = rkl1_iteration_matrix(N, s)
    m = O.m_eff(s, N, d, kmax=N // 2) / s
    ev, V = np.linalg.eigh(R)
    v = V[:, int(np.argmax(np.abs(ev)))]
    need = math.ceil(m)
    x = v.copy()
    for _ in range(need - 1):
        x = R @ x
    assert np.linalg.norm(x) > 10 ** -d
    x = R @ x
    assert np.linalg.norm(x) <= 10 ** -d * (1 + 1e-12)


def test_m_eff_curve_of_fig_spectral_iteration():
    # the paper: m_eff decreases with s up to s = 35, then oscillates, with its
    # global minimum at s = 56 (N of the figure not stated; N = 64 reproduces both)
    g = GOLDEN["m_eff_curve"]
    N = g["N_reading"]
    m = [O.m_eff(s, N, 2.0) for s in range(1, N + 1)]
    onset = g["monotone_up_to_s"]
    assert all(m[s] < m[s - 1] for s in range(1, onset))
    assert m[onset] > m[onset - 1]
    assert int(np.argmin(m)) + 1 == g["global_min_s"]


def test_first_zero_by_brute_force():
    for N in (16, 32, 64, 128):
        for k in range(1, N // 2 + 1):
            x = math.cos(k * math.pi / N)
            s = 1
            while P(s, x) > 0.0:
                s += 1
            assert O.first_zero_s(k, N) == s, (N, k)


def test_global_s_opt_over_the_whole_range():
    # App. A.4: restricting the search to [first zero of lambda_1, N] does not
    # change the minimiser of the six-mode spectral radius over 1 <= s <= N
    for N in (32, 64, 100):
        radii = [max(abs(P(s, math.cos(k * math.pi / N))) for k in range(1, 7)) for s in range(1, N + 1)]
        assert O.s_opt_global(N) == int(np.argmin(radii)) + 1


def test_sk_opt_table_of_fig_sk_opt():
    # Fig. sk_opt: s_k,opt against k (Eq. sk_optimal) at N = 64 lies within one
    # of the first zero of P_s(cos k pi / N) for every k <= N/2 and never grows with k
    N = 64
    table = [O.s_k_opt(k, N) for k in range(1, N // 2 + 1)]
    assert all(a >= b for a, b in zip(table, table[1:]))
    for k, s in enumerate(table, start=1):
        assert abs(s - O.first_zero_s(k, N)) <= 1, k
    assert table[0] == 48 and table[-1] == 1


# ---------------------------------------------------------------------------
# Planted mistakes
# ---------------------------------------------------------------------------

def _pins():
    return [
        lambda: test_direct_solve_matches_dense_lu(*DENSE_CASES[0]),
        lambda: test_direct_solve_matches_dense_lu(*DENSE_CASES[1]),
        lambda: test_direct_solve_matches_dense_lu(*DENSE_CASES[2]),
        lambda: test_direct_solve_dirichlet_sinusoid_closed_form(),
        lambda: test_direct_solve_periodic_mode_closed_form(),
        lambda: test_m_eff_against_iteration_matrix_eigenvalues(32, 12),
        lambda: test_m_eff_counts_super_steps_that_gain_d_decades(),
        lambda: test_m_eff_curve_of_fig_spectral_iteration(),
        lambda: test_first_zero_by_brute_force(),
    ]


def _failures():
    n = 0
    for pin in _pins():
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:
            n += 1
    return n


def _eig_no_half(n, hd, periodic):
    m = np.arange(n) if periodic else np.arange(1, n + 1)
    return -(4.0 / (hd * hd)) * np.sin(np.pi * m / n) ** 2


def _eig_dst1(n, hd, periodic):
    m = np.arange(n) if periodic else np.arange(1, n + 1)
    arg = np.pi * m / n if periodic else np.pi * m / (2.0 * n + 2.0)
    return -(4.0 / (hd * hd)) * np.sin(arg) ** 2


def _m_eff_ln(s, N, d=2.0, kmax=6):
    rho = S.spectral_radius(s, N, kmax)
    return s * d / (-math.log(rho))


def _m_eff_no_s(s, N, d=2.0, kmax=6):
    rho = S.spectral_radius(s, N, kmax)
    return d / (-math.log10(rho))


ORIG_FZ = S.first_zero_s


@pytest.mark.parametrize("name,fn", [
    ("_axis_eigenvalues", _eig_no_half),
    ("_axis_eigenvalues", _eig_dst1),
    ("m_eff", _m_eff_ln),
    ("m_eff", _m_eff_no_s),
    ("first_zero_s", lambda k, N: ORIG_FZ(k, N) + 1),
])
def test_planted_mistakes_are_caught(monkeypatch, name, fn):
    monkeypatch.setattr(S, name, fn)
    if hasattr(oracle, name):
        monkeypatch.setattr(oracle, name, fn)
    assert _failures() >= 1


def test_planted_boundary_term_without_factor_two_is_caught(monkeypatch):
    orig = S.direct_solve

    def half_faces(rho, lo, hi, bc, faces=None, four_pi_G=1.0):
        return orig(rho, lo, hi, bc, None if faces is None else [0.5 * f for f in faces], four_pi_G)

    monkeypatch.setattr(S, "direct_solve", half_faces)
    monkeypatch.setattr(oracle, "direct_solve", half_faces)
    assert _failures() >= 1


def test_unmutated_pins_pass():
    assert _failures() == 0
