"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types an oracle formula: each compares the oracle with an
independent route (numpy's Legendre series, a Kronecker-product matrix, FFT or
DST diagonalisation, an eigendecomposition, brute force, closed forms, or a
number printed in the paper).  A plausible slip in the oracle (a sign, a
dropped term, a wrong coefficient, a transposed axis, a wrong ghost rule)
fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest
import scipy.fft as sfft
import scipy.special as sps
from numpy.polynomial import legendre as npleg

import oracle as O
import workloads as W

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def P(s, x):
    """Legendre P_s via numpy's series evaluation (independent of the oracle)."""
    c = np.zeros(s + 1)
    c[s] = 1.0
    return npleg.legval(x, c)


# ---------------------------------------------------------------------------
# RKL stage recursion vs stability polynomials (App. A)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("s", [1, 2, 3, 5, 8, 13, 24])
def test_rkl1_stages_are_legendre(s):
    co = O.rkl1_coefficients(s)
    z = np.linspace(-2.0 / co.w1, 0.0, 41)
    Y = O.rkl_scalar_stages(1, s, z)
    for j in range(s + 1):
        np.testing.assert_allclose(Y[j], P(j, 1.0 + co.w1 * z), atol=1e-12, rtol=0)
    assert abs(co.w1 - 2.0 / (s * s + s)) < 1e-15


@pytest.mark.parametrize("s", [2, 3, 4, 5, 8, 13])
def test_rkl2_stages_are_shifted_legendre(s):
    co = O.rkl2_coefficients(s)
    z = np.linspace(-2.0 / co.w1, 0.0, 41)
    Y = O.rkl_scalar_stages(2, s, z)
    for j in range(s + 1):
        bj = 1.0 / 3.0 if j <= 2 else (j * j + j - 2.0) / (2.0 * j * (j + 1.0))
        np.testing.assert_allclose(Y[j], (1.0 - bj) + bj * P(j, 1.0 + co.w1 * z), atol=1e-12, rtol=0)


@pytest.mark.parametrize("order,s", [(1, 3), (1, 8), (2, 3), (2, 7)])
def test_rkl_order_of_accuracy(order, s):
    # R_s(z) matches exp(z) to first (RKL1) or second (RKL2) order.
    errs = []
    for z in (-4e-3, -2e-3):
        R = float(O.rkl_scalar_stages(order, s, np.array(z))[-1])
        taylor = 1.0 + z + (z * z / 2.0 if order == 2 else 0.0)
        errs.append(abs(R - taylor))
    ratio = errs[0] / errs[1]
    assert abs(ratio - 2.0 ** (order + 1)) < 0.25 * 2.0 ** (order + 1)


@pytest.mark.parametrize("order,s", [(1, 2), (1, 7), (2, 3), (2, 6)])
def test_rkl_stable_up_to_tau_max(order, s):
    co = O.rkl_coefficients(order, s)
    z = np.linspace(-2.0 / co.w1, 0.0, 2001)
    R = O.rkl_scalar_stages(order, s, z)[-1]
    assert np.max(np.abs(R)) <= 1.0 + 1e-12
    # tau_max maps the largest |lambda| to x = -1 (Eq. tau_max)
    h = (0.1, 0.2, 0.3)
    lam = -4.0 * sum(1.0 / hd ** 2 for hd in h)
    tau = O.tau_step(order, s, h, 1.0)
    assert abs(1.0 + co.w1 * tau * lam + 1.0) < 1e-12


# ---------------------------------------------------------------------------
# Operator: Laplacian and ghost rules vs a Kronecker-product matrix
# ---------------------------------------------------------------------------

def kron_operator(shape, h, bc):
    """L_h assembled from 1D second differences (cell-centred, Dirichlet ghost
    = -active -> corner entry -3; periodic -> circulant)."""
    def d2(n, b):
        T = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        if b == O.PERIODIC:
            T[0, -1] += 1.0
            T[-1, 0] += 1.0
        else:
            T[0, 0] -= 1.0
            T[-1, -1] -= 1.0
        return T
    nz, ny, nx = shape
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)
    return (np.kron(Iz, np.kron(Iy, d2(nx, bc[0]))) / h[0] ** 2
            + np.kron(Iz, np.kron(d2(ny, bc[1]), Ix)) / h[1] ** 2
            + np.kron(d2(nz, bc[2]), np.kron(Iy, Ix)) / h[2] ** 2)


@pytest.mark.parametrize("shape,bc", [((4, 3, 5), (0, 0, 0)), ((4, 6, 2), (1, 1, 1)),
                                      ((3, 4, 4), (1, 0, 1)), ((6, 4, 8), (0, 1, 0))])
def test_laplacian_matches_kronecker_matrix(shape, bc):
    h = (0.3, 0.5, 0.7)
    A = kron_operator(shape, h, bc)
    np.testing.assert_allclose(O.dense_operator(shape, h, bc), A, atol=1e-12, rtol=0)


def test_dirichlet_faces_enter_as_two_g_over_h2():
    shape, h, bc = (3, 4, 5), (0.25, 0.5, 0.125), (0, 0, 0)
    faces = W.random_faces(shape, 3)
    b = O.laplacian(np.zeros(shape), h, bc, faces)
    expect = np.zeros(shape)
    expect[:, :, 0] += 2 * faces[0] / h[0] ** 2
    expect[:, :, -1] += 2 * faces[1] / h[0] ** 2
    expect[:, 0, :] += 2 * faces[2] / h[1] ** 2
    expect[:, -1, :] += 2 * faces[3] / h[1] ** 2
    expect[0, :, :] += 2 * faces[4] / h[2] ** 2
    expect[-1, :, :] += 2 * faces[5] / h[2] ** 2
    np.testing.assert_allclose(b, expect, atol=1e-12, rtol=0)


def test_laplacian_is_symmetric_homogeneous():
    for bc in [(0, 0, 0), (1, 1, 1), (0, 1, 0)]:
        shape, h = (6, 5, 8), (0.1, 0.2, 0.15)
        u, v = W.random_field(shape, 1), W.random_field(shape, 2)
        a = np.sum(O.laplacian(u, h, bc) * v)
        b = np.sum(u * O.laplacian(v, h, bc))
        assert abs(a - b) <= 1e-11 * abs(a)


def test_sinusoid_is_exact_eigenvector():
    p = W.sinusoid(32)
    h = O.spacing(p.shape, p.lo, p.hi)
    lam = -(12.0 / h[0] ** 2) * math.sin(math.pi * h[0] / 2.0) ** 2
    Lr = O.laplacian(p.rho, h, p.bc)
    np.testing.assert_allclose(Lr, lam * p.rho, atol=1e-10 * abs(lam), rtol=0)
    assert abs(lam / (-3 * math.pi ** 2) - 0.999197) < 1e-6


# ---------------------------------------------------------------------------
# RKL super-step on the 3D operator
# ---------------------------------------------------------------------------

def test_jacobi_special_case():
    # RKL1, s = 1, tau = tau_max = h^2/6 is Jacobi: u <- (sum nb - h^2 f) / 6.
    shape, h = (6, 6, 6), (0.2, 0.2, 0.2)
    u, f = W.random_field(shape, 4), W.random_field(shape, 5)
    out = O.rkl_superstep(u, f, h, (1, 1, 1), None, 1, 1, 1.0)
    nb = sum(np.roll(u, sh, axis=a) for a in range(3) for sh in (1, -1))
    np.testing.assert_allclose(out, (nb - h[0] ** 2 * f) / 6.0, atol=1e-12, rtol=0)
    # homogeneous Dirichlet: ghost = -u via a negated symmetric pad
    p = np.pad(u, 1, mode="symmetric")
    for ax in range(3):
        sl_lo = [slice(None)] * 3
        sl_hi = [slice(None)] * 3
        sl_lo[ax], sl_hi[ax] = 0, -1
        p[tuple(sl_lo)] *= -1.0
        p[tuple(sl_hi)] *= -1.0
    nb = (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] + p[1:-1, :-2, 1:-1] + p[1:-1, 2:, 1:-1]
          + p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:])
    out = O.rkl_superstep(u, f, h, (0, 0, 0), None, 1, 1, 1.0)
    np.testing.assert_allclose(out, (nb - h[0] ** 2 * f) / 6.0, atol=1e-12, rtol=0)


@pytest.mark.parametrize("order,s,c", [(1, 4, 1.0), (1, 3, 0.7), (2, 3, 1.0), (2, 5, 0.8)])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_superstep_error_propagation_matrix(order, s, c, bc):
    # e^(1) = R e^(0) with R = a_s + b_s P_s(I + w1 tau A) (Eqs. Iteration_matrix, error).
    shape, h = (4, 4, 6), (0.25, 0.25, 0.2)
    A = kron_operator(shape, h, bc)
    lam, V = np.linalg.eigh(A)
    co = O.rkl_coefficients(order, s)
    tau = O.tau_step(order, s, h, c)
    x = 1.0 + co.w1 * tau * lam
    if order == 1:
        Rl = P(s, x)
    else:
        bs = (s * s + s - 2.0) / (2.0 * s * (s + 1.0))
        Rl = (1.0 - bs) + bs * P(s, x)
    R = (V * Rl) @ V.T
    f = W.random_field(shape, 7)
    if bc == (1, 1, 1):
        f -= f.mean()
    exact = np.linalg.lstsq(A, f.ravel(), rcond=None)[0]
    exact -= exact.mean() if bc == (1, 1, 1) else 0.0
    u0 = W.random_field(shape, 8)
    u1 = O.rkl_superstep(u0, f, h, bc, None, order, s, c)
    e0 = exact - u0.ravel()
    e1 = exact - u1.ravel()
    if bc == (1, 1, 1):
        e0 -= e0.mean()
        e1 -= e1.mean()
    np.testing.assert_allclose(e1, R @ e0, atol=1e-10 * np.abs(e0).max(), rtol=0)


def test_single_level_rkl1_closed_form():
    # Config-1 closed form: from phi = 0 the error shrinks by P_s(cos(pi/N))
    # per super-step (only the (1,1,1) mode is present, tau = tau_max).
    p = W.sinusoid(32)
    h = O.spacing(p.shape, p.lo, p.hi)
    lam = -(12.0 / h[0] ** 2) * math.sin(math.pi * h[0] / 2.0) ** 2
    exact = p.rho / lam
    s = O.s_k_opt(1, 32)
    assert s == 24
    g = P(s, math.cos(math.pi / 32))
    phi = np.zeros(p.shape)
    for m in range(1, 4):
        phi = O.rkl_superstep(phi, p.rho, h, p.bc, None, 1, s, 1.0)
        np.testing.assert_allclose(phi - exact, -(g ** m) * exact, atol=1e-13 * np.abs(exact).max() + 1e-15, rtol=0)
    opts = O.Options(single_s=24, single_tau_frac=1.0)
    phi, info = O.solve(p.rho, p.lo, p.hi, p.bc, None, 1.0, tol=1e-10, levels=1, opts=opts)
    assert info.cycles == 3
    np.testing.assert_allclose(info.history[1], abs(g), rtol=1e-9)


def test_residual_and_error_decay_monotonically():
    shape = (8, 8, 8)
    lo, hi = (0, 0, 0), (1, 1, 1)
    h = O.spacing(shape, lo, hi)
    f = W.random_field(shape, 11)
    u = np.zeros(shape)
    exact = O.dense_solve(f, lo, hi, (0, 0, 0))
    prev_e = prev_r = np.inf
    for s in (1, 2, 3, 5, 8):
        for _ in range(3):
            u = O.rkl_superstep(u, f, h, (0, 0, 0), None, 1, s, 1.0)
            e = np.linalg.norm(u - exact)
            r = np.linalg.norm(O.residual(u, f, h, (0, 0, 0)))
            assert e <= prev_e * (1 + 1e-12) and r <= prev_r * (1 + 1e-12)
            prev_e, prev_r = e, r


# ---------------------------------------------------------------------------
# Transfer operators
# ---------------------------------------------------------------------------

def test_restriction_and_prolongation_invariants():
    rng = np.random.default_rng(0)
    fine = np.full((8, 6, 4), 3.5)
    np.testing.assert_allclose(O.restrict(fine), 3.5, atol=1e-15)
    # restriction of a random field: explicit 8-child average of one coarse cell
    r = rng.standard_normal((8, 6, 4))
    rc = O.restrict(r)
    assert abs(rc[1, 2, 1] - r[2:4, 4:6, 2:4].mean()) < 1e-14
    # periodic prolongation preserves constants and the mean
    c = np.full((4, 3, 2), -1.25)
    np.testing.assert_allclose(O.prolong(c, (1, 1, 1)), -1.25, atol=1e-15)
    e = rng.standard_normal((4, 4, 4))
    assert abs(O.prolong(e, (1, 1, 1)).mean() - e.mean()) < 1e-14
    # linear functions are reproduced away from the walls
    X, Y, Z = W.mesh((4, 4, 4), (0, 0, 0), (1, 1, 1))
    lin = 0.3 + 1.7 * X - 0.9 * Y + 2.2 * Z
    Xf, Yf, Zf = W.mesh((8, 8, 8), (0, 0, 0), (1, 1, 1))
    linf = 0.3 + 1.7 * Xf - 0.9 * Yf + 2.2 * Zf
    pf = O.prolong(lin, (0, 0, 0))
    np.testing.assert_allclose(pf[1:-1, 1:-1, 1:-1], linf[1:-1, 1:-1, 1:-1], atol=1e-13)
    # Dirichlet wall: error ghost -e makes the first fine cell half the coarse value
    line = np.zeros((2, 2, 2))
    line[:, :, 0] = 1.0
    pe = O.prolong(line, (0, 1, 1))                # x Dirichlet, y and z periodic
    assert abs(pe[0, 0, 0] - 0.5) < 1e-15          # (3*1 + 1*(-1))/4 in x, flat in y, z
    assert abs(pe[0, 0, 1] - 0.75) < 1e-15         # (3*1 + 1*0)/4


def test_prolongation_weights_27_9_3_1():
    # a single unit coarse value spreads with tensor weights (3/4, 1/4)^3
    c = np.zeros((3, 3, 3))
    c[1, 1, 1] = 64.0
    pf = O.prolong(c, (1, 1, 1))
    assert pf[2, 2, 2] == 27.0 and pf[3, 3, 3] == 27.0
    assert pf[1, 2, 2] == 9.0 and pf[2, 1, 2] == 9.0 and pf[2, 2, 1] == 9.0
    assert pf[1, 1, 2] == 3.0 and pf[1, 2, 1] == 3.0 and pf[2, 1, 1] == 3.0
    assert pf[1, 1, 1] == 1.0 and pf[4, 4, 4] == 1.0
    assert pf[0, 2, 2] == 0.0


# ---------------------------------------------------------------------------
# Whole solves vs direct solvers
# ---------------------------------------------------------------------------

def dst_solve(f, h, faces):
    """Cell-centred Dirichlet: modes sin(pi m (i+1/2)/N), m = 1..N, i.e. DST-II."""
    rhs = f - O_boundary(f.shape, h, faces)
    nz, ny, nx = f.shape
    lam = lambda n, hd: -(4.0 / hd ** 2) * np.sin(np.pi * np.arange(1, n + 1) / (2 * n)) ** 2
    Lz, Ly, Lx = np.meshgrid(lam(nz, h[2]), lam(ny, h[1]), lam(nx, h[0]), indexing="ij")
    fk = sfft.dstn(rhs, type=2)
    return sfft.idstn(fk / (Lx + Ly + Lz), type=2)


def O_boundary(shape, h, faces):
    b = np.zeros(shape)
    if faces is None:
        return b
    b[:, :, 0] += 2 * faces[0] / h[0] ** 2
    b[:, :, -1] += 2 * faces[1] / h[0] ** 2
    b[:, 0, :] += 2 * faces[2] / h[1] ** 2
    b[:, -1, :] += 2 * faces[3] / h[1] ** 2
    b[0, :, :] += 2 * faces[4] / h[2] ** 2
    b[-1, :, :] += 2 * faces[5] / h[2] ** 2
    return b


def fft_solve(f, h):
    nz, ny, nx = f.shape
    k = lambda n, hd: -(4.0 / hd ** 2) * np.sin(np.pi * np.fft.fftfreq(n) * n / n) ** 2
    Lz, Ly, Lx = np.meshgrid(k(nz, h[2]), k(ny, h[1]), k(nx, h[0]), indexing="ij")
    den = Lx + Ly + Lz
    fk = np.fft.fftn(f - f.mean())
    den[0, 0, 0] = 1.0
    fk[0, 0, 0] = 0.0
    return np.real(np.fft.ifftn(fk / den))


def test_multigrid_matches_dst_direct_solve():
    p = W.sphere(32)
    h = O.spacing(p.shape, p.lo, p.hi)
    ref = dst_solve(p.four_pi_G * p.rho, h, p.faces)
    opts = O.Options(rkl_order=2, s_smooth=3)
    phi, info = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, tol=1e-13, levels=4, opts=opts)
    assert info.rel_residual <= 1e-13
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-11


def test_multigrid_matches_fft_direct_solve_periodic():
    p = W.grf(32, seed=3)
    p.rho = p.rho + 2.0            # a positive density: the mean must be removed
    h = O.spacing(p.shape, p.lo, p.hi)
    ref = fft_solve(p.rho, h)
    opts = O.Options(rkl_order=1, s_smooth=2, tau_frac=0.75)
    phi, info = O.solve(p.rho, p.lo, p.hi, p.bc, None, 1.0, tol=1e-13, opts=opts)
    assert info.rel_residual <= 1e-13
    assert abs(phi.mean()) < 1e-14
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-11


@pytest.mark.parametrize("shape,bc,box", [((8, 8, 8), (0, 0, 0), (1, 1, 1)),
                                          ((6, 4, 8), (0, 0, 0), (1, 2, 0.5)),
                                          ((8, 8, 8), (1, 1, 1), (1, 1, 1)),
                                          ((4, 8, 8), (1, 0, 1), (2, 1, 1))])
def test_solve_matches_kronecker_direct(shape, bc, box):
    lo = (0.0, 0.0, 0.0)
    hi = box
    h = O.spacing(shape, lo, hi)
    rho = W.random_field(shape, 21)
    faces = None if all(b == 1 for b in bc) else W.random_faces(shape, 22)
    f = O.source(rho, 1.0, bc)
    A = kron_operator(shape, h, bc)
    b = np.zeros(shape)
    if faces is not None:
        for d in range(3):
            if bc[d] == O.DIRICHLET:
                ax = 2 - d
                lo_idx = [slice(None)] * 3
                hi_idx = [slice(None)] * 3
                lo_idx[ax], hi_idx[ax] = 0, -1
                b[tuple(lo_idx)] += 2 * faces[2 * d] / h[d] ** 2
                b[tuple(hi_idx)] += 2 * faces[2 * d + 1] / h[d] ** 2
    if all(x == 1 for x in bc):
        ref = np.linalg.lstsq(A, (f - b).ravel(), rcond=None)[0]
        ref -= ref.mean()
    else:
        ref = np.linalg.solve(A, (f - b).ravel())
    ref = ref.reshape(shape)
    np.testing.assert_allclose(O.dense_solve(rho, lo, hi, bc, faces), ref, atol=1e-10 * np.abs(ref).max())
    opts = O.Options(rkl_order=1, s_smooth=2, tau_frac=0.75, coarse_tol=1e-6, coarse_max_ss=200)
    phi, info = O.solve(rho, lo, hi, bc, faces, 1.0, tol=1e-13, opts=opts)
    assert info.rel_residual <= 1e-13
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-11


def test_vcycle_fixed_point():
    shape, lo, hi = (16, 16, 16), (0, 0, 0), (1, 1, 1)
    h = O.spacing(shape, lo, hi)
    rho = W.random_field(shape, 31)
    faces = W.random_faces(shape, 32)
    exact = dst_solve(rho, h, faces)
    opts = O.Options()
    out = O.vcycle(exact.copy(), rho, h, (0, 0, 0), faces, 3, opts)
    np.testing.assert_allclose(out, exact, atol=1e-11 * np.abs(exact).max())


@pytest.mark.parametrize("order,s,c", [(2, 2, 1.0), (2, 4, 1.0), (2, 3, 1.0), (2, 2, 0.8),
                                       (1, 3, 1.0), (1, 2, 0.75)])
@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_vcycle_leaves_checkerboard_to_the_smoother(order, s, c, bc):
    # (-1)^(i+j+k) is an eigenvector of the homogeneous Dirichlet and of the
    # periodic operator (even sizes) with the top eigenvalue -4 sum 1/h^2, and
    # its 8-child means vanish, so the coarse correction is zero and one
    # V-cycle (f = 0) scales it by the smoother alone: tau = c tau_max puts it
    # at x = 1 - 2c of the stability polynomial, R = P_s(x) (RKL1) or
    # a_s + b_s P_s(x) (RKL2), applied n_pre + n_post times.  For RKL2 with
    # even s and c = 1 that factor is exactly 1.
    shape = (8, 12, 16)
    h = O.spacing(shape, (0, 0, 0), (1.0, 1.5, 2.4))
    k, j, i = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    u0 = np.where((i + j + k) % 2 == 0, 1.0, -1.0)
    opts = O.Options(rkl_order=order, s_smooth=s, tau_frac=c)
    out = O.vcycle(u0.copy(), np.zeros(shape), h, bc, None, 3, opts)
    x = 1.0 - 2.0 * c
    if order == 1:
        R = P(s, x)
    else:
        b = (s * s + s - 2.0) / (2.0 * s * (s + 1.0)) if s > 2 else 1.0 / 3.0
        R = (1.0 - b) + b * P(s, x)
    np.testing.assert_allclose(out, R ** (opts.n_pre + opts.n_post) * u0, atol=1e-12, rtol=0)
    if order == 2 and s % 2 == 0 and c == 1.0:
        np.testing.assert_allclose(out, u0, atol=1e-12, rtol=0)


# ---------------------------------------------------------------------------
# Behaviour printed in the paper
# ---------------------------------------------------------------------------

def test_gsrb_vcycle_reduces_residual_about_tenfold():
    # Sec. 4.1: GS-RB smoothing, RKL coarse solve, N_pre = 2, N_post = 1:
    # about one order of magnitude per V-cycle.
    g = GOLDEN["vcycle_residual_reduction"]["value"]
    p = W.smooth_sphere(32)
    opts = O.Options(smoother="gsrb", n_pre=GOLDEN["n_pre"]["value"], n_post=GOLDEN["n_post"]["value"])
    phi, info = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, opts=opts, cycles=5)
    h = info.history
    factors = [h[i] / h[i + 1] for i in range(len(h) - 1)]
    assert all(g / 2.0 <= f <= g * 5.0 for f in factors), factors


def test_second_order_accuracy_smooth_model_problem():
    # Sec. 4.1, Fig. error: error of the potential scales as h^2.
    errs = []
    for n in (32, 64):
        p = W.smooth_sphere(n)
        phi, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, tol=1e-12,
                         opts=O.Options(rkl_order=1, s_smooth=2, tau_frac=0.75))
        errs.append(O.l2norm(phi - p.exact) / O.l2norm(p.exact))
    order = math.log2(errs[0] / errs[1])
    assert abs(order - GOLDEN["accuracy_order"]["value"]) < 0.35, errs


# ---------------------------------------------------------------------------
# Spectral toolkit and schedules (App. A.4, A.5)
# ---------------------------------------------------------------------------

def test_legendre_recursion():
    x = np.linspace(-1, 1, 101)
    for s in (0, 1, 2, 7, 24, 56):
        np.testing.assert_allclose(O.legendre(s, x), P(s, x), atol=1e-12)


def test_1d_model_spectrum():
    # Eqs. M_matrix, eigenvalue_M, eigenvalue_RKL: eigenvalues of the (N-1)x(N-1)
    # matrix, mapped through P_s(1 + w1 tau_max lambda), give P_s(cos k pi/N).
    N, dx = 24, 0.1
    M = (np.diag(-2 * np.ones(N - 1)) + np.diag(np.ones(N - 2), 1) + np.diag(np.ones(N - 2), -1)) / dx ** 2
    lam = np.sort(np.linalg.eigvalsh(M))[::-1]            # k = 1 first
    k = np.arange(1, N)
    np.testing.assert_allclose(lam, -4 / dx ** 2 * np.sin(k * np.pi / (2 * N)) ** 2, rtol=1e-10)
    for s in (3, 8, 20):
        w1 = 2.0 / (s * s + s)
        tau_max = (dx ** 2 / 2.0) * (s * s + s) / 2.0
        lam_rkl = P(s, 1 + w1 * tau_max * lam)
        np.testing.assert_allclose(lam_rkl, [O.rkl_eigenvalue(s, kk, N) for kk in k], atol=1e-11)
        # Eq. RKL_symmetry
        np.testing.assert_allclose(np.abs(lam_rkl), np.abs(lam_rkl[::-1]), atol=1e-11)
        rho_full = np.max(np.abs(lam_rkl))
        assert abs(O.spectral_radius(s, N, kmax=N // 2) - rho_full) < 1e-12


def test_bessel_zero_and_sk_opt():
    z = GOLDEN["bessel_j0_first_zero"]["value"]
    assert abs(sps.j0(z)) < 1e-4
    assert O.BESSEL_J0_FIRST_ZERO == z
    # Eq. sk_optimal puts s near the first zero of P_s(cos k pi / N)
    for N in (64, 128):
        for k in (1, 2, 5, 12, 32):
            if k > N // 2:
                continue
            assert abs(O.s_k_opt(k, N) - O.first_zero_s(k, N)) <= 1
    assert O.s_k_opt(1, 32) == 24 and O.s_k_opt(1, 16) == 12


def test_bessel_approximation_error_within_one_percent():
    # Fig. approximation: |lambda - lambda_apprx| <~ 1% up to k = 32 ("<~":
    # the largest gap, at s = 1, is 1.16%, so the bound is read as 1.5%).
    tol = GOLDEN["bessel_approx_max_abs_error"]["value"]
    N = 128
    for k in (1, 5, 32):
        th = k * np.pi / N
        s = np.arange(1, N + 1)
        exact = np.array([float(O.rkl_eigenvalue(int(si), k, N)) for si in s])
        approx = math.sqrt(th / math.sin(th)) * sps.j0((s + 0.5) * th)
        assert np.max(np.abs(exact - approx)) <= 1.5 * tol
        assert np.max(np.abs(exact - approx)[s >= 3]) <= tol


def test_accelerated_schedule_skips_repeats():
    N = 16
    sched = O.accelerated_schedule(N, 12)
    brute = []
    last = 0
    for k in range(N // 2, 0, -1):
        s = int(math.floor(2.4048 * N / (math.pi * k) - 0.5 + 0.5))
        if s != last:
            brute.append(s)
            last = s
    assert sched[:len(brute)] == brute
    assert all(s == brute[-1] for s in sched[len(brute):])


def test_global_s_opt_minimises_spectral_radius():
    N = 64
    s_opt = O.s_opt_global(N)
    s0 = O.first_zero_s(1, N)
    radii = {s: max(abs(P(s, math.cos(k * math.pi / N))) for k in range(1, 7)) for s in range(s0, N + 1)}
    assert radii[s_opt] == min(radii.values())


def test_level_count_rule():
    assert O.level_count((256, 256, 256)) == 8
    assert O.level_count((96, 96, 96)) == 5
    assert O.level_count((32, 32, 32)) == 5
    assert O.level_count((8, 4, 6)) == 1
    assert O.level_count((12, 12, 12)) == 2


def test_sor_omega_reduces_to_textbook_cube():
    n, h = 32, 1.0 / 32
    om = O.sor_omega((n, n, n), (h, h, h))
    rj = math.cos(math.pi / n)
    assert abs(om - 2.0 / (1.0 + math.sqrt(1.0 - rj * rj))) < 1e-14


def _colour(shape):
    K, J, I = np.meshgrid(*(np.arange(n) for n in shape), indexing="ij")
    return (I + J + K) % 2


def _sweep_matrix(shape, h, bc, omega):
    """Iteration matrix of one oracle GS-RB sweep (rhs = 0, homogeneous ghosts)."""
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        M[:, i] = O.gs_rb_sweep(e.reshape(shape), np.zeros(shape), h, bc, None, omega).ravel()
    return M


@pytest.mark.parametrize("shape,bc", [((4, 4, 6), (0, 0, 0)), ((4, 6, 4), (1, 0, 1)),
                                      ((6, 4, 4), (0, 1, 1))])
def test_gsrb_sweep_radius_follows_young(shape, bc):
    # The 7-point graph is bipartite under the red-black colouring (periodic
    # extents even), so the ordering is consistent (Young): one Gauss-Seidel
    # sweep has spectral radius rho(J)^2, and above the optimal omega every
    # SOR eigenvalue has modulus omega - 1.  J from the Kronecker matrix.
    h = (0.3, 0.5, 0.4)
    A = kron_operator(shape, h, bc)
    J = np.eye(A.shape[0]) - A / np.diag(A)[:, None]
    rj = max(abs(np.linalg.eigvals(J)))
    assert 0.5 < rj < 1.0
    rgs = max(abs(np.linalg.eigvals(_sweep_matrix(shape, h, bc, 1.0))))
    assert abs(rgs - rj ** 2) < 1e-10
    w_opt = 2.0 / (1.0 + math.sqrt(1.0 - rj ** 2))
    w = 0.5 * (w_opt + 2.0)
    mods = abs(np.linalg.eigvals(_sweep_matrix(shape, h, bc, w)))
    np.testing.assert_allclose(mods, w - 1.0, atol=1e-6, rtol=0)


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1)])
def test_gsrb_half_sweeps_solve_their_rows(bc):
    # omega = 1: the first half-sweep makes the residual of every even cell
    # zero with the odd cells as they came in; the second makes every odd
    # cell's residual zero.  Residuals through the Kronecker matrix and the
    # 2 g / h^2 face vector, with Dirichlet data on the walls.
    shape, h = (6, 4, 8), (0.3, 0.2, 0.25)
    faces = W.random_faces(shape, 11)
    u, f = W.random_field(shape, 12), W.random_field(shape, 13)
    out = O.gs_rb_sweep(u, f, h, bc, faces, 1.0)
    A = kron_operator(shape, h, bc)
    b = np.zeros(shape)
    if bc[0] == 0:
        b[:, :, 0] += 2 * faces[0] / h[0] ** 2
        b[:, :, -1] += 2 * faces[1] / h[0] ** 2
    if bc[1] == 0:
        b[:, 0, :] += 2 * faces[2] / h[1] ** 2
        b[:, -1, :] += 2 * faces[3] / h[1] ** 2
    if bc[2] == 0:
        b[0, :, :] += 2 * faces[4] / h[2] ** 2
        b[-1, :, :] += 2 * faces[5] / h[2] ** 2
    res = lambda v: (A @ v.ravel()).reshape(shape) + b - f
    odd = _colour(shape) == 1
    half = np.where(odd, u, out)
    scale = np.abs(f).max() + np.abs(b).max()
    assert np.abs(res(half)[~odd]).max() < 1e-12 * scale
    assert np.abs(res(out)[odd]).max() < 1e-12 * scale
    assert np.abs(res(out)[~odd]).max() > 1e-3 * scale


@pytest.mark.parametrize("omega", [1.0, 0.0])
def test_single_level_gsrb_solve_reaches_direct_solution(omega):
    # levels = 1 with the GS-RB smoother: Gauss-Seidel (omega = 1) or App. B's
    # SOR (omega = 0 picks its omega) converge to the Kronecker direct solution.
    shape, lo, hi, bc = (8, 6, 10), (0, 0, 0), (1.0, 0.6, 0.8), (0, 1, 0)
    rho = W.random_field(shape, 21)
    faces = W.random_faces(shape, 22)
    opts = O.Options(smoother="gsrb", omega=omega, max_cycles=2000)
    phi, info = O.solve(rho, lo, hi, bc, faces, 1.0, tol=1e-11, levels=1, opts=opts)
    ref = O.dense_solve(rho, lo, hi, bc, faces, 1.0)
    assert info.rel_residual <= 1e-11
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-8
    if omega == 0.0:
        gs = O.solve(rho, lo, hi, bc, faces, 1.0, tol=1e-11, levels=1,
                     opts=O.Options(smoother="gsrb", max_cycles=2000))[1]
        assert info.cycles < gs.cycles / 2


# ---------------------------------------------------------------------------
# Fourth-order acceleration (Sec. 3)
# ---------------------------------------------------------------------------

def _centres(shape, lo, hi):
    nz, ny, nx = shape
    ax = [lo[d] + (np.arange(n) + 0.5) * (hi[d] - lo[d]) / n for d, n in enumerate((nx, ny, nz))]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X, Y, Z


def _faces_of(fn, shape, lo, hi):
    """Face-centre values of fn(x, y, z) in the face layout of the oracle."""
    X, Y, Z = _centres(shape, lo, hi)
    return [fn(np.full_like(X[:, :, 0], lo[0]), Y[:, :, 0], Z[:, :, 0]),
            fn(np.full_like(X[:, :, 0], hi[0]), Y[:, :, 0], Z[:, :, 0]),
            fn(X[:, 0, :], np.full_like(Y[:, 0, :], lo[1]), Z[:, 0, :]),
            fn(X[:, 0, :], np.full_like(Y[:, 0, :], hi[1]), Z[:, 0, :]),
            fn(X[0, :, :], Y[0, :, :], np.full_like(Z[0, :, :], lo[2])),
            fn(X[0, :, :], Y[0, :, :], np.full_like(Z[0, :, :], hi[2]))]


def test_gravity_exact_for_quartics_away_from_walls():
    # the five-point central difference is exact for polynomials of degree 4
    shape, lo, hi = (9, 8, 10), (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)
    X, Y, Z = _centres(shape, lo, hi)
    phi = 0.7 * X ** 4 - X ** 3 + 2 * Y ** 4 + Y * Z ** 2 - 3 * Z ** 4 + X * Y * Z + 0.5
    gx = -(2.8 * X ** 3 - 3 * X ** 2 + Y * Z)
    gy = -(8 * Y ** 3 + Z ** 2 + X * Z)
    gz = -(2 * Y * Z - 12 * Z ** 3 + X * Y)
    g = O.gravity(phi, O.spacing(shape, lo, hi), (0, 0, 0), None)
    inner = (slice(2, -2),) * 3
    for d, ref in enumerate((gx, gy, gz)):
        np.testing.assert_allclose(g[d][inner], ref[inner], rtol=0, atol=1e-10 * np.abs(ref).max())


def test_gravity_of_linear_field_exact_at_the_walls():
    # with the face values of a linear field the reflected ghosts continue it
    shape, lo, hi = (6, 7, 5), (-1.0, 0.0, 0.5), (1.0, 0.7, 1.3)
    fn = lambda x, y, z: 0.3 - 1.5 * x + 2.5 * y + 0.75 * z
    X, Y, Z = _centres(shape, lo, hi)
    g = O.gravity(fn(X, Y, Z), O.spacing(shape, lo, hi), (0, 0, 0), _faces_of(fn, shape, lo, hi))
    for d, v in enumerate((1.5, -2.5, -0.75)):
        np.testing.assert_allclose(g[d], v, rtol=0, atol=1e-12)


def test_gravity_periodic_sinusoid_closed_form():
    # d/dx sin(kx) by the stencil: cos(kx) (8 sin(kh) - sin(2kh)) / (6h)
    shape, lo, hi = (6, 4, 16), (0.0, 0.0, 0.0), (2.0, 1.0, 1.0)
    X, Y, Z = _centres(shape, lo, hi)
    k, h = 2 * np.pi * 3 / 2.0, 2.0 / 16
    g = O.gravity(np.sin(k * X + 0.3), (h, 0.25, 1.0 / 6), (1, 1, 1))
    np.testing.assert_allclose(g[0], -np.cos(k * X + 0.3) * (8 * np.sin(k * h) - np.sin(2 * k * h)) / (6 * h),
                               rtol=0, atol=1e-12)
    np.testing.assert_allclose(g[1], 0.0, atol=1e-12)
    np.testing.assert_allclose(g[2], 0.0, atol=1e-12)


def test_gravity_is_fourth_order_and_second_order_after_the_solve():
    # smooth periodic field: error falls 16x per halving of h; Sec. 4.1 model
    # problem: g of the discrete solution against Eq. acceleration_3D falls
    # about 4x (the potential's h^2 error dominates, Fig. error_map)
    errs = []
    for n in (16, 32):
        X, Y, Z = _centres((n, n, n), (0, 0, 0), (1, 1, 1))
        phi = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * Y)
        g = O.gravity(phi, (1.0 / n,) * 3, (1, 1, 1))
        errs.append(np.abs(g[0] + 2 * np.pi * np.cos(2 * np.pi * X) * np.cos(2 * np.pi * Y)).max())
    assert 14.0 < errs[0] / errs[1] < 18.0
    errs = []
    for n in (32, 64):
        p = W.smooth_sphere(n)
        phi, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, tol=1e-12)
        X, Y, Z = _centres(p.shape, p.lo, p.hi)
        r = np.sqrt(X * X + Y * Y + Z * Z)
        r0, rho0 = 0.25, 1.0
        M = 32 * np.pi * rho0 * r0 ** 3 / 105
        gr = np.where(r <= r0, -4 * np.pi * rho0 * (r / 3 - 0.4 * r ** 3 / r0 ** 2 + r ** 5 / (7 * r0 ** 4)),
                      -M / r ** 2)
        g = O.gravity(phi, O.spacing(p.shape, p.lo, p.hi), p.bc, p.faces)
        err = np.sqrt(sum((g[d] - gr * c / r) ** 2 for d, c in enumerate((X, Y, Z))))
        errs.append(O.l2norm(err) / O.l2norm(np.abs(gr)))
    assert 3.3 < errs[0] / errs[1] < 5.0


# ---------------------------------------------------------------------------
# Adjoint
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 1, 1)])
def test_adjoint_matches_finite_differences(bc):
    shape, lo, hi = (8, 8, 8), (0, 0, 0), (1, 1, 1)
    rho = W.random_field(shape, 41)
    faces = None if bc == (1, 1, 1) else W.random_faces(shape, 42)
    w = W.loss_weights(shape, 43)
    g, _ = O.adjoint(w, lo, hi, bc, four_pi_G=2.5, tol=1e-13)
    eps = 1e-3
    for cell in W.sample_cells(shape, 6, 44):
        rp, rm = rho.copy(), rho.copy()
        rp[cell] += eps
        rm[cell] -= eps
        Lp = np.sum(w * O.dense_solve(rp, lo, hi, bc, faces, 2.5))
        Lm = np.sum(w * O.dense_solve(rm, lo, hi, bc, faces, 2.5))
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g[cell]) <= 1e-8 * max(1.0, abs(fd))
