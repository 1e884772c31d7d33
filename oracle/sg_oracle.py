"""Plain FP64 CPU oracle of the RKL-multigrid Poisson solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import or call this
module: it is used by ``tests/``, by ``__graft_entry__.smoke()`` and by the CPU
baseline leg of ``bench.py``.  It shares no code with the CUDA path.

The oracle is written for a reader who checks it against the paper by eye
(Mandal, Mukherjee & Mignone, "A self-gravity module for the PLUTO code"):
every step is the paper's formula applied to whole numpy arrays, in FP64, with
no blocking, fusion or reordering.  Arrays are C order ``[nz][ny][nx]`` (x
fastest); physical axis d (0 = x, 1 = y, 2 = z) is numpy axis ``2 - d``.

Passages followed
-----------------
* Sec. 2.1, V-cycle list                       -> ``vcycle``, ``solve``
* Sec. 2.2.1, Eq. discrete_laplace_3D          -> ``laplacian``
* Sec. 2.1, Eq. residual                       -> ``residual``
* Sec. 2.2.2, Eqs. restriction_equation_3D /
  restriction_example_3D                       -> ``restrict``
* Sec. 2.2.3, Eq. prolongation_example_3D      -> ``prolong``
* Sec. 2.3, Eqs. solution_ghost, error_ghost,
  periodic, source_modification                -> ``pad_ghosts``, ``source``
* App. A, Eqs. RKL stability poly, RKL_intermediate_source, tau_max
                                               -> ``rkl1_coefficients``, ``rkl_superstep``
* RKL2 (the a_s + b_s P_s family of App. A with Meyer et al. 2014's
  coefficients)                                -> ``rkl2_coefficients``
* App. A.4, Eqs. eigenvalue_RKL, spectral_rad_RKL, sopt_theory
                                               -> ``spectral_radius``, ``s_opt_global``
* App. A.5, Eq. sk_optimal and the accelerated schedule with skipped repeats
                                               -> ``s_k_opt``, ``accelerated_schedule``
* Sec. 3, Eq. 4thorder_acceleration            -> ``gravity``
* Sec. 4.1, L2 norm with cell volumes          -> ``l2norm``
* Sec. 4.1, level-count rule                   -> ``level_count``
* Sec. 2.1-2.3, the discrete solution the V-cycle converges to (Kronecker
  sum of 1D second differences, DST-II / DFT diagonalisation)
                                               -> ``direct_solve``
* App. B, SOR omega and GS-RB (Sec. 2.2.4)      -> ``gs_rb_sweep``, ``sor_omega``

Readings where the paper is silent or ambiguous (all listed in the design
notes): cell-centred coordinates x_i = lo + (i + 1/2) h; the V-cycle increments
the level once per pass; prolongation fills coarse ghosts with the level's
boundary rule; the coarsest-level and single-level solver uses
tau = cos^2(pi / 2N) tau_max unless told otherwise; in the Legendre-zero schedule
N is the level's largest extent and the bracket [N/k] is plain division;
periodic potentials are returned with zero mean; the second ghost layer of the
fourth-order gradient reflects through the face value like the first.

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, FFT/DST direct solves, a dense direct solve, and Legendre identities.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
PERIODIC = 1
BESSEL_J0_FIRST_ZERO = 2.4048          # App. A.5, first zero of J0


# ---------------------------------------------------------------------------
# Grid helpers
# ---------------------------------------------------------------------------

def spacing(shape, lo, hi):
    """(hx, hy, hz) of a [nz][ny][nx] grid on the box [lo, hi]."""
    nz, ny, nx = shape
    return ((hi[0] - lo[0]) / nx, (hi[1] - lo[1]) / ny, (hi[2] - lo[2]) / nz)


def level_count(shape):
    """Largest L such that N / 2^(L-1) is even on every axis (Sec. 4.1)."""
    L = 1
    while all((n % (2 ** L) == 0) and (n // 2 ** L) % 2 == 0 for n in shape):
        L += 1
    return L


def all_periodic(bc):
    return all(b == PERIODIC for b in bc)


def _face_slices(ax, idx, full):
    s = [slice(None) if full else slice(1, -1)] * 3
    s[ax] = idx
    return tuple(s)


def pad_ghosts(u, bc, faces=None):
    """u with one ghost layer on every side.

    Dirichlet with ``faces`` (finest level): Eq. solution_ghost,
        ghost = 2 * phi_face - phi_active   (face ghosts only; the 7-point
        stencil never reads edges or corners).
    Dirichlet without faces (error equation, levels l > 0, or a homogeneous
    solve): Eq. error_ghost, ghost = -active.
    Periodic: Eq. periodic, ghost = the active cell on the opposite side.
    Without faces the rules are applied axis after axis over the whole padded
    extent, so edge and corner ghosts (read by the prolongation stencil) are
    the repeated odd reflection / periodic image.
    """
    nz, ny, nx = u.shape
    p = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.float64)
    p[1:-1, 1:-1, 1:-1] = u
    full = faces is None
    for d in range(3):
        ax = 2 - d
        lo_g, lo_a = _face_slices(ax, 0, full), _face_slices(ax, 1, full)
        hi_g, hi_a = _face_slices(ax, -1, full), _face_slices(ax, -2, full)
        if bc[d] == PERIODIC:
            p[lo_g] = p[hi_a]
            p[hi_g] = p[lo_a]
        elif faces is not None:
            p[lo_g] = 2.0 * faces[2 * d] - p[lo_a]
            p[hi_g] = 2.0 * faces[2 * d + 1] - p[hi_a]
        else:
            p[lo_g] = -p[lo_a]
            p[hi_g] = -p[hi_a]
    return p


def laplacian(u, h, bc, faces=None):
    """Seven-point Laplacian, Eq. discrete_laplace_3D, with the ghost rules."""
    hx, hy, hz = h
    p = pad_ghosts(u, bc, faces)
    c = p[1:-1, 1:-1, 1:-1]
    return ((p[1:-1, 1:-1, :-2] - 2.0 * c + p[1:-1, 1:-1, 2:]) / (hx * hx)
            + (p[1:-1, :-2, 1:-1] - 2.0 * c + p[1:-1, 2:, 1:-1]) / (hy * hy)
            + (p[:-2, 1:-1, 1:-1] - 2.0 * c + p[2:, 1:-1, 1:-1]) / (hz * hz))


def gravity(phi, h, bc, faces=None):
    """g = -grad phi by the fourth-order central difference of Sec. 3, Eq.
    4thorder_acceleration, along each axis d:

        g_d = -(4/3) (phi_{+1} - phi_{-1}) / (2 h_d) + (1/3) (phi_{+2} - phi_{-2}) / (4 h_d).

    The stencil reaches two cells past a wall; the paper fills only the first
    ghost (Eq. solution_ghost).  Both ghost layers here continue that rule as a
    reflection through the face value: the ghost m + 1 cells beyond the wall is
    2 phi_face - (the m-th cell from the wall), m = 0, 1 (zero face values when
    ``faces`` is None).  Periodic axes wrap (Eq. periodic).
    Returns [3][nz][ny][nx], the x component first."""
    phi = np.asarray(phi, dtype=np.float64)
    out = np.empty((3,) + phi.shape)
    for d in range(3):
        ax = 2 - d
        n = phi.shape[ax]
        if bc[d] == PERIODIC:
            p = np.take(phi, np.arange(-2, n + 2) % n, axis=ax)
        else:
            lo = np.expand_dims(faces[2 * d], ax) if faces is not None else 0.0
            hi = np.expand_dims(faces[2 * d + 1], ax) if faces is not None else 0.0
            below = 2.0 * lo - np.take(phi, [1, 0], axis=ax)          # ghosts -2, -1
            above = 2.0 * hi - np.take(phi, [n - 1, n - 2], axis=ax)  # ghosts n, n + 1
            p = np.concatenate([below, phi, above], axis=ax)

        def at(off):                      # phi_{i + off} for every cell i along the axis
            return np.take(p, np.arange(2 + off, n + 2 + off), axis=ax)

        hd = h[d]
        out[d] = (-(4.0 / 3.0) * (at(1) - at(-1)) / (2.0 * hd)
                  + (1.0 / 3.0) * (at(2) - at(-2)) / (4.0 * hd))
    return out


def residual(u, rhs, h, bc, faces=None):
    """Eq. residual: r = L u - f (the paper's sign)."""
    return laplacian(u, h, bc, faces) - rhs


def l2norm(F, h=(1.0, 1.0, 1.0)):
    """Sec. 4.1: [sum F^2 dV / V]^(1/2); on a uniform grid dV / V = 1 / n."""
    dV = h[0] * h[1] * h[2]
    V = dV * F.size
    return math.sqrt(float(np.sum(F * F) * dV / V))


def source(rho, four_pi_G, bc):
    """f = 4 pi G rho; with periodic boundaries rho -> rho - mean(rho) first
    (Eq. source_modification)."""
    rho = np.asarray(rho, dtype=np.float64)
    if all_periodic(bc):
        rho = rho - rho.mean()
    return four_pi_G * rho


# ---------------------------------------------------------------------------
# Transfer operators
# ---------------------------------------------------------------------------

def restrict(r):
    """Eq. restriction_example_3D: the coarse value is the mean of its 8 children."""
    a = r[0::2, 0::2, 0::2]
    b = r[0::2, 0::2, 1::2]
    c = r[0::2, 1::2, 0::2]
    d = r[0::2, 1::2, 1::2]
    e = r[1::2, 0::2, 0::2]
    f = r[1::2, 0::2, 1::2]
    g = r[1::2, 1::2, 0::2]
    hh = r[1::2, 1::2, 1::2]
    return (a + b + c + d + e + f + g + hh) / 8.0


def prolong(e, bc):
    """Eq. prolongation_example_3D: a = (27A + 9B + 9D + 9E + 3C + 3F + 3H + G)/64.

    A is the coarse parent, B/D/E the three face neighbours towards the fine
    cell, C/F/H the three edge neighbours and G the corner neighbour.  Coarse
    ghosts follow the level's boundary rule (-e for Dirichlet, copy for
    periodic), so the stencil is applied uniformly up to the wall.
    """
    nz, ny, nx = e.shape
    p = pad_ghosts(e, bc, None)
    out = np.empty((2 * nz, 2 * ny, 2 * nx), dtype=np.float64)
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                # neighbour offset towards the fine cell on each axis
                sz, sy, sx = (-1 if oz == 0 else 1), (-1 if oy == 0 else 1), (-1 if ox == 0 else 1)
                acc = np.zeros((nz, ny, nx), dtype=np.float64)
                for az in (0, 1):
                    for ay in (0, 1):
                        for ax in (0, 1):
                            w = (3 if az == 0 else 1) * (3 if ay == 0 else 1) * (3 if ax == 0 else 1)
                            dz, dy, dx = az * sz, ay * sy, ax * sx
                            acc = acc + w * p[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
                out[oz::2, oy::2, ox::2] = acc / 64.0
    return out


# ---------------------------------------------------------------------------
# RKL super-time-stepping (App. A)
# ---------------------------------------------------------------------------

@dataclass
class RKLCoefficients:
    order: int
    s: int
    w1: float
    mu: np.ndarray        # index j = 0..s (0 unused)
    nu: np.ndarray
    mu_t: np.ndarray
    gamma_t: np.ndarray   # zero for RKL1
    a: np.ndarray         # a_j (zero for RKL1)
    b: np.ndarray         # b_j (one for RKL1)
    tau_max_over_dtpar: float


def rkl1_coefficients(s):
    """First-order RKL: R_s = P_s(1 + w1 z), w1 = 2/(s^2+s); mu_j = (2j-1)/j,
    nu_j = (1-j)/j, mu~_j = mu_j w1; tau_max = dt_par (s^2+s)/2 (App. A)."""
    if s < 1:
        raise ValueError("RKL1 needs s >= 1")
    w1 = 2.0 / (s * s + s)
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mu_t = np.zeros(s + 1)
    for j in range(1, s + 1):
        mu[j] = (2.0 * j - 1.0) / j
        nu[j] = (1.0 - j) / j
        mu_t[j] = mu[j] * w1
    return RKLCoefficients(1, s, w1, mu, nu, mu_t, np.zeros(s + 1),
                           np.zeros(s + 1), np.ones(s + 1), (s * s + s) / 2.0)


def rkl2_coefficients(s):
    """Second-order RKL: R_s = a_s + b_s P_s(1 + w1 z) with w0 = 1 (App. A's
    general form), using Meyer et al. (2014)'s choice b_j = (j^2+j-2)/(2j(j+1)),
    b_0 = b_1 = b_2 = 1/3, a_j = 1 - b_j, w1 = 4/(s^2+s-2); stage weights
    mu_j = (2j-1)/j b_j/b_{j-1}, nu_j = -(j-1)/j b_j/b_{j-2}, mu~_1 = b_1 w1,
    mu~_j = mu_j w1, gamma~_j = -a_{j-1} mu~_j; tau_max = dt_par (s^2+s-2)/4."""
    if s < 2:
        raise ValueError("RKL2 needs s >= 2")
    w1 = 4.0 / (s * s + s - 2.0)
    b = np.zeros(s + 1)
    for j in range(s + 1):
        b[j] = 1.0 / 3.0 if j <= 2 else (j * j + j - 2.0) / (2.0 * j * (j + 1.0))
    a = 1.0 - b
    mu = np.zeros(s + 1)
    nu = np.zeros(s + 1)
    mu_t = np.zeros(s + 1)
    gamma_t = np.zeros(s + 1)
    mu_t[1] = b[1] * w1
    for j in range(2, s + 1):
        mu[j] = (2.0 * j - 1.0) / j * b[j] / b[j - 1]
        nu[j] = -(j - 1.0) / j * b[j] / b[j - 2]
        mu_t[j] = mu[j] * w1
        gamma_t[j] = -a[j - 1] * mu_t[j]
    return RKLCoefficients(2, s, w1, mu, nu, mu_t, gamma_t, a, b, (s * s + s - 2.0) / 4.0)


def rkl_coefficients(order, s):
    return rkl1_coefficients(s) if order == 1 else rkl2_coefficients(s)


def lambda_max(h):
    """Largest |eigenvalue| of the cell-centred 7-point Laplacian: 4 sum_d 1/h_d^2."""
    return 4.0 * sum(1.0 / (hd * hd) for hd in h)


def tau_step(order, s, h, tau_frac):
    """tau = tau_frac * tau_max, tau_max = dt_par * (s^2+s)/2 (RKL1) or
    dt_par * (s^2+s-2)/4 (RKL2), dt_par = 2 / |lambda_max| (Eq. tau_max)."""
    dt_par = 2.0 / lambda_max(h)
    return tau_frac * dt_par * rkl_coefficients(order, s).tau_max_over_dtpar


def rkl_superstep(u, rhs, h, bc, faces, order, s, tau_frac):
    """One s-stage RKL super-step of du/dt = M u - f (Eq. RKL_intermediate_source).

    RKL1:  Y1 = Y0 + mu~_1 tau (M Y0 - f)
           Yj = mu_j Y_{j-1} + nu_j Y_{j-2} + mu~_j tau (M Y_{j-1} - f)
    RKL2:  Y1 = Y0 + mu~_1 tau (M Y0 - f)
           Yj = mu_j Y_{j-1} + nu_j Y_{j-2} + (1 - mu_j - nu_j) Y0
                + mu~_j tau (M Y_{j-1} - f) + gamma~_j tau (M Y0 - f)
    M is the Laplacian with the level's ghost rule; returns Y_s.
    """
    co = rkl_coefficients(order, s)
    tau = tau_step(order, s, h, tau_frac)

    def M_minus_f(y):
        return laplacian(y, h, bc, faces) - rhs

    Y0 = u
    MY0 = M_minus_f(Y0)
    Yjm2 = Y0
    Yjm1 = Y0 + co.mu_t[1] * tau * MY0
    for j in range(2, s + 1):
        Yj = co.mu[j] * Yjm1 + co.nu[j] * Yjm2 + co.mu_t[j] * tau * M_minus_f(Yjm1)
        if order == 2:
            Yj = Yj + (1.0 - co.mu[j] - co.nu[j]) * Y0 + co.gamma_t[j] * tau * MY0
        Yjm2, Yjm1 = Yjm1, Yj
    return Yjm1


def rkl_scalar_stages(order, s, z):
    """The stage recursion on the scalar test equation y' = lambda y with
    z = tau lambda, Y0 = 1, f = 0; returns [Y_0 .. Y_s]."""
    co = rkl_coefficients(order, s)
    z = np.asarray(z, dtype=np.float64)
    Y = [np.ones_like(z)]
    Y.append(Y[0] + co.mu_t[1] * z * Y[0])
    for j in range(2, s + 1):
        Yj = co.mu[j] * Y[j - 1] + co.nu[j] * Y[j - 2] + co.mu_t[j] * z * Y[j - 1]
        if order == 2:
            Yj = Yj + (1.0 - co.mu[j] - co.nu[j]) * Y[0] + co.gamma_t[j] * z * Y[0]
        Y.append(Yj)
    return Y


# ---------------------------------------------------------------------------
# Spectral toolkit and s schedules (App. A.4 / A.5)
# ---------------------------------------------------------------------------

def legendre(s, x):
    """P_s(x) by the three-term recursion, Eq. LP_recursion."""
    x = np.asarray(x, dtype=np.float64)
    if s == 0:
        return np.ones_like(x)
    p_prev, p = np.ones_like(x), x.copy()
    for j in range(2, s + 1):
        p_prev, p = p, (2.0 * j - 1.0) / j * x * p - (j - 1.0) / j * p_prev
    return p


def rkl_eigenvalue(s, k, N):
    """Eq. eigenvalue_RKL: lambda_k,RKL = P_s(cos(k pi / N)) at tau = tau_max."""
    return legendre(s, math.cos(k * math.pi / N))


def spectral_radius(s, N, kmax=6):
    """Eq. spectral_rad_RKL with k restricted to 1..kmax (App. A.4, step 1)."""
    ks = range(1, min(kmax, max(1, N // 2)) + 1)
    return max(abs(float(rkl_eigenvalue(s, k, N))) for k in ks)


def m_eff(s, N, d=2.0, kmax=6):
    """Single-loop iterations s * m_RKL to gain d decades (Eqs. iteration, sopt_theory)."""
    rho = spectral_radius(s, N, kmax)
    if rho <= 0.0:
        return 0.0
    if rho >= 1.0:
        return math.inf
    return s * d / (-math.log10(rho))


def round_half_up(p):
    """'Round(p) ... the nearest integer' of Eq. sk_optimal; halves round up."""
    return int(math.floor(p + 0.5))


def s_k_opt(k, N):
    """Eq. sk_optimal: s_k = Round(2.4048 / pi * N / k - 1/2)."""
    return round_half_up(BESSEL_J0_FIRST_ZERO / math.pi * (N / k) - 0.5)


def first_zero_s(k, N):
    """Smallest s from the first zero of lambda_1,RKL(s) search (App. A.4)."""
    x = math.cos(k * math.pi / N)
    prev = 1.0
    s = 0
    while True:
        s += 1
        cur = float(legendre(s, x))
        if cur == 0.0 or (cur > 0) != (prev > 0):
            return s
        prev = cur


def s_opt_global(N, kmax=6):
    """App. A.4 two-step search: minimise the spectral radius over s between
    the first zero of lambda_1,RKL(s) and N."""
    s0 = first_zero_s(1, N)
    best_s, best_rho = s0, math.inf
    for s in range(s0, N + 1):
        rho = spectral_radius(s, N, kmax)
        if rho < best_rho:
            best_s, best_rho = s, rho
    return best_s


def accelerated_schedule(N, count):
    """The first `count` stage numbers of the accelerated RKL iteration
    (App. A.5, the variant that skips a k whose s repeats): k runs from N/2
    down to 1, then stays at s_1,opt."""
    out = []
    k = max(1, N // 2)
    s_old = 0
    while len(out) < count:
        s = s_k_opt(k, N)
        if not (s == s_old and k != 1):
            out.append(s)
            s_old = s
        k -= 1
        if k < 1:
            k = 1
    return out


def coarse_tau_frac(N):
    """tau / tau_max for the coarsest-level (and single-level) RKL solve:
    cos^2(pi / 2N) maps the cell-centred checkerboard mode to x = -cos(pi / N),
    where the paper's spectrum (App. A.4, Eq. eigenvalue_RKL) ends."""
    return math.cos(math.pi / (2.0 * N)) ** 2


# ---------------------------------------------------------------------------
# Solver options and the V-cycle (Sec. 2.1)
# ---------------------------------------------------------------------------

@dataclass
class Options:
    rkl_order: int = 2         # smoother order (1 or 2)
    s_smooth: int = 3          # stages per smoothing super-step
    tau_frac: float = 1.0      # smoother tau / tau_max
    n_pre: int = 2             # Sec. 4.1: N_pre = 2, N_post = 1
    n_post: int = 1
    inner_n_pre: int = -1      # smoothing counts on levels 1 .. L-2 (-1: n_pre / n_post)
    inner_n_post: int = -1
    coarse_tol: float = 1e-2   # coarsest-level relative residual target (0 = fixed count)
    coarse_max_ss: int = 64    # cap on coarsest-level super-steps
    coarse_tau_frac: float = 0.0   # 0 = coarse_tau_frac(N)
    max_cycles: int = 100
    single_s: int = 0          # levels == 1: fixed s (0 = accelerated schedule,
                               # -1 = App. A.4's global s_opt of the largest extent)
    single_tau_frac: float = 0.0   # levels == 1: 0 = coarse_tau_frac(N)
    smoother: str = "rkl"      # "rkl" (RKL super-steps) or "gsrb" (the paper's GS-RB)
    omega: float = 1.0         # GS-RB relaxation factor: 1 = Gauss-Seidel, (1, 2) = SOR;
                               # 0 = App. B's SOR omega of the level (``sor_omega``)


@dataclass
class SolveInfo:
    cycles: int = 0
    history: list = field(default_factory=list)
    rel_residual: float = math.inf
    r0: float = 0.0
    coarse_ss: list = field(default_factory=list)
    levels: int = 1


def level_shapes(shape, L):
    return [tuple(n // 2 ** l for n in shape) for l in range(L)]


def level_spacings(h, L):
    return [tuple(hd * 2 ** l for hd in h) for l in range(L)]


def coarse_solve(rhs, h, bc, faces, opts, u0=None, record=None):
    """Coarsest-grid solve of L u = rhs by the accelerated RKL1 iteration
    (App. A.5): super-steps with s from the Legendre-zero schedule until the
    residual falls below coarse_tol of its initial value, or coarse_max_ss
    super-steps have run (coarse_tol = 0 runs exactly coarse_max_ss)."""
    N = max(rhs.shape)
    c = opts.coarse_tau_frac if opts.coarse_tau_frac > 0 else coarse_tau_frac(N)
    u = np.zeros_like(rhs) if u0 is None else u0.copy()
    r_init = l2norm(residual(u, rhs, h, bc, faces))
    sched = accelerated_schedule(N, opts.coarse_max_ss)
    done = 0
    for s in sched:
        if opts.coarse_tol > 0.0:
            rn = l2norm(residual(u, rhs, h, bc, faces))
            if rn <= opts.coarse_tol * r_init:
                break
        u = rkl_superstep(u, rhs, h, bc, faces, 1, s, c)
        done += 1
    if record is not None:
        record.append(done)
    return u


def relax(u, rhs, h, bc, faces, opts, count):
    """`count` smoothing iterations: RKL super-steps of s_smooth stages, or
    GS-RB sweeps (Sec. 2.2.4) when opts.smoother == "gsrb"."""
    for _ in range(count):
        if opts.smoother == "gsrb":
            om = opts.omega if opts.omega > 0 else sor_omega(u.shape, h)
            u = gs_rb_sweep(u, rhs, h, bc, faces, om)
        else:
            u = rkl_superstep(u, rhs, h, bc, faces, opts.rkl_order, opts.s_smooth, opts.tau_frac)
    return u


def vcycle(phi, f, h, bc, faces, L, opts, record=None):
    """One correction-scheme V-cycle (Sec. 2.1), levels 0..L-1, one increment
    of l per pass (step 2), upstroke l = L-2..1 (step 3), then step 4 on l = 0.
    Levels 1..L-2 smooth opts.inner_n_pre / inner_n_post times when those are
    set (the paper uses N_pre / N_post on every level)."""
    hs = level_spacings(h, L)
    pre_in = opts.inner_n_pre if opts.inner_n_pre >= 0 else opts.n_pre
    post_in = opts.inner_n_post if opts.inner_n_post >= 0 else opts.n_post
    per = all_periodic(bc)
    u = [None] * L
    rhs = [None] * L
    u[0], rhs[0] = phi, f
    # step 1
    u[0] = relax(u[0], rhs[0], hs[0], bc, faces, opts, opts.n_pre)
    # step 2
    for l in range(1, L):
        r = residual(u[l - 1], rhs[l - 1], hs[l - 1], bc, faces if l - 1 == 0 else None)   # 2a
        fl = restrict(r)                                                                    # 2b
        if per:
            fl = fl - fl.mean()            # Sec. 2.3: coarse residual mean removed
        rhs[l] = -fl                       # relax L dphi = -f^l
        u[l] = np.zeros_like(fl)           # 2c
        if l < L - 1:
            u[l] = relax(u[l], rhs[l], hs[l], bc, None, opts, pre_in)                      # 2d-i
        else:
            u[l] = coarse_solve(rhs[l], hs[l], bc, None, opts, record=record)               # 2e
    # step 3
    for l in range(L - 2, 0, -1):
        u[l] = u[l] + prolong(u[l + 1], bc)                                                  # 3a
        u[l] = relax(u[l], rhs[l], hs[l], bc, None, opts, post_in)                          # 3b
    # step 4
    if L > 1:
        u[0] = u[0] + prolong(u[1], bc)                                                      # 4a
        u[0] = relax(u[0], rhs[0], hs[0], bc, faces, opts, opts.n_post)                     # 4b
    return u[0]


def solve(rho, lo, hi, bc, faces=None, four_pi_G=1.0, tol=1e-10, levels=0,
          opts=None, phi0=None, cycles=None, homogeneous=False):
    """Solve grad^2 phi = four_pi_G rho: repeat V-cycles while the relative L2
    residual ||L phi - f|| / ||L 0 - f|| is above tol (Sec. 2.1, Sec. 4.1).

    ``cycles`` forces an exact cycle count (tolerance ignored).  levels = 1 is
    the single-level solver: each "cycle" is one RKL1 super-step, with the
    accelerated schedule (opts.single_s = 0) or a fixed s, or, with
    opts.smoother == "gsrb", one red-black Gauss-Seidel / SOR sweep (App. B).
    Returns (phi, SolveInfo).
    """
    opts = opts or Options()
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    h = spacing(shape, lo, hi)
    L = levels if levels > 0 else level_count(shape)
    if homogeneous:
        faces = None
    f = source(rho, four_pi_G, bc)
    phi = np.zeros(shape) if phi0 is None else np.array(phi0, dtype=np.float64)
    info = SolveInfo(levels=L)
    info.r0 = l2norm(residual(np.zeros(shape), f, h, bc, faces))
    r0 = info.r0 if info.r0 > 0 else 1.0
    N = max(shape)
    single_c = opts.single_tau_frac if opts.single_tau_frac > 0 else coarse_tau_frac(N)
    single_rkl = L == 1 and opts.smoother != "gsrb"
    sched = accelerated_schedule(N, opts.max_cycles + 1) if single_rkl and opts.single_s == 0 else None
    limit = cycles if cycles is not None else opts.max_cycles
    m = 0
    while True:
        rel = l2norm(residual(phi, f, h, bc, faces)) / r0
        info.history.append(rel)
        info.rel_residual = rel
        if cycles is None and rel <= tol:
            break
        if m >= limit:
            break
        if L == 1 and not single_rkl:
            phi = relax(phi, f, h, bc, faces, opts, 1)
        elif L == 1:
            if opts.single_s > 0:
                s = opts.single_s
            elif opts.single_s < 0:
                s = s_opt_global(N)
            else:
                s = sched[m]
            phi = rkl_superstep(phi, f, h, bc, faces, 1, s, single_c)
        else:
            phi = vcycle(phi, f, h, bc, faces, L, opts, record=info.coarse_ss)
        m += 1
    info.cycles = m
    if all_periodic(bc):
        phi = phi - phi.mean()
    return phi, info


def adjoint(w, lo, hi, bc, four_pi_G=1.0, tol=1e-12, levels=0, opts=None, cycles=None):
    """dL/drho for L = sum(w * phi): phi is affine in rho with the symmetric
    operator L_h, so dL/drho = four_pi_G * L_h^{-1} w with homogeneous
    boundaries (periodic: w and the result projected to zero mean)."""
    w = np.asarray(w, dtype=np.float64)
    lam, info = solve(w, lo, hi, bc, None, 1.0, tol, levels, opts, cycles=cycles, homogeneous=True)
    g = four_pi_G * lam
    if all_periodic(bc):
        g = g - g.mean()
    return g, info


# ---------------------------------------------------------------------------
# Dense direct solve (small grids) and the paper's other relaxations
# ---------------------------------------------------------------------------

def dense_operator(shape, h, bc):
    """The matrix of the homogeneous-boundary Laplacian, column by column."""
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    e = np.zeros(n)
    for i in range(n):
        e[:] = 0.0
        e[i] = 1.0
        A[:, i] = laplacian(e.reshape(shape), h, bc, None).ravel()
    return A


def dense_solve(rho, lo, hi, bc, faces=None, four_pi_G=1.0):
    """Exact discrete solution by a dense direct solve (n <= 8^3 or so):
    L0 phi = f - L(0; faces); periodic: least-squares with zero mean."""
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    h = spacing(shape, lo, hi)
    f = source(rho, four_pi_G, bc)
    A = dense_operator(shape, h, bc)
    bvec = laplacian(np.zeros(shape), h, bc, faces).ravel()
    rhs = f.ravel() - bvec
    if all_periodic(bc):
        n = A.shape[0]
        Aa = np.vstack([A, np.ones((1, n))])
        ra = np.concatenate([rhs, [0.0]])
        x = np.linalg.lstsq(Aa, ra, rcond=None)[0]
    else:
        x = np.linalg.solve(A, rhs)
    return x.reshape(shape)


def _axis_eigenvalues(n, hd, periodic):
    """Eigenvalues of the 1D cell-centred second difference on n cells.
    Dirichlet (ghost = -active, Eqs. solution_ghost / error_ghost): modes
    sin(pi m (i + 1/2) / n), m = 1..n (the DST-II basis), lambda_m =
    -(4 / h^2) sin^2(pi m / (2 n)).  Periodic (Eq. periodic): modes
    exp(2 pi i m j / n), m = 0..n-1 (the DFT basis), lambda_m =
    -(4 / h^2) sin^2(pi m / n)."""
    m = np.arange(n) if periodic else np.arange(1, n + 1)
    arg = np.pi * m / n if periodic else np.pi * m / (2.0 * n)
    return -(4.0 / (hd * hd)) * np.sin(arg) ** 2


def direct_solve(rho, lo, hi, bc, faces=None, four_pi_G=1.0):
    """The exact discrete solution of L_h phi = f at any size, the result the
    V-cycle of Sec. 2.1 converges to (Eq. discrete_laplace_3D with the ghost
    rules of Sec. 2.3): L_h is a Kronecker sum of 1D second differences, each
    diagonalised by the DST-II (Dirichlet axis) or the DFT (periodic axis).

        b   = 2 phi_face / h_d^2 in the cells next to each Dirichlet face
              (the known part of the ghost 2 phi_face - phi_active)
        phi = V diag(1 / (lx + ly + lz)) V^-1 (f - b)

    With every axis periodic, f is mean-free (Eq. source_modification), the
    zero mode is dropped and phi has zero mean."""
    import scipy.fft as sfft
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    h = spacing(shape, lo, hi)
    f = source(rho, four_pi_G, bc)
    b = np.zeros(shape)
    if faces is not None:
        for d in range(3):
            if bc[d] == PERIODIC:
                continue
            ax = 2 - d
            lo_cells = [slice(None)] * 3
            hi_cells = [slice(None)] * 3
            lo_cells[ax], hi_cells[ax] = 0, -1
            b[tuple(lo_cells)] += 2.0 * np.asarray(faces[2 * d]) / (h[d] * h[d])
            b[tuple(hi_cells)] += 2.0 * np.asarray(faces[2 * d + 1]) / (h[d] * h[d])
    c = f - b
    lam = np.zeros(shape)
    for d in range(3):
        ax = 2 - d
        ev = _axis_eigenvalues(shape[ax], h[d], bc[d] == PERIODIC)
        sh = [1, 1, 1]
        sh[ax] = shape[ax]
        lam = lam + ev.reshape(sh)
    dirichlet_axes = [2 - d for d in range(3) if bc[d] != PERIODIC]
    periodic_axes = [2 - d for d in range(3) if bc[d] == PERIODIC]
    ck = c
    for ax in dirichlet_axes:
        ck = sfft.dst(ck, type=2, axis=ax)
    if periodic_axes:
        ck = sfft.fftn(ck, axes=periodic_axes)
    if all_periodic(bc):
        lam[0, 0, 0] = 1.0
        ck[0, 0, 0] = 0.0
    ck = ck / lam
    if periodic_axes:
        ck = np.real(sfft.ifftn(ck, axes=periodic_axes))
    for ax in dirichlet_axes:
        ck = sfft.idst(ck, type=2, axis=ax)
    phi = np.asarray(ck, dtype=np.float64)
    if all_periodic(bc):
        phi = phi - phi.mean()
    return phi


def operator_diagonal(shape, h, bc):
    """Diagonal of L_h: -2 sum 1/h^2, plus -1/h_d^2 on each Dirichlet wall the
    cell touches (its ghost is minus itself, Eqs. solution_ghost / error_ghost)."""
    nz, ny, nx = shape
    diag = np.full(shape, -2.0 * sum(1.0 / (hd * hd) for hd in h))
    for d in range(3):
        if bc[d] == PERIODIC:
            continue
        ax = 2 - d
        idx = [slice(None)] * 3
        for end in (0, -1):
            idx[ax] = end
            diag[tuple(idx)] -= 1.0 / (h[d] * h[d])
    return diag


def gs_rb_sweep(u, rhs, h, bc, faces=None, omega=1.0):
    """One red-black Gauss-Seidel (omega = 1) or SOR sweep (Sec. 2.2.4, App. B):
    cells with (i+j+k) even first, then odd; each update solves the cell's
    row of L u = rhs for its own value."""
    nz, ny, nx = u.shape
    diag = operator_diagonal(u.shape, h, bc)
    K, J, I = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = u.copy()
    for colour in (0, 1):
        mask = ((I + J + K) % 2) == colour
        r = laplacian(u, h, bc, faces) - rhs
        u[mask] = u[mask] - omega * r[mask] / diag[mask]
    return u


def sor_omega(shape, h):
    """App. B: omega = 2 / (1 + sqrt(1 - rho_J^2)) with the Jacobi spectral radius
    rho_J = 2 dt [cos(pi/J)/dx^2 + cos(pi/L)/dy^2 + cos(pi/K)/dz^2].  The printed
    dt = 2 [1/dx^2 + 1/dy^2 + 1/dz^2]^-1 would make rho_J > 1; it is read as
    dt = (2 [1/dx^2 + 1/dy^2 + 1/dz^2])^-1, which gives the textbook Jacobi radius
    (a weighted mean of the cosines)."""
    nz, ny, nx = shape
    hx, hy, hz = h
    dt = 1.0 / (2.0 * (1.0 / hx ** 2 + 1.0 / hy ** 2 + 1.0 / hz ** 2))
    rho_j = 2.0 * dt * (math.cos(math.pi / nx) / hx ** 2 + math.cos(math.pi / ny) / hy ** 2
                        + math.cos(math.pi / nz) / hz ** 2)
    return 2.0 / (1.0 + math.sqrt(1.0 - rho_j ** 2))
