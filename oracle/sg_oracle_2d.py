"""Plain FP64 CPU oracle of the two-dimensional solver of Sec. 2.2.

TEST INFRASTRUCTURE ONLY, under the same rules as ``sg_oracle``: only
``tests/`` may import it; it shares no code with the CUDA path.

The method is the one of the 3D oracle with the two-dimensional operators of
the paper: the five-point Laplacian, the four-cell restriction and the
9/3/3/1 prolongation.  The RKL coefficients, the Legendre-zero schedule and
the coarse-level tau are dimension-free and come from ``sg_oracle``.  Arrays
are C order ``[ny][nx]`` (x fastest); physical axis d (0 = x, 1 = y) is numpy
axis ``1 - d``.  Dirichlet face values: ``faces[0]``, ``faces[1]`` (the x
walls) have shape [ny], ``faces[2]``, ``faces[3]`` (the y walls) [nx].

Passages followed
-----------------
* Sec. 2.2.1, Eq. discrete_laplace_2D           -> ``laplacian2d``
* Sec. 2.2.2, Eqs. restriction_equation_2D /
  restriction_example_2D                        -> ``restrict2d``
* Sec. 2.2.3, Eq. prolongation_example_2D        -> ``prolong2d``
* Sec. 2.3, Eqs. solution_ghost, error_ghost,
  periodic (two axes)                           -> ``pad_ghosts2d``
* App. A, Eq. RKL_intermediate_source            -> ``rkl_superstep2d``
* Sec. 2.1, V-cycle list                         -> ``vcycle2d``, ``solve2d``

Readings: those of the 3D oracle restricted to two axes (cell centres, one
level increment per pass, coarse ghosts by the level's rule before the
prolongation, the coarsest solve by the accelerated RKL1 schedule with N the
level's larger extent, periodic potentials returned with zero mean).
"""

from __future__ import annotations

import math

import numpy as np

from .sg_oracle import (DIRICHLET, PERIODIC, Options, SolveInfo, accelerated_schedule, all_periodic,  # noqa: F401
                        coarse_tau_frac, level_count, rkl_coefficients, source, tau_step)


def spacing2d(shape, lo, hi):
    """(hx, hy) of a [ny][nx] grid on the rectangle [lo, hi] (x, y order)."""
    ny, nx = shape
    return ((hi[0] - lo[0]) / nx, (hi[1] - lo[1]) / ny)


def pad_ghosts2d(u, bc, faces=None):
    """u with one ghost layer on every side: 2 phi_face - active on a Dirichlet
    wall with face data (Eq. solution_ghost), -active without (Eq.
    error_ghost), the opposite active cell on a periodic axis (Eq. periodic).
    Without face data the rules run axis after axis over the padded extent, so
    the corner ghosts the prolongation reads are the repeated image."""
    ny, nx = u.shape
    p = np.zeros((ny + 2, nx + 2), dtype=np.float64)
    p[1:-1, 1:-1] = u
    full = faces is None
    inner = slice(None) if full else slice(1, -1)
    # x axis (numpy axis 1)
    if bc[0] == PERIODIC:
        p[inner, 0] = p[inner, -2]
        p[inner, -1] = p[inner, 1]
    elif faces is not None:
        p[1:-1, 0] = 2.0 * faces[0] - p[1:-1, 1]
        p[1:-1, -1] = 2.0 * faces[1] - p[1:-1, -2]
    else:
        p[inner, 0] = -p[inner, 1]
        p[inner, -1] = -p[inner, -2]
    # y axis (numpy axis 0)
    if bc[1] == PERIODIC:
        p[0, inner] = p[-2, inner]
        p[-1, inner] = p[1, inner]
    elif faces is not None:
        p[0, 1:-1] = 2.0 * faces[2] - p[1, 1:-1]
        p[-1, 1:-1] = 2.0 * faces[3] - p[-2, 1:-1]
    else:
        p[0, inner] = -p[1, inner]
        p[-1, inner] = -p[-2, inner]
    return p


def laplacian2d(u, h, bc, faces=None):
    """Five-point Laplacian, Eq. discrete_laplace_2D, with the ghost rules."""
    hx, hy = h
    p = pad_ghosts2d(u, bc, faces)
    c = p[1:-1, 1:-1]
    return ((p[1:-1, :-2] - 2.0 * c + p[1:-1, 2:]) / (hx * hx)
            + (p[:-2, 1:-1] - 2.0 * c + p[2:, 1:-1]) / (hy * hy))


def residual2d(u, rhs, h, bc, faces=None):
    """Eq. residual: r = L u - f."""
    return laplacian2d(u, h, bc, faces) - rhs


def l2norm2d(F, h=(1.0, 1.0)):
    """Sec. 4.1's norm with cell areas: [sum F^2 dA / A]^(1/2)."""
    dA = h[0] * h[1]
    return math.sqrt(float(np.sum(F * F) * dA / (dA * F.size)))


def restrict2d(r):
    """Eq. restriction_example_2D: the coarse value is the mean of its 4 children."""
    return (r[0::2, 0::2] + r[0::2, 1::2] + r[1::2, 0::2] + r[1::2, 1::2]) / 4.0


def prolong2d(e, bc):
    """Eq. prolongation_example_2D: each fine cell takes (9A + 3B + 3C + D)/16,
    A its coarse parent, B and C the parent's neighbours towards the fine cell
    along x and along y, D the diagonal neighbour between them.  Coarse ghosts
    follow the level's rule (-e for Dirichlet, copy for periodic)."""
    ny, nx = e.shape
    p = pad_ghosts2d(e, bc, None)
    out = np.empty((2 * ny, 2 * nx), dtype=np.float64)
    for oy in (0, 1):
        for ox in (0, 1):
            sy, sx = (-1 if oy == 0 else 1), (-1 if ox == 0 else 1)
            A = p[1:1 + ny, 1:1 + nx]
            B = p[1:1 + ny, 1 + sx:1 + sx + nx]
            C = p[1 + sy:1 + sy + ny, 1:1 + nx]
            D = p[1 + sy:1 + sy + ny, 1 + sx:1 + sx + nx]
            out[oy::2, ox::2] = (9.0 * A + 3.0 * B + 3.0 * C + D) / 16.0
    return out


def rkl_superstep2d(u, rhs, h, bc, faces, order, s, tau_frac):
    """One s-stage RKL super-step of du/dt = M u - f (Eq. RKL_intermediate_source)
    with M the five-point operator; tau = tau_frac tau_max, dt_par = 2 / (4
    sum_d 1/h_d^2).  The stage recursion is the 3D oracle's."""
    co = rkl_coefficients(order, s)
    tau = tau_step(order, s, h, tau_frac)

    def M_minus_f(y):
        return laplacian2d(y, h, bc, faces) - rhs

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


def coarse_solve2d(rhs, h, bc, opts, record=None):
    """Coarsest level: the accelerated RKL1 schedule (App. A.5) from u = 0 until
    the residual falls below coarse_tol of its start (0: exactly coarse_max_ss)."""
    N = max(rhs.shape)
    c = opts.coarse_tau_frac if opts.coarse_tau_frac > 0 else coarse_tau_frac(N)
    u = np.zeros_like(rhs)
    r_init = l2norm2d(residual2d(u, rhs, h, bc))
    done = 0
    for s in accelerated_schedule(N, opts.coarse_max_ss):
        if opts.coarse_tol > 0.0 and l2norm2d(residual2d(u, rhs, h, bc)) <= opts.coarse_tol * r_init:
            break
        u = rkl_superstep2d(u, rhs, h, bc, None, 1, s, c)
        done += 1
    if record is not None:
        record.append(done)
    return u


def vcycle2d(phi, f, h, bc, faces, L, opts, record=None):
    """One correction-scheme V-cycle (Sec. 2.1) on levels 0..L-1."""
    hs = [(h[0] * 2 ** l, h[1] * 2 ** l) for l in range(L)]
    per = all_periodic(bc)

    def relax(u, rhs, l, fc, count):
        for _ in range(count):
            u = rkl_superstep2d(u, rhs, hs[l], bc, fc, opts.rkl_order, opts.s_smooth, opts.tau_frac)
        return u

    u, rhs = [None] * L, [None] * L
    u[0], rhs[0] = relax(phi, f, 0, faces, opts.n_pre), f
    for l in range(1, L):
        fl = restrict2d(residual2d(u[l - 1], rhs[l - 1], hs[l - 1], bc, faces if l - 1 == 0 else None))
        if per:
            fl = fl - fl.mean()
        rhs[l] = -fl
        u[l] = np.zeros_like(fl)
        if l < L - 1:
            u[l] = relax(u[l], rhs[l], l, None, opts.n_pre)
        else:
            u[l] = coarse_solve2d(rhs[l], hs[l], bc, opts, record)
    for l in range(L - 2, 0, -1):
        u[l] = relax(u[l] + prolong2d(u[l + 1], bc), rhs[l], l, None, opts.n_post)
    if L > 1:
        u[0] = relax(u[0] + prolong2d(u[1], bc), rhs[0], 0, faces, opts.n_post)
    return u[0]


def solve2d(rho, lo, hi, bc, faces=None, four_pi_G=1.0, tol=1e-10, levels=0, opts=None, cycles=None):
    """Solve grad^2 phi = four_pi_G rho on a [ny][nx] grid: V-cycles while
    ||L phi - f|| / ||L 0 - f|| > tol (or exactly ``cycles``).  bc = (x, y)."""
    opts = opts or Options()
    rho = np.asarray(rho, dtype=np.float64)
    shape = rho.shape
    h = spacing2d(shape, lo, hi)
    L = levels if levels > 0 else level_count(shape)
    f = source(rho, four_pi_G, bc)
    phi = np.zeros(shape)
    info = SolveInfo(levels=L)
    info.r0 = l2norm2d(residual2d(np.zeros(shape), f, h, bc, faces))
    r0 = info.r0 if info.r0 > 0 else 1.0
    limit = cycles if cycles is not None else opts.max_cycles
    m = 0
    while True:
        rel = l2norm2d(residual2d(phi, f, h, bc, faces)) / r0
        info.history.append(rel)
        info.rel_residual = rel
        if (cycles is None and rel <= tol) or m >= limit:
            break
        phi = vcycle2d(phi, f, h, bc, faces, L, opts, record=info.coarse_ss)
        m += 1
    info.cycles = m
    if all_periodic(bc):
        phi = phi - phi.mean()
    return phi, info
