"""Plant plausible mistakes in the oracle (on the CPU) and check that the pins
catch every one of them.

Each mutation replaces one oracle routine by a subtly wrong variant (a sign,
a factor, a direction, a dropped term); the pins of ``test_oracle_pins`` are
then run directly and at least one must fail.
"""

import math

import numpy as np
import pytest

import oracle
import oracle.sg_oracle as S
import tests.test_oracle_pins as T

ORIG = {name: getattr(S, name) for name in dir(S) if callable(getattr(S, name))}


def _patch(monkeypatch, name, fn):
    monkeypatch.setattr(S, name, fn)
    monkeypatch.setattr(oracle, name, fn)


def _any_pin_fails():
    pins = [
        lambda: T.test_laplacian_matches_kronecker_matrix((4, 3, 5), (0, 0, 0)),
        lambda: T.test_laplacian_matches_kronecker_matrix((4, 6, 2), (1, 1, 1)),
        lambda: T.test_dirichlet_faces_enter_as_two_g_over_h2(),
        lambda: T.test_jacobi_special_case(),
        lambda: T.test_rkl1_stages_are_legendre(5),
        lambda: T.test_rkl2_stages_are_shifted_legendre(5),
        lambda: T.test_rkl_stable_up_to_tau_max(2, 3),
        lambda: T.test_superstep_error_propagation_matrix(2, 3, 1.0, (0, 0, 0)),
        lambda: T.test_superstep_error_propagation_matrix(1, 4, 1.0, (1, 1, 1)),
        lambda: T.test_restriction_and_prolongation_invariants(),
        lambda: T.test_prolongation_weights_27_9_3_1(),
        lambda: T.test_multigrid_matches_dst_direct_solve(),
        lambda: T.test_multigrid_matches_fft_direct_solve_periodic(),
        lambda: T.test_solve_matches_kronecker_direct((6, 4, 8), (0, 0, 0), (1, 2, 0.5)),
        lambda: T.test_vcycle_fixed_point(),
        lambda: T.test_accelerated_schedule_skips_repeats(),
        lambda: T.test_gsrb_sweep_radius_follows_young((4, 4, 6), (0, 0, 0)),
        lambda: T.test_gsrb_half_sweeps_solve_their_rows((0, 0, 0)),
        lambda: T.test_gravity_exact_for_quartics_away_from_walls(),
        lambda: T.test_gravity_of_linear_field_exact_at_the_walls(),
        lambda: T.test_gravity_periodic_sinusoid_closed_form(),
    ]
    failed = 0
    for pin in pins:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:
            failed += 1
    return failed


def m_restrict_quarter(r):
    return ORIG["restrict"](r) * 2.0


def m_prolong_wrong_direction(e, bc):
    # neighbours taken away from the fine cell instead of towards it
    nz, ny, nx = e.shape
    p = S.pad_ghosts(e, bc, None)
    out = np.empty((2 * nz, 2 * ny, 2 * nx))
    for oz in (0, 1):
        for oy in (0, 1):
            for ox in (0, 1):
                sz, sy, sx = (1 if oz == 0 else -1), (1 if oy == 0 else -1), (1 if ox == 0 else -1)
                acc = np.zeros((nz, ny, nx))
                for az in (0, 1):
                    for ay in (0, 1):
                        for ax in (0, 1):
                            w = (3 if az == 0 else 1) * (3 if ay == 0 else 1) * (3 if ax == 0 else 1)
                            dz, dy, dx = az * sz, ay * sy, ax * sx
                            acc = acc + w * p[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
                out[oz::2, oy::2, ox::2] = acc / 64.0
    return out


def m_error_ghost_even(u, bc, faces=None):
    p = ORIG["pad_ghosts"](u, bc, faces)
    if faces is None:
        p[:, :, 0] = p[:, :, 1]
    return p


def m_face_ghost_no_two(u, bc, faces=None):
    if faces is None:
        return ORIG["pad_ghosts"](u, bc, faces)
    half = [0.5 * f for f in faces]
    return ORIG["pad_ghosts"](u, bc, half)


def m_rkl2_gamma_sign(s):
    co = ORIG["rkl2_coefficients"](s)
    co.gamma_t = -co.gamma_t
    return co


def m_rkl1_nu_sign(s):
    co = ORIG["rkl1_coefficients"](s)
    co.nu = -co.nu
    return co


def m_laplacian_axes_swapped(u, h, bc, faces=None):
    return ORIG["laplacian"](u, (h[2], h[1], h[0]), bc, faces)


def m_tau_rkl2_like_rkl1(order, s, h, tau_frac):
    return ORIG["tau_step"](order, s, h, tau_frac) * ((s * s + s) / 2.0 / ((s * s + s - 2.0) / 4.0)
                                                      if order == 2 else 1.0)


def m_source_no_mean(rho, four_pi_G, bc):
    return four_pi_G * np.asarray(rho, dtype=np.float64)


def m_coarse_tau_one(N):
    return 1.0


def m_sk_opt_floor(k, N):
    return int(math.floor(S.BESSEL_J0_FIRST_ZERO / math.pi * (N / k) - 0.5))


def m_diagonal_no_wall(shape, h, bc):
    # the Dirichlet ghost's -1/h^2 left out of the row's diagonal
    return np.full(shape, -2.0 * sum(1.0 / (hd * hd) for hd in h))


def m_gsrb_colour_by_rows(u, rhs, h, bc, faces=None, omega=1.0):
    # colours by (j + k) only: neighbours along x share a colour
    nz, ny, nx = u.shape
    diag = S.operator_diagonal(u.shape, h, bc)
    K, J, _ = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    u = u.copy()
    for colour in (0, 1):
        mask = ((J + K) % 2) == colour
        r = S.laplacian(u, h, bc, faces) - rhs
        u[mask] = u[mask] - omega * r[mask] / diag[mask]
    return u


def m_gsrb_omega_dropped(u, rhs, h, bc, faces=None, omega=1.0):
    return ORIG["gs_rb_sweep"](u, rhs, h, bc, faces, 1.0)


def m_gravity_second_ghost_even(phi, h, bc, faces=None):
    # the second ghost layer copied from the second cell (even) instead of
    # reflected through the face value
    phi = np.asarray(phi, dtype=np.float64)
    out = np.empty((3,) + phi.shape)
    for d in range(3):
        ax = 2 - d
        n = phi.shape[ax]
        if bc[d] == S.PERIODIC:
            p = np.take(phi, np.arange(-2, n + 2) % n, axis=ax)
        else:
            lo = np.expand_dims(faces[2 * d], ax) if faces is not None else 0.0
            hi = np.expand_dims(faces[2 * d + 1], ax) if faces is not None else 0.0
            below = np.concatenate([np.take(phi, [1], axis=ax), 2.0 * lo - np.take(phi, [0], axis=ax)], axis=ax)
            above = np.concatenate([2.0 * hi - np.take(phi, [n - 1], axis=ax), np.take(phi, [n - 2], axis=ax)],
                                   axis=ax)
            p = np.concatenate([below, phi, above], axis=ax)
        at = lambda off: np.take(p, np.arange(2 + off, n + 2 + off), axis=ax)
        out[d] = -(4.0 / 3.0) * (at(1) - at(-1)) / (2.0 * h[d]) + (1.0 / 3.0) * (at(2) - at(-2)) / (4.0 * h[d])
    return out


def m_gravity_coefficient(phi, h, bc, faces=None):
    # 4/3 read as 3/4
    g = ORIG["gravity"](phi, h, bc, faces)
    return g * 0.5625


MUTATIONS = [
    ("restrict", m_restrict_quarter),
    ("prolong", m_prolong_wrong_direction),
    ("pad_ghosts", m_error_ghost_even),
    ("pad_ghosts", m_face_ghost_no_two),
    ("rkl2_coefficients", m_rkl2_gamma_sign),
    ("rkl1_coefficients", m_rkl1_nu_sign),
    ("laplacian", m_laplacian_axes_swapped),
    ("tau_step", m_tau_rkl2_like_rkl1),
    ("source", m_source_no_mean),
    ("coarse_tau_frac", m_coarse_tau_one),
    ("s_k_opt", m_sk_opt_floor),
    ("operator_diagonal", m_diagonal_no_wall),
    ("gs_rb_sweep", m_gsrb_colour_by_rows),
    ("gs_rb_sweep", m_gsrb_omega_dropped),
    ("gravity", m_gravity_second_ghost_even),
    ("gravity", m_gravity_coefficient),
]


@pytest.mark.parametrize("name,mutant", MUTATIONS, ids=[m[1].__name__ for m in MUTATIONS])
def test_pins_catch_planted_mistake(monkeypatch, name, mutant):
    _patch(monkeypatch, name, mutant)
    if name in ("rkl1_coefficients", "rkl2_coefficients"):
        orig_rc = ORIG["rkl_coefficients"]
        monkeypatch.setattr(S, "rkl_coefficients",
                            lambda order, s: (S.rkl1_coefficients(s) if order == 1 else S.rkl2_coefficients(s)))
        monkeypatch.setattr(oracle, "rkl_coefficients", S.rkl_coefficients)
        del orig_rc
    assert _any_pin_fails() > 0
