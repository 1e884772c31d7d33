"""Pins of the two-dimensional oracle (Sec. 2.2) against routes of its own:
a Kronecker-product matrix, the exact sinusoidal eigenvector, impulse
responses and invariants of the transfer operators, dense direct solves, and
the pinned 3D oracle on a z-invariant problem (one periodic plane pair, where
the seven-point operator is the five-point one)."""

import math

import numpy as np
import pytest

import oracle as O
import oracle.sg_oracle_2d as O2
import workloads as W


def kron2d(shape, h, bc):
    """The five-point operator from 1D second differences (Dirichlet corner
    entry -3 for the ghost = -active rule, circulant for periodic)."""
    def d2(n, b):
        T = np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
        if b == O.PERIODIC:
            T[0, -1] += 1.0
            T[-1, 0] += 1.0
        else:
            T[0, 0] -= 1.0
            T[-1, -1] -= 1.0
        return T
    ny, nx = shape
    return np.kron(np.eye(ny), d2(nx, bc[0])) / h[0] ** 2 + np.kron(d2(ny, bc[1]), np.eye(nx)) / h[1] ** 2


def faces2d(shape, seed):
    rng = np.random.default_rng(seed)
    ny, nx = shape
    return [rng.standard_normal(ny), rng.standard_normal(ny), rng.standard_normal(nx), rng.standard_normal(nx)]


def face_vector(shape, h, bc, faces):
    b = np.zeros(shape)
    if bc[0] == O.DIRICHLET:
        b[:, 0] += 2 * faces[0] / h[0] ** 2
        b[:, -1] += 2 * faces[1] / h[0] ** 2
    if bc[1] == O.DIRICHLET:
        b[0, :] += 2 * faces[2] / h[1] ** 2
        b[-1, :] += 2 * faces[3] / h[1] ** 2
    return b


@pytest.mark.parametrize("shape,bc", [((5, 7), (0, 0)), ((6, 4), (1, 1)), ((4, 6), (1, 0)), ((7, 8), (0, 1))])
def test_laplacian2d_matches_kronecker_matrix_and_face_vector(shape, bc):
    h = (0.3, 0.45)
    u = W.random_field(shape, 1)
    A = kron2d(shape, h, bc)
    np.testing.assert_allclose(O2.laplacian2d(u, h, bc), (A @ u.ravel()).reshape(shape), atol=1e-11, rtol=0)
    fc = faces2d(shape, 2)
    np.testing.assert_allclose(O2.laplacian2d(u, h, bc, fc) - O2.laplacian2d(u, h, bc),
                               face_vector(shape, h, bc, fc), atol=1e-11, rtol=0)


def test_sinusoid_is_exact_eigenvector():
    n = 16
    x = (np.arange(n) + 0.5) / n
    u = np.outer(np.sin(np.pi * x), np.sin(np.pi * x))
    lam = -(8.0 * n * n) * math.sin(math.pi / (2 * n)) ** 2
    np.testing.assert_allclose(O2.laplacian2d(u, (1.0 / n, 1.0 / n), (0, 0)), lam * u, atol=1e-10, rtol=0)


def test_restriction_and_prolongation():
    rng = np.random.default_rng(3)
    r = rng.standard_normal((8, 12))
    c = O2.restrict2d(r)
    assert c.shape == (4, 6)
    assert abs(c.mean() - r.mean()) < 1e-14
    assert abs(c[1, 2] - r[2:4, 4:6].mean()) < 1e-14
    np.testing.assert_allclose(O2.restrict2d(np.full((6, 4), 2.5)), 2.5, rtol=0, atol=1e-15)
    # impulse response: the four fine children of a cell get 9/16, the
    # neighbours' children towards it 3/16, the diagonal ones 1/16
    e = np.zeros((5, 6))
    e[2, 3] = 16.0
    P = O2.prolong2d(e, (1, 1))
    assert P[4, 6] == 9.0 and P[5, 7] == 9.0
    assert P[4, 5] == 3.0 and P[3, 6] == 3.0 and P[3, 5] == 1.0
    assert P[4, 4] == 0.0 and P[2, 6] == 0.0
    assert abs(P.sum() - 4 * 16.0) < 1e-12
    # constants (periodic) and linear functions (interior) are reproduced
    np.testing.assert_allclose(O2.prolong2d(np.full((4, 6), 1.75), (1, 1)), 1.75, rtol=0, atol=1e-15)
    xc, yc = (np.arange(6) + 0.5) * 2, (np.arange(5) + 0.5) * 2
    xf, yf = np.arange(12) + 0.5, np.arange(10) + 0.5
    lin = O2.prolong2d(0.3 + 0.7 * xc[None, :] - 1.1 * yc[:, None], (0, 0))
    ref = 0.3 + 0.7 * xf[None, :] - 1.1 * yf[:, None]
    np.testing.assert_allclose(lin[1:-1, 1:-1], ref[1:-1, 1:-1], rtol=0, atol=1e-12)
    # wall: with e_ghost = -e the wall-adjacent fine value is linear through zero
    w = O2.prolong2d(np.ones((4, 4)), (0, 1))
    np.testing.assert_allclose(w[:, 0], 0.5, rtol=0, atol=1e-15)


@pytest.mark.parametrize("bc", [(0, 0), (1, 0), (1, 1)])
def test_multigrid_reaches_dense_solution(bc):
    shape, lo, hi = (16, 24), (0.0, -0.5), (1.2, 0.3)
    rho = W.random_field(shape, 4)
    fc = None if bc == (1, 1) else faces2d(shape, 5)
    phi, info = O2.solve2d(rho, lo, hi, bc, fc, 2.0, tol=1e-12)
    assert info.levels == 3 and info.cycles < 40
    h = O2.spacing2d(shape, lo, hi)
    A = kron2d(shape, h, bc)
    f = O.source(rho, 2.0, bc).ravel()
    if bc == (1, 1):
        Aa = np.vstack([A, np.ones((1, A.shape[0]))])
        ref = np.linalg.lstsq(Aa, np.concatenate([f, [0.0]]), rcond=None)[0]
    else:
        ref = np.linalg.solve(A, f - face_vector(shape, h, bc, fc).ravel())
    ref = ref.reshape(shape)
    assert np.linalg.norm(phi - ref) / np.linalg.norm(ref) < 1e-10


def test_equals_z_invariant_3d_problem():
    # two periodic planes in z carrying the same data: the 7-point operator
    # on a z-constant field is the 5-point one, so the 3D discrete solution is
    # the 2D one on both planes (3D dense solve of the pinned 3D oracle)
    shape2, lo, hi = (8, 10), (0.0, 0.0), (1.0, 0.8)
    rho2 = W.random_field(shape2, 6)
    fc2 = faces2d(shape2, 7)
    phi2, _ = O2.solve2d(rho2, lo, hi, (0, 0), fc2, 1.5, tol=1e-13)
    rho3 = np.stack([rho2, rho2])
    z = np.zeros
    fc3 = [np.stack([fc2[0], fc2[0]]), np.stack([fc2[1], fc2[1]]),
           np.stack([fc2[2], fc2[2]]), np.stack([fc2[3], fc2[3]]), z((8, 10)), z((8, 10))]
    phi3 = O.dense_solve(rho3, (lo[0], lo[1], 0.0), (hi[0], hi[1], 0.25), (0, 0, 1), fc3, 1.5)
    np.testing.assert_allclose(phi3[0], phi2, rtol=0, atol=1e-10 * np.abs(phi2).max())
    np.testing.assert_allclose(phi3[1], phi2, rtol=0, atol=1e-10 * np.abs(phi2).max())


def test_vcycle_reduces_residual_about_tenfold():
    # Sec. 4.1 reports about a decade per V-cycle; 64^2, six levels, RKL1 s = 2
    # at 0.75 tau_max with N_pre = 2, N_post = 1, and RKL2 s = 3 at 0.9 tau_max
    # with N_pre = 5, N_post = 3 (RKL2 with (2, 1) gains only about 2.5x: its
    # polynomial stays near a_s on the high modes)
    rho = W.random_field((64, 64), 8)
    for opts in (O.Options(rkl_order=1, s_smooth=2, tau_frac=0.75),
                 O.Options(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3)):
        _, info = O2.solve2d(rho, (0, 0), (1, 1), (0, 0), None, 1.0, opts=opts, cycles=6)
        f = [info.history[m] / info.history[m + 1] for m in range(1, 6)]
        assert all(5.0 < f_ < 20.0 for f_ in f), f


# planted mistakes, each of which some pin above must catch
def _m_restrict_half(r):
    return (r[0::2, 0::2] + r[0::2, 1::2] + r[1::2, 0::2] + r[1::2, 1::2]) / 2.0


def _m_prolong_swapped_weights(e, bc):
    ny, nx = e.shape
    p = O2.pad_ghosts2d(e, bc, None)
    out = np.empty((2 * ny, 2 * nx))
    for oy in (0, 1):
        for ox in (0, 1):
            sy, sx = (-1 if oy == 0 else 1), (-1 if ox == 0 else 1)
            A = p[1:1 + ny, 1:1 + nx]
            B = p[1:1 + ny, 1 + sx:1 + sx + nx]
            C = p[1 + sy:1 + sy + ny, 1:1 + nx]
            D = p[1 + sy:1 + sy + ny, 1 + sx:1 + sx + nx]
            out[oy::2, ox::2] = (9.0 * A + 3.0 * B + C + 3.0 * D) / 16.0
    return out


_ORIG_PAD = O2.pad_ghosts2d


def _m_pad_even_faces(u, bc, faces=None):
    # face ghost without the factor 2
    p = _ORIG_PAD(u, bc, None if faces is None else [0.5 * f for f in faces])
    return p


@pytest.mark.parametrize("name,mutant", [("restrict2d", _m_restrict_half),
                                         ("prolong2d", _m_prolong_swapped_weights),
                                         ("pad_ghosts2d", _m_pad_even_faces)])
def test_pins_catch_planted_mistakes(monkeypatch, name, mutant):
    monkeypatch.setattr(O2, name, mutant)
    pins = [lambda: test_restriction_and_prolongation(),
            lambda: test_multigrid_reaches_dense_solution((0, 0)),
            lambda: test_laplacian2d_matches_kronecker_matrix_and_face_vector((5, 7), (0, 0)),
            lambda: test_equals_z_invariant_3d_problem()]
    failed = 0
    for pin in pins:
        try:
            with np.errstate(all="ignore"):
                pin()
        except Exception:
            failed += 1
    assert failed > 0
