"""GPU parity of the FP64 residual r = f - A phi that confirms a mixed solve
(Sec. 2.1), computed with the neighbour sum in exact 64-bit fixed point
(sg_op_residual_exact).

Two references:
* the exact residual, in rational arithmetic (Python fractions) from the same
  FP64 inputs and the same FP64 coefficients 1/h_d^2: the kernel must lie
  within the error its design allows -- the truncation of every operand to the
  level's fixed-point unit 2^(M - 1079) (M the largest biased exponent of phi
  and, one above, of the face values), at most 18 units in the sum with equal
  h (6 per axis otherwise), plus one FP64 rounding of each sum and FMA;
* the oracle's FP64 residual, within FP64 evaluation error.
A near-constant potential (every value close to 1024, so the conversion drops
no bit) shows the sum is exact where an FP64 evaluation rounds.
"""

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# nx % 4 == 0: the fixed-point strip kernel; the last shape (nx = 18) takes the FP64 stencil
SHAPES_BC = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
             ((8, 36, 12), (0, 1, 0)), ((10, 14, 18), (0, 1, 0))]


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def make_grid(shape, bc, uniform, faces_seed=5):
    sg = _sg()
    nz, ny, nx = shape
    if uniform:
        lo, hi = (0.0, 0.0, 0.0), (nx / 16.0, ny / 16.0, nz / 16.0)      # h = 1/16 on every axis
    else:
        lo, hi = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)
    g = sg.Grid(shape, lo, hi, bc, precision="mixed")
    faces = None
    if any(b == 0 for b in bc):
        faces = W.random_faces(shape, faces_seed)
        g.set_boundary(faces)
    return g, O.spacing(shape, lo, hi), faces


def biased_exponent(v):
    v = float(v)
    if v == 0.0:
        return 0
    return math.frexp(v)[1] + 1022          # |v| = m 2^e, m in [0.5, 1): IEEE biased exponent e - 1 + 1023


def fixed_point_exponent(u, bc, faces):
    m = max(biased_exponent(np.max(np.abs(u))), 0)
    if faces is not None:
        for d in range(3):
            if bc[d] != O.PERIODIC:
                for s in range(2):
                    m = max(m, biased_exponent(np.max(np.abs(faces[2 * d + s]))) + 1)
    return m


def exact_residual(u, f, ih2, bc, faces):
    """r = f - sum_d ih2_d (u[-d] + u[+d] - 2 u) in rational arithmetic, with the
    ghost rules of Sec. 2.3 (2 phi_face - u, -u, periodic image), and per cell
    the axis second differences D_d."""
    nz, ny, nx = u.shape
    U = [[[Fraction(float(u[k, j, i])) for i in range(nx)] for j in range(ny)] for k in range(nz)]
    n = (nx, ny, nz)
    r = np.empty(u.shape, dtype=object)
    D = np.empty(u.shape + (3,), dtype=object)
    ihf = [Fraction(float(v)) for v in ih2]

    def ghost(d, side, c, k, j, i):
        if bc[d] == O.PERIODIC:
            idx = [i, j, k]
            idx[d] = n[d] - 1 if side == 0 else 0
            return U[idx[2]][idx[1]][idx[0]]
        if faces is not None:
            fc = faces[2 * d + side]
            fv = fc[k, j] if d == 0 else (fc[k, i] if d == 1 else fc[j, i])
            return 2 * Fraction(float(fv)) - c
        return -c

    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = U[k][j][i]
                acc = Fraction(float(f[k, j, i]))
                idx = (i, j, k)
                for d in range(3):
                    lo_i, hi_i = list(idx), list(idx)
                    lo_i[d] -= 1
                    hi_i[d] += 1
                    a = U[lo_i[2]][lo_i[1]][lo_i[0]] if lo_i[d] >= 0 else ghost(d, 0, c, k, j, i)
                    b = U[hi_i[2]][hi_i[1]][hi_i[0]] if hi_i[d] < n[d] else ghost(d, 1, c, k, j, i)
                    D[k, j, i, d] = a + b - 2 * c
                    acc -= ihf[d] * D[k, j, i, d]
                r[k, j, i] = acc
    return r, D


def truncate_to_f32(r64):
    """The FP32 copy the kernel writes: the FP64 significand truncated to 24 bits."""
    b = r64.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    return b.view(np.float64).astype(np.float32)


def run(g, u, f):
    shape = u.shape
    r64 = torch.full(shape, float("nan"), dtype=torch.float64, device="cuda")
    r32 = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    sumsq, mx = g.op_residual_exact(dev(u), dev(f), r64, r32)
    torch.cuda.synchronize()
    return r64.cpu().numpy(), r32.cpu().numpy(), sumsq, mx


def check_against_exact(r_gpu, u, f, h, bc, faces, fixed):
    ih2 = [1.0 / (hd * hd) for hd in h]
    r_ex, D = exact_residual(u, f, ih2, bc, faces)
    uniform = ih2[0] == ih2[1] == ih2[2]
    M = fixed_point_exponent(u, bc, faces)
    unit = 2.0 ** (M - 1079)
    trunc_units = 18.0 * ih2[0] if uniform else 6.0 * sum(ih2)
    worst = 0.0
    for idx in np.ndindex(u.shape):
        err = abs(Fraction(float(r_gpu[idx])) - r_ex[idx])
        mag = abs(float(f[idx])) + sum(ih2[d] * abs(float(D[idx + (d,)])) for d in range(3))
        bound = unit * trunc_units + 2.0 ** -50 * mag
        if not fixed:      # the FP64 stencil: a few roundings of every partial sum
            bound = 2.0 ** -48 * (mag + 4.0 * sum(ih2) * float(np.max(np.abs(u))))
        worst = max(worst, float(err) / bound)
    assert worst <= 1.0, worst
    return r_ex


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
@pytest.mark.parametrize("uniform", [True, False])
def test_exact_residual_matches_exact_and_oracle(shape, bc, uniform):
    g, h, faces = make_grid(shape, bc, uniform)
    X = np.linspace(0.0, 1.0, shape[2])[None, None, :]
    u = 300.0 * np.cos(3.0 * X) + W.random_field(shape, 61)     # a smooth part and noise
    f = W.random_field(shape, 62)
    r64, r32, sumsq, mx = run(g, u, f)
    fixed = shape[2] % 4 == 0
    assert np.all(np.isfinite(r64))
    check_against_exact(r64, u, f, h, bc, faces, fixed)
    # the oracle's FP64 residual (paper sign: A u - f), within FP64 evaluation error
    ref = -O.residual(u, f, h, bc, faces)
    scale = 4.0 * sum(1.0 / (hd * hd) for hd in h) * np.max(np.abs(u)) + np.max(np.abs(f))
    assert np.max(np.abs(r64 - ref)) <= 64 * 2.0 ** -52 * scale
    # the FP32 copy and the norms of it
    if fixed:
        np.testing.assert_array_equal(r32, truncate_to_f32(r64))
    else:
        np.testing.assert_allclose(r32, r64, rtol=2.0 ** -23, atol=0)
    r32d = r32.astype(np.float64)
    assert abs(sumsq - np.sum(r32d ** 2)) <= 1e-5 * np.sum(r32d ** 2)
    assert mx == np.max(np.abs(r32d))


@pytest.mark.parametrize("uniform", [True, False])
def test_exact_residual_near_constant_potential_is_exact(uniform):
    # every value of u and of the faces within 1e-8 of 1024, on both sides:
    # the conversion to the fixed-point scale drops no bit (no value lies more
    # than four binades below the largest), the neighbour sum is exact, and only
    # the final roundings remain; an FP64 evaluation rounds wherever a partial
    # sum of values on different sides of 1024 lands in a coarser binade
    shape, bc = (6, 8, 12), (0, 1, 0)
    g, h, _ = make_grid(shape, bc, uniform)
    faces = [1024.0 + 1e-9 * fc for fc in W.random_faces(shape, 63)]
    g.set_boundary(faces)
    u = 1024.0 + 1e-9 * W.random_field(shape, 64)
    assert u.min() < 1024.0 < u.max()
    f = 1e-7 * W.random_field(shape, 65)
    r64, _, _, _ = run(g, u, f)
    r_ex = check_against_exact(r64, u, f, h, bc, faces, True)
    ex = np.array([float(v) for v in r_ex.ravel()]).reshape(shape)
    err_gpu = np.max(np.abs(r64 - ex))
    err_fp64 = np.max(np.abs(-O.residual(u, f, h, bc, faces) - ex))
    assert err_fp64 > 0.0
    assert err_gpu <= 1e-3 * err_fp64
    # with equal h the only roundings left are those of the sum (|ih2 S| = |f - r|)
    # and of the final FMA
    if uniform:
        assert err_gpu <= 2.0 ** -51 * np.max(np.abs(f) + np.abs(f - ex))


def test_exact_residual_not_finite_potential_reports_nan():
    shape, bc = (8, 8, 8), (0, 0, 0)
    g, h, faces = make_grid(shape, bc, True)
    u = W.random_field(shape, 66)
    u[3, 4, 5] = np.inf
    f = W.random_field(shape, 67)
    r64, _, sumsq, _ = run(g, u, f)
    assert not np.isfinite(sumsq)
    assert not np.isfinite(r64[3, 4, 5])
    # far from the bad cell the FP64 stencil still gives the residual
    ref = -O.residual(np.where(np.isfinite(u), u, 0.0), f, h, bc, faces)
    assert abs(r64[0, 0, 0] - ref[0, 0, 0]) <= 1e-12 * np.max(np.abs(ref))


def test_mixed_solve_confirmation_matches_oracle_residual():
    # the rel. residual a mixed solve reports is the confirmation's; it agrees
    # with the oracle's FP64 residual of the returned potential
    p = W.sphere(64)
    sg = _sg()
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed")
    g.set_boundary(p.faces)
    g.set_density(p.rho, p.four_pi_G)
    info = g.solve(tol=1e-9, levels=4)
    phi = g.potential()
    h = O.spacing(p.shape, p.lo, p.hi)
    f = O.source(p.rho, p.four_pi_G, p.bc)
    rel = O.l2norm(O.residual(phi, f, h, p.bc, p.faces)) / O.l2norm(O.residual(np.zeros(p.shape), f, h, p.bc,
                                                                                   p.faces))
    assert info["rel_residual"] <= 1e-9
    assert abs(info["rel_residual"] - rel) <= 1e-3 * rel


@pytest.mark.parametrize("scale", [1e-300, 1e300])
@pytest.mark.parametrize("shape,bc", [((8, 12, 16), (0, 0, 0)), ((6, 10, 20), (1, 0, 1))])
def test_exact_residual_far_magnitudes_take_the_fp64_stencil(shape, bc, scale):
    # values beyond 2^-900 .. 2^900 are outside the fixed-point scale's range:
    # the kernel computes those levels in FP64, within FP64 evaluation error
    g, h, faces = make_grid(shape, bc, True)
    if faces is not None:
        faces = [scale * fc for fc in faces]
        g.set_boundary(faces)
    u = scale * W.random_field(shape, 68)
    f = scale * W.random_field(shape, 69)
    r64, r32, _, _ = run(g, u, f)
    ref = -O.residual(u, f, h, bc, faces)
    assert np.all(np.isfinite(r64))
    assert np.max(np.abs(r64 - ref)) <= 1e-12 * np.max(np.abs(ref))
