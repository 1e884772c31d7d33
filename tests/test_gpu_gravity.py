"""The acceleration of Sec. 3 (Eq. 4thorder_acceleration) on the GPU against
the FP64 oracle's ``gravity`` on the same seeded potentials, through the C ABI
(sg_gravity), on ragged grids with every boundary kind, extents of two cells,
host and device buffers, and at full size (256^3) on the analytic sphere
potential.

Tolerance: 1e-12 relative (max-norm of the difference over the max-norm of the
result).  The kernel forms 8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})
exactly in 64-bit fixed point on the level's scale and multiplies it by
-1 / (12 h) in FP64, the oracle evaluates the paper's form in FP64, so they
differ by rounding only; a second test bounds the kernel's distance from the
exact (rational) acceleration by the fixed-point design's own error.
"""

from fractions import Fraction

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
LO, HI = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)

# nx % 4 == 0 takes the 4-cell strip kernel (tiles of 128 x 8 cells): ragged
# rows (ny = 12, 10, 17, 9: a last tile of 4, 2, 1, 1 rows), two x tiles with a
# ragged second (132 cells: one strip) or two full ones (256), one strip
# (nx = 4, both x walls in one lane), two planes on a Dirichlet z axis, every
# boundary kind at a tile edge and a level edge; the other shapes the one
# cell per thread kernel
SHAPES_BC = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
             ((9, 37, 13), (0, 1, 0)), ((2, 6, 5), (0, 0, 1)), ((7, 2, 3), (1, 1, 0)),
             ((40, 19, 70), (0, 0, 0)), ((33, 17, 66), (1, 0, 1)),
             ((6, 10, 132), (1, 1, 0)), ((5, 17, 4), (0, 1, 0)), ((3, 9, 256), (0, 0, 1)), ((2, 8, 12), (0, 0, 0)),
             ((4, 9, 132), (0, 0, 0))]


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def relerr(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_grid(shape, bc, precision="fp64", faces=True):
    sg = _sg()
    g = sg.Grid(shape, LO, HI, bc, precision=precision)
    fc = None
    if faces and any(b == 0 for b in bc):
        fc = W.random_faces(shape, 5)
        g.set_boundary(fc)
    return g, O.spacing(shape, LO, HI), fc


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
@pytest.mark.parametrize("faces", [True, False])
def test_gravity_matches_oracle_device_buffers(shape, bc, faces):
    g, h, fc = make_grid(shape, bc, faces=faces)
    phi = W.random_field(shape, 6)
    out = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=torch.tensor(phi, device="cuda"))
    torch.cuda.synchronize()
    ref = O.gravity(phi, h, bc, fc)
    assert relerr(out, ref) < TOL


@pytest.mark.parametrize("shape,bc", SHAPES_BC[:3])
def test_host_buffers_equal_device_buffers(shape, bc):
    g, _, _ = make_grid(shape, bc, precision="mixed")
    phi = W.random_field(shape, 7)
    host = g.gravity(phi=phi)
    dev = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=dev, phi=torch.tensor(phi, device="cuda"))
    torch.cuda.synchronize()
    assert np.array_equal(host, dev.cpu().numpy())


def test_gravity_of_the_solution():
    p = W.smooth_sphere(32)
    sg = _sg()
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="fp64")
    g.set_boundary(p.faces)
    g.set_density(p.rho, p.four_pi_G)
    with pytest.raises(sg.SGError) as e:
        g.gravity()
    assert e.value.status == 7
    g.set_profiling(True)
    g.solve(tol=1e-12)
    a = g.gravity()
    assert g.kernel_stats()["gravity"]["launches"] == 1
    phi = g.potential()
    assert np.array_equal(a, g.gravity(phi=phi))
    ref = O.gravity(phi, O.spacing(p.shape, p.lo, p.hi), p.bc, p.faces)
    assert relerr(a, ref) < TOL


def test_full_size_256_analytic_sphere_potential():
    # the 256^3 workload's grid and faces, phi = the analytic sphere potential
    p = W.sphere(256)
    g, fc = _sg().Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed"), p.faces
    g.set_boundary(fc)
    out = torch.empty((3,) + p.shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=torch.tensor(p.exact, device="cuda"))
    torch.cuda.synchronize()
    ref = O.gravity(p.exact, O.spacing(p.shape, p.lo, p.hi), p.bc, fc)
    assert relerr(out, ref) < TOL


def test_overlapping_output_is_rejected():
    sg = _sg()
    g, _, _ = make_grid((8, 6, 10), (0, 0, 0))
    out = torch.zeros((3, 8, 6, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SGError) as e:
        g.gravity(out=out, phi=out[1])
    assert e.value.status == 1


def _exact_gravity(phi, h, bc, faces):
    """g_d = -(8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2})) / (12 h_d) in rational
    arithmetic from the FP64 inputs (ghosts: 2 phi_face - mirror past a
    Dirichlet wall, zero faces without data; periodic images), and the
    magnitude of the four-term combination per cell."""
    nz, ny, nx = phi.shape
    n = (nx, ny, nz)
    P = {}

    def val(i, j, k):
        key = (i, j, k)
        if key not in P:
            P[key] = Fraction(float(phi[k, j, i]))
        return P[key]

    def at(d, idx, off):
        p = list(idx)
        p[d] += off
        if 0 <= p[d] < n[d]:
            return val(*p)
        if bc[d] == O.PERIODIC:
            p[d] %= n[d]
            return val(*p)
        side = 0 if p[d] < 0 else 1
        m = list(idx)
        m[d] = -1 - p[d] if side == 0 else 2 * n[d] - 1 - p[d]
        fv = 0.0
        if faces is not None:
            fc = faces[2 * d + side]
            i, j, k = idx
            fv = fc[k, j] if d == 0 else (fc[k, i] if d == 1 else fc[j, i])
        return 2 * Fraction(float(fv)) - val(*m)

    out = np.empty((3,) + phi.shape, dtype=object)
    mag = np.zeros((3,) + phi.shape)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                idx = (i, j, k)
                for d in range(3):
                    a1, b1, a2, b2 = at(d, idx, 1), at(d, idx, -1), at(d, idx, 2), at(d, idx, -2)
                    comb = 8 * (a1 - b1) - (a2 - b2)
                    out[d, k, j, i] = -comb / (12 * Fraction(h[d]))
                    mag[d, k, j, i] = float(abs(comb))
    return out, mag


@pytest.mark.parametrize("shape,bc", [((10, 12, 16), (0, 0, 0)), ((8, 9, 12), (1, 0, 1)), ((5, 17, 4), (0, 1, 0)),
                                      ((2, 9, 136), (0, 0, 1)), ((9, 6, 10), (0, 0, 0))])
def test_gravity_fixed_point_within_its_error_bound(shape, bc):
    # the combination is exact on the level's fixed-point scale (unit
    # 2^(M - 1079), M the largest biased exponent of phi and, one above, of the
    # face data); a truncated operand is off by less than one unit (a ghost by
    # two), so the combination by less than 36 units, and two FP64 roundings follow
    g, h, fc = make_grid(shape, bc)
    X = np.linspace(0.0, 1.0, shape[2])[None, None, :]
    phi = 300.0 * np.cos(3.0 * X) + W.random_field(shape, 8)
    out = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=torch.tensor(phi, device="cuda"))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    exact, mag = _exact_gravity(phi, h, bc, fc)
    m = np.frexp(np.max(np.abs(phi)))[1] + 1022
    if fc is not None:
        for d in range(3):
            if bc[d] != O.PERIODIC:
                m = max(m, max(np.frexp(np.max(np.abs(fc[2 * d + s])))[1] + 1022 + 1 for s in range(2)))
    unit = 2.0 ** (m - 1079)
    worst = 0.0
    for idx in np.ndindex(got.shape):
        d = idx[0]
        c = 1.0 / (12.0 * h[d])
        ex = exact[idx]
        # truncation, then the rounding of the combination and of the product
        bound = c * 36.0 * unit + 2.0 ** -52 * (c * mag[idx] + abs(float(ex)))
        worst = max(worst, float(abs(Fraction(float(got[idx])) - ex)) / bound)
    assert worst <= 1.0, worst


@pytest.mark.parametrize("scale", [1e-300, 1e300])
@pytest.mark.parametrize("shape,bc", [((8, 12, 16), (0, 0, 0)), ((6, 10, 20), (1, 0, 1)), ((7, 9, 13), (0, 1, 0))])
def test_gravity_far_magnitudes_take_fp64_arithmetic(shape, bc, scale):
    # potentials beyond 2^-900 .. 2^900 fall outside the fixed-point scale:
    # both kernels (strips for nx % 4 == 0, one thread per cell otherwise)
    # then compute in FP64
    g, h, _ = make_grid(shape, bc, faces=False)
    fc = None
    if any(b == 0 for b in bc):
        fc = [scale * f for f in W.random_faces(shape, 5)]
        g.set_boundary(fc)
    phi = scale * W.random_field(shape, 9)
    out = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=torch.tensor(phi, device="cuda"))
    torch.cuda.synchronize()
    ref = O.gravity(phi, h, bc, fc)
    assert torch.isfinite(out).all()
    assert relerr(out, ref) < TOL


def test_gravity_not_finite_potential_stays_local():
    # a non-finite value makes the scale unusable (FP64 arithmetic); cells whose
    # stencil does not reach it keep their values
    shape, bc = (8, 12, 16), (0, 0, 0)
    g, h, fc = make_grid(shape, bc)
    phi = W.random_field(shape, 10)
    phi[4, 6, 8] = np.inf
    out = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=torch.tensor(phi, device="cuda"))
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert not np.isfinite(got[0, 4, 6, 7])
    phi0 = np.where(np.isfinite(phi), phi, 0.0)
    ref = O.gravity(phi0, h, bc, fc)
    assert abs(got[0, 0, 0, 0] - ref[0, 0, 0, 0]) <= 1e-12 * np.max(np.abs(ref))
