"""The acceleration of Sec. 3 (Eq. 4thorder_acceleration) on the GPU against
the FP64 oracle's ``gravity`` on the same seeded potentials, through the C ABI
(sg_gravity), on ragged grids with every boundary kind, extents of two cells,
host and device buffers, and at full size (256^3) on the analytic sphere
potential.

Tolerance: 1e-12 relative (max-norm of the difference over the max-norm of the
result): both sides evaluate the same four differences in FP64, the kernel in
the form 8 (phi_{+1} - phi_{-1}) - (phi_{+2} - phi_{-2}) times -1 / (12 h), the
oracle in the paper's form, so they differ by rounding only.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12
LO, HI = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)

SHAPES_BC = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
             ((9, 37, 13), (0, 1, 0)), ((2, 6, 5), (0, 0, 1)), ((7, 2, 3), (1, 1, 0)),
             ((40, 19, 70), (0, 0, 0)), ((33, 17, 66), (1, 0, 1))]


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
