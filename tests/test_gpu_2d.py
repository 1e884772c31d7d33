"""GPU parity of the two-dimensional variants of Sec. 2.2 (five-point
operator, 4-cell restriction, 9/3/3/1 prolongation, the same RKL V-cycle)
against the pinned 2D oracle, element by element, through the C ABI
(sg_create_grid_2d and the operator / solve entry points).

Tolerances: FP64 1e-12 relative (max-norm of the difference over the max-norm
of the result; only the rounding order differs), FP32 operators 2e-5 (a few
hundred FP32 ulps after the stencil's cancellation), mixed-precision solves
1e-8 relative L2 after refinement to a residual of 1e-11.
"""

import numpy as np
import pytest

import oracle as O
import oracle.sg_oracle_2d as O2
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64, TOL32 = 1e-12, 2e-5
LO, HI = (0.0, -0.5), (1.3, 0.4)
CASES = [((24, 40), (0, 0)), ((32, 16), (1, 1)), ((20, 36), (1, 0)), ((12, 8), (0, 1))]


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def relerr(a, b):
    a = a.detach().double().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def faces2d(shape, seed):
    rng = np.random.default_rng(seed)
    ny, nx = shape
    return [rng.standard_normal(ny), rng.standard_normal(ny), rng.standard_normal(nx), rng.standard_normal(nx)]


def make(shape, bc, precision, seed=5):
    sg = _sg()
    g = sg.Grid2D(shape, LO, HI, bc, precision=precision)
    faces = faces2d(shape, seed)
    g.set_boundary(faces)
    return g, O2.spacing2d(shape, LO, HI), [f if b == 0 else np.zeros_like(f)
                                             for f, b in zip(faces, (bc[0], bc[0], bc[1], bc[1]))]


def test_level_rule_and_shapes():
    g, _, _ = make((48, 80), (0, 0), "fp64")
    assert g.max_levels == O.level_count((48, 80)) == 4
    assert g.level_shape(1) == (24, 40)


@pytest.mark.parametrize("shape,bc", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_residual_restrict_2d(shape, bc, precision):
    g, h, faces = make(shape, bc, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    u = W.random_field(shape, 11)
    rhs = 40.0 * W.random_field(shape, 12)
    coarse = torch.full((shape[0] // 2, shape[1] // 2), float("nan"), dtype=dt, device="cuda")
    if precision == "fp64":
        # level 0 with its face data (Eq. solution_ghost)
        sumsq, mx = g.op_residual_restrict(0, dev(u), dev(rhs), coarse)
        r = -O2.residual2d(u, rhs, h, bc, faces)
        assert abs(sumsq - float(np.sum(r * r))) <= 1e-12 * float(np.sum(r * r))
        assert abs(mx - float(np.max(np.abs(r)))) <= 1e-12 * float(np.max(np.abs(r)))
        assert relerr(coarse, O2.restrict2d(r)) < TOL64
    else:
        u32, r32 = u.astype(np.float32).astype(np.float64), rhs.astype(np.float32).astype(np.float64)
        g.op_residual_restrict(0, dev(u, dt), dev(rhs, dt), coarse, homogeneous=True)
        r = -O2.residual2d(u32, r32, h, bc, None)
        assert relerr(coarse, O2.restrict2d(r)) < TOL32


@pytest.mark.parametrize("shape,bc", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prolong_correct_2d(shape, bc, precision):
    g, _, _ = make(shape, bc, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    e = W.random_field((shape[0] // 2, shape[1] // 2), 13)
    fine = W.random_field(shape, 14)
    out = dev(fine, dt)
    g.op_prolong_correct(0, dev(e, dt), out)
    if precision == "mixed":
        e, fine = e.astype(np.float32).astype(np.float64), fine.astype(np.float32).astype(np.float64)
    ref = fine + O2.prolong2d(e, bc)
    assert relerr(out, ref) < (TOL64 if precision == "fp64" else TOL32)


@pytest.mark.parametrize("shape,bc", CASES)
@pytest.mark.parametrize("order,s", [(2, 3), (1, 4)])
def test_superstep_2d_fp64(shape, bc, order, s):
    g, h, faces = make(shape, bc, "fp64")
    u, rhs = W.random_field(shape, 15), 30.0 * W.random_field(shape, 16)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    g.op_superstep(0, order, s, 0.9, dev(u), dev(rhs), out)
    ref = O2.rkl_superstep2d(u, rhs, h, bc, faces, order, s, 0.9)
    assert relerr(out, ref) < TOL64


@pytest.mark.parametrize("shape,bc", CASES)
def test_superstep_2d_fp32_homogeneous(shape, bc):
    g, h, _ = make(shape, bc, "mixed")
    u, rhs = W.random_field(shape, 17), 30.0 * W.random_field(shape, 18)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    g.op_superstep(0, 2, 3, 1.0, dev(u, torch.float32), dev(rhs, torch.float32), out, homogeneous=True)
    u32, r32 = u.astype(np.float32).astype(np.float64), rhs.astype(np.float32).astype(np.float64)
    ref = O2.rkl_superstep2d(u32, r32, h, bc, None, 2, 3, 1.0)
    assert relerr(out, ref) < 5e-5


def _problem(shape, bc, seed):
    rho = W.random_field(shape, seed) + (0.0 if bc == (1, 1) else 0.5)
    faces = faces2d(shape, seed + 1)
    faces = [f if b == 0 else np.zeros_like(f) for f, b in zip(faces, (bc[0], bc[0], bc[1], bc[1]))]
    return rho, faces


@pytest.mark.parametrize("shape,bc", [((64, 64), (0, 0)), ((48, 80), (1, 0)), ((64, 32), (1, 1))])
@pytest.mark.parametrize("order,s,c", [(2, 3, 1.0), (1, 2, 0.75)])
def test_solve_2d_fp64_fixed_cycles_match_oracle(shape, bc, order, s, c):
    sg = _sg()
    rho, faces = _problem(shape, bc, 21)
    g = sg.Grid2D(shape, LO, HI, bc, precision="fp64")
    g.set_boundary(faces)
    g.set_density(rho, 2.0)
    g.set_options(rkl_order=order, s_smooth=s, tau_frac=c, coarse_tol=0.0, coarse_max_ss=10, fixed_cycles=4)
    info = g.solve(tol=0.0)
    phi = g.potential()
    opts = O.Options(rkl_order=order, s_smooth=s, tau_frac=c, coarse_tol=0.0, coarse_max_ss=10)
    ref, rinfo = O2.solve2d(rho, LO, HI, bc, faces, 2.0, opts=opts, cycles=4)
    assert info["levels"] == rinfo.levels and info["cycles"] == 4
    assert rel_l2(phi, ref) < TOL64
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("shape,bc", [((128, 128), (0, 0)), ((96, 160), (1, 1)), ((64, 128), (0, 1))])
def test_solve_2d_mixed_refined_matches_converged_oracle(shape, bc):
    sg = _sg()
    rho, faces = _problem(shape, bc, 31)
    g = sg.Grid2D(shape, LO, HI, bc, precision="mixed")
    g.set_boundary(faces)
    g.set_density(rho, 1.0)
    info = g.solve(tol=1e-11)
    phi = g.potential()
    assert info["rel_residual"] <= 1e-11
    ref, rinfo = O2.solve2d(rho, LO, HI, bc, faces, 1.0, tol=1e-13)
    assert rel_l2(phi, ref) < 1e-8
    # the V-cycle reduces the residual like the oracle's (same algorithm, FP32 inner cycle)
    _, rtol = O2.solve2d(rho, LO, HI, bc, faces, 1.0, tol=1e-11)
    assert abs(info["cycles"] - rtol.cycles) <= 1
    if bc == (1, 1):
        assert abs(phi.mean()) < 1e-12 * np.abs(phi).max()


def test_solve_2d_tolerance_stop_matches_oracle_cycle_counts():
    sg = _sg()
    shape, bc = (128, 96), (0, 0)
    rho, faces = _problem(shape, bc, 41)
    g = sg.Grid2D(shape, LO, HI, bc, precision="fp64")
    g.set_boundary(faces)
    g.set_density(rho, 1.0)
    info = g.solve(tol=1e-9)
    ref, rinfo = O2.solve2d(rho, LO, HI, bc, faces, 1.0, tol=1e-9)
    assert info["cycles"] == rinfo.cycles
    assert info["coarse_ss"] == rinfo.coarse_ss
    assert rel_l2(g.potential(), ref) < TOL64


def test_grid2d_rejects_wrong_faces():
    sg = _sg()
    g = sg.Grid2D((16, 24), LO, HI, (0, 0), precision="fp64")
    with pytest.raises(ValueError):
        g.set_boundary([np.zeros(16), np.zeros(16), np.zeros(16), np.zeros(24)])
    with pytest.raises(ValueError):
        g.set_boundary([np.zeros(16)] * 6)


@pytest.mark.parametrize("shape,bc", CASES)
def test_gravity_2d_against_3d_oracle_on_one_plane(shape, bc):
    # a 2D grid's acceleration: x and y components of the fourth-order
    # difference (Sec. 3), z component zero; the 3D oracle on one periodic plane
    g, h, faces = make(shape, bc, "fp64")
    phi = W.random_field(shape, 19)
    out = torch.empty((3,) + shape, dtype=torch.float64, device="cuda")
    g.gravity(out=out, phi=dev(phi))
    ny, nx = shape
    f3 = [faces[0].reshape(1, ny), faces[1].reshape(1, ny), faces[2].reshape(1, nx), faces[3].reshape(1, nx),
          np.zeros((ny, nx)), np.zeros((ny, nx))]
    ref = O.gravity(phi[None], (h[0], h[1], 1.0), (bc[0], bc[1], 1), f3)
    got = out.cpu().numpy()
    assert relerr(got[:2], ref[:2, 0]) < TOL64
    assert np.all(got[2] == 0.0)
