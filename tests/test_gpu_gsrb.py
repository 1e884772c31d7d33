"""The paper's own smoother on the GPU: red-black Gauss-Seidel / SOR sweeps
(Sec. 2.2.4, App. B) as a single operator, as the V-cycle's smoother (the
paper's configuration: GS-RB with N_pre = 2, N_post = 1, accelerated RKL1 on
the coarsest level) and as the single-level solver, against the FP64 oracle on
the same seeded inputs, through the C ABI.

Tolerances: FP64 sweeps agree with the oracle to 1e-12 relative (the rounding
order differs, and the kernel multiplies by the row's reciprocal diagonal
where the oracle divides); FP32 sweeps to 2e-5 relative, as for the other
FP32 operators.  Solves run the same fixed number of cycles on both sides and
compare potentials and residual histories; the mixed-precision solve is
compared at convergence.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5
LO, HI = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)

# ragged tiles, every boundary kind; odd extents on Dirichlet axes are allowed
SHAPES_BC = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
             ((9, 36, 13), (0, 1, 0))]


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def relerr(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make_grid(shape, bc, precision):
    sg = _sg()
    g = sg.Grid(shape, LO, HI, bc, precision=precision)
    faces = None
    if any(b == 0 for b in bc):
        faces = W.random_faces(shape, 5)
        g.set_boundary(faces)
    return g, O.spacing(shape, LO, HI), faces


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
@pytest.mark.parametrize("omega", [1.0, 1.6, 0.0])
def test_sweep_fp64_with_faces(shape, bc, omega):
    g, h, faces = make_grid(shape, bc, "fp64")
    u, rhs = W.random_field(shape, 6), 50.0 * W.random_field(shape, 7)
    ud = dev(u)
    g.op_gsrb_sweep(0, ud, dev(rhs), omega=omega)
    torch.cuda.synchronize()
    om = omega if omega > 0 else O.sor_omega(shape, h)
    ref = O.gs_rb_sweep(u, rhs, h, bc, faces, om)
    assert relerr(ud, ref) < TOL64


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
def test_sweep_fp32_homogeneous(shape, bc):
    g, h, _ = make_grid(shape, bc, "mixed")
    u, rhs = W.random_field(shape, 8), 50.0 * W.random_field(shape, 9)
    ud = dev(u, torch.float32)
    g.op_gsrb_sweep(0, ud, dev(rhs, torch.float32), omega=1.3, homogeneous=True)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.gs_rb_sweep(u32, r32, h, bc, None, 1.3)
    assert relerr(ud.double(), ref) < TOL32


def test_sweep_on_a_coarse_level_ignores_faces():
    shape, bc = (20, 12, 36), (0, 1, 0)
    g, h, _ = make_grid(shape, bc, "fp64")
    cs = (10, 6, 18)
    hc = tuple(2 * x for x in h)
    u, rhs = W.random_field(cs, 10), W.random_field(cs, 11)
    ud = dev(u)
    g.op_gsrb_sweep(1, ud, dev(rhs))
    torch.cuda.synchronize()
    assert relerr(ud, O.gs_rb_sweep(u, rhs, hc, bc, None, 1.0)) < TOL64


def grid_for(p, precision, **opts):
    sg = _sg()
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision=precision)
    if p.faces is not None:
        g.set_boundary(p.faces)
    g.set_density(p.rho, p.four_pi_G)
    g.set_options(**opts)
    return g


def test_vcycle_with_gsrb_smoother_fp64_matches_oracle():
    # the paper's configuration (Sec. 4.1) on the 64^3 sphere, 4 levels, 4 cycles
    p = W.sphere(64)
    g = grid_for(p, "fp64", smoother="gsrb", coarse_tol=0.0, coarse_max_ss=12, fixed_cycles=4)
    g.set_profiling(True)
    info = g.solve(tol=0.0, levels=4)
    st = g.kernel_stats()
    phi = g.potential()
    opts = O.Options(smoother="gsrb", coarse_tol=0.0, coarse_max_ss=12)
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, levels=4, opts=opts, cycles=4)
    assert rel_l2(phi, ref) < 1e-12
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)
    # (N_pre + N_post) sweeps on each of the three finer levels, two colours each
    assert st["gsrb_sweep"]["launches"] == 4 * 3 * 3 * 2
    assert st["rkl_stage_l0"]["launches"] == 0 and st["bottom_levels"]["launches"] == 0
    # the paper's figure: about one decade per V-cycle
    h = info["history"]
    assert all(h[m + 1] < h[m] / 4 for m in range(1, 4))


@pytest.mark.parametrize("bc", [(0, 0, 0), (1, 0, 1)])
def test_vcycle_with_gsrb_smoother_mixed_converges_to_oracle(bc):
    p = W.sphere(64)
    if bc != (0, 0, 0):
        p = W.grf(64, seed=3)
        p.bc = bc
        p.faces = W.random_faces(p.shape, 12)
    g = grid_for(p, "mixed", smoother="gsrb")
    info = g.solve(tol=1e-11, levels=4)
    phi = g.potential()
    assert info["rel_residual"] <= 1e-11
    ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, tol=1e-13, levels=4,
                     opts=O.Options(smoother="gsrb"))
    assert rel_l2(phi, ref) < 1e-8


@pytest.mark.parametrize("omega", [1.0, 0.0])
def test_single_level_gs_and_sor_fp64_match_oracle(omega):
    p = W.smooth_sphere(32)
    g = grid_for(p, "fp64", smoother="gsrb", omega=omega, fixed_cycles=30)
    info = g.solve(tol=0.0, levels=1)
    phi = g.potential()
    opts = O.Options(smoother="gsrb", omega=omega)
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, levels=1, opts=opts, cycles=30)
    assert rel_l2(phi, ref) < 1e-12
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_max_residual_stop(precision):
    # App. B's test: stop at the first sweep whose max |L phi - f| is below the bound
    p = W.smooth_sphere(32)
    f = O.source(p.rho, p.four_pi_G, p.bc)
    h = O.spacing(p.shape, p.lo, p.hi)
    bound = 1e-6 * float(np.abs(O.residual(np.zeros(p.shape), f, h, p.bc, p.faces)).max())
    g = grid_for(p, precision, smoother="gsrb", omega=0.0, max_residual_tol=bound, max_cycles=250)
    info = g.solve(tol=0.0, levels=1)
    phi = g.potential()
    assert info["max_residual"] <= bound
    assert float(np.abs(O.residual(phi, f, h, p.bc, p.faces)).max()) <= bound * 1.001
    g.set_options(max_residual_tol=0.0, fixed_cycles=info["cycles"] - 1)
    before = g.solve(tol=0.0, levels=1)
    assert before["max_residual"] > bound


def test_odd_periodic_extent_is_rejected():
    sg = _sg()
    g = sg.Grid((16, 24, 9), LO, HI, (1, 1, 0), precision="fp64")
    g.set_density(W.random_field((16, 24, 9), 1), 1.0)
    g.set_options(smoother="gsrb")
    with pytest.raises(sg.SGError) as e:
        g.solve(tol=1e-6, levels=1)
    assert e.value.status == 1
    u = dev(W.random_field((16, 24, 9), 2))
    with pytest.raises(sg.SGError):
        g.op_gsrb_sweep(0, u, dev(W.random_field((16, 24, 9), 3)))
    with pytest.raises(sg.SGError):
        g.set_options(omega=2.0)


@pytest.mark.parametrize("smoother,precision", [("rkl", "fp64"), ("gsrb", "fp64"), ("gsrb", "mixed")])
def test_no_pre_smoothing_matches_oracle(smoother, precision):
    # N_pre = 0: each coarser level's correction starts from zero and goes
    # straight to the restriction
    p = W.sphere(32)
    g = grid_for(p, precision, smoother=smoother, n_pre=0, n_post=2, coarse_tol=0.0, coarse_max_ss=8,
                 fixed_cycles=3)
    g.solve(tol=0.0, levels=3)
    opts = O.Options(smoother=smoother, n_pre=0, n_post=2, coarse_tol=0.0, coarse_max_ss=8)
    ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, levels=3, opts=opts, cycles=3)
    assert rel_l2(g.potential(), ref) < (1e-12 if precision == "fp64" else 1e-5)


def test_backward_with_gsrb_smoother_matches_oracle_adjoint():
    # the adjoint solve runs the same smoother (homogeneous boundaries)
    p = W.sphere(32)
    g = grid_for(p, "fp64", smoother="gsrb")
    g.solve(tol=1e-12, levels=3)
    w = W.loss_weights(p.shape, 9)
    grad = np.empty(p.shape)
    g.backward(w, grad, tol=1e-12)
    ref, _ = O.adjoint(w, p.lo, p.hi, p.bc, p.four_pi_G, tol=1e-13, levels=3, opts=O.Options(smoother="gsrb"))
    assert rel_l2(grad, ref) < 1e-9


def test_batch_with_gsrb_smoother_equals_single_solves():
    sg = _sg()
    probs = [W.sphere(32), W.smooth_sphere(32)]
    grids = [grid_for(q, "mixed", smoother="gsrb") for q in probs]
    infos = sg.solve_batch(grids, tol=1e-9)
    batch = [gr.potential() for gr in grids]
    for q, gr, info, b in zip(probs, grids, infos, batch):
        gr.set_density(q.rho, q.four_pi_G)
        single = gr.solve(tol=1e-9)
        assert single["cycles"] == info["cycles"]
        assert np.array_equal(gr.potential(), b)
