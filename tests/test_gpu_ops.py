"""GPU parity of every single operator against the FP64 oracle, element by
element, on seeded inputs with ragged tiles (sizes not multiples of the
32 x 8 thread tile) and every boundary kind.  All calls go through the C ABI
(sg_op_*).

Tolerances: FP64 kernels agree with the oracle to 1e-12 relative (max-norm of
the difference over max-norm of the result; only the rounding order differs).
FP32 kernels (the mixed-precision inner cycle) agree to 2e-5 relative, a few
hundred FP32 ulps after the cancellation of the 7-point stencil.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 2e-5

SHAPES_BC = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
             ((8, 36, 12), (0, 1, 0))]


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def relerr(a, b):
    a = a.detach().cpu().numpy() if isinstance(a, torch.Tensor) else a
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def make_grid(shape, bc, precision, faces_seed=5):
    sg = _sg()
    lo, hi = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)
    g = sg.Grid(shape, lo, hi, bc, precision=precision)
    faces = None
    if any(b == 0 for b in bc):
        faces = W.random_faces(shape, faces_seed)
        g.set_boundary(faces)
    return g, O.spacing(shape, lo, hi), faces


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
@pytest.mark.parametrize("order,s,c", [(1, 1, 1.0), (1, 4, 0.8), (2, 2, 1.0), (2, 3, 1.0), (2, 6, 0.9)])
def test_superstep_fp64(shape, bc, order, s, c):
    g, h, faces = make_grid(shape, bc, "fp64")
    u, rhs = W.random_field(shape, 6), 50.0 * W.random_field(shape, 7)
    out = torch.empty(shape, dtype=torch.float64, device="cuda")
    g.op_superstep(0, order, s, c, dev(u), dev(rhs), out)
    torch.cuda.synchronize()
    ref = O.rkl_superstep(u, rhs, h, bc, faces, order, s, c)
    assert relerr(out, ref) < TOL64


@pytest.mark.parametrize("shape,bc", SHAPES_BC[:2])
@pytest.mark.parametrize("order,s,c", [(1, 2, 0.75), (2, 3, 1.0), (2, 5, 1.0)])
@pytest.mark.parametrize("fused", [0, 1])
def test_superstep_fp32_homogeneous(shape, bc, order, s, c, fused):
    g, h, _ = make_grid(shape, bc, "mixed")
    g.set_options(fused=fused)
    u, rhs = W.random_field(shape, 8), 50.0 * W.random_field(shape, 9)
    out = torch.empty(shape, dtype=torch.float32, device="cuda")
    g.op_superstep(0, order, s, c, dev(u, torch.float32), dev(rhs, torch.float32), out, homogeneous=True)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.rkl_superstep(u32, r32, h, bc, None, order, s, c)
    assert relerr(out.double(), ref) < TOL32


# The FP32 per-stage kernel on 4-cell strips (nx % 4 == 0): an odd ny with a
# periodic x axis, a row of 33 strips (two blocks in x, the second ragged), a
# row of 16 strips (16 x 16 blocks), a level a single strip wide; every
# boundary kind on some axis.
STRIP_STAGE_SHAPES = [((24, 37, 44), (1, 0, 1)), ((9, 20, 132), (0, 1, 0)), ((12, 18, 64), (1, 1, 1)),
                      ((6, 5, 4), (0, 0, 0))]


@pytest.mark.parametrize("shape,bc", STRIP_STAGE_SHAPES)
@pytest.mark.parametrize("order,s,c", [(1, 3, 0.75), (2, 3, 0.9), (2, 4, 1.0)])
def test_strip_stage_kernel_matches_oracle(shape, bc, order, s, c):
    g, h, _ = make_grid(shape, bc, "mixed")
    g.set_options(fused=0)
    u, rhs = W.random_field(shape, 50), 50.0 * W.random_field(shape, 51)
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    g.op_superstep(0, order, s, c, dev(u, torch.float32), dev(rhs, torch.float32), out, homogeneous=True)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.rkl_superstep(u32, r32, h, bc, None, order, s, c)
    assert torch.isfinite(out).all()
    assert relerr(out.double(), ref) < TOL32


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
def test_residual_restrict_fp64(shape, bc):
    g, h, faces = make_grid(shape, bc, "fp64")
    u, rhs = W.random_field(shape, 10), W.random_field(shape, 11)
    coarse = torch.empty(tuple(n // 2 for n in shape), dtype=torch.float64, device="cuda")
    sumsq, mx = g.op_residual_restrict(0, dev(u), dev(rhs), coarse)
    r_paper = O.residual(u, rhs, h, bc, faces)          # L u - f
    ref = O.restrict(-r_paper)                            # the kernel restricts f - L u
    assert relerr(coarse, ref) < TOL64
    assert abs(sumsq - np.sum(r_paper ** 2)) <= 1e-12 * np.sum(r_paper ** 2)
    assert abs(mx - np.max(np.abs(r_paper))) <= 1e-12 * np.max(np.abs(r_paper))
    # norm only (no restriction) at a coarser, homogeneous level
    u1 = W.random_field(coarse.shape, 12)
    r1 = W.random_field(coarse.shape, 13)
    sumsq1, mx1 = g.op_residual_restrict(1, dev(u1), dev(r1), None)
    h1 = tuple(2 * x for x in h)
    rr = O.residual(u1, r1, h1, bc, None)
    assert abs(sumsq1 - np.sum(rr ** 2)) <= 1e-12 * np.sum(rr ** 2)


@pytest.mark.parametrize("shape,bc", SHAPES_BC[:2])
def test_residual_restrict_fp32(shape, bc):
    g, h, _ = make_grid(shape, bc, "mixed")
    u, rhs = W.random_field(shape, 14), W.random_field(shape, 15)
    coarse = torch.empty(tuple(n // 2 for n in shape), dtype=torch.float32, device="cuda")
    g.op_residual_restrict(0, dev(u, torch.float32), dev(rhs, torch.float32), coarse, homogeneous=True)
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.restrict(-O.residual(u32, r32, h, bc, None))
    assert relerr(coarse.double(), ref) < TOL32


@pytest.mark.parametrize("shape,bc", SHAPES_BC)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_prolong_correct(shape, bc, precision):
    g, h, _ = make_grid(shape, bc, precision)
    dt = torch.float64 if precision == "fp64" else torch.float32
    fine0 = W.random_field(shape, 16)
    coarse = W.random_field(tuple(n // 2 for n in shape), 17)
    fine = dev(fine0, dt)
    g.op_prolong_correct(0, dev(coarse, dt), fine)
    torch.cuda.synchronize()
    if precision == "mixed":
        fine0 = fine0.astype(np.float32).astype(np.float64)
        coarse = coarse.astype(np.float32).astype(np.float64)
    ref = fine0 + O.prolong(coarse, bc)
    assert relerr(fine.double(), ref) < (TOL64 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("shape,bc,level", [((32, 32, 32), (0, 0, 0), 2), ((32, 16, 64), (1, 1, 1), 2),
                                            ((16, 16, 16), (0, 0, 0), 1)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_coarse_solve_fixed_count(shape, bc, level, precision):
    g, h, _ = make_grid(shape, bc, precision)
    g.set_options(coarse_tol=0.0, coarse_max_ss=9)
    cshape = tuple(n >> level for n in shape)
    hl = tuple(x * 2 ** level for x in h)
    rhs = W.random_field(cshape, 18)
    if all(b == 1 for b in bc):
        rhs -= rhs.mean()
    dt = torch.float64 if precision == "fp64" else torch.float32
    out = torch.empty(cshape, dtype=dt, device="cuda")
    done = g.op_coarse_solve(level, dev(rhs, dt), out)
    assert done == 9
    opts = O.Options(coarse_tol=0.0, coarse_max_ss=9)
    ref = O.coarse_solve(rhs.astype(np.float32).astype(np.float64) if precision == "mixed" else rhs,
                         hl, bc, None, opts)
    assert relerr(out.double(), ref) < (1e-11 if precision == "fp64" else 1e-4)


def test_coarse_solve_tolerance_stop():
    g, h, _ = make_grid((16, 16, 16), (0, 0, 0), "fp64")
    g.set_options(coarse_tol=1e-6, coarse_max_ss=200)
    rhs = W.random_field((8, 8, 8), 19)
    out = torch.empty((8, 8, 8), dtype=torch.float64, device="cuda")
    done = g.op_coarse_solve(1, dev(rhs), out)
    rec = []
    ref = O.coarse_solve(rhs, tuple(2 * x for x in h), (0, 0, 0), None,
                         O.Options(coarse_tol=1e-6, coarse_max_ss=200), record=rec)
    assert done == rec[0]
    assert relerr(out, ref) < 1e-11


# ---------------------------------------------------------------------------
# Fused (temporally blocked) FP32 super-step: every stage count it supports,
# both orders, Y0 = 0 and general Y0, every boundary mix, ragged and tiny shapes.
# ---------------------------------------------------------------------------
FUSED_SHAPES = [((20, 12, 36), (0, 0, 0)), ((16, 24, 8), (1, 1, 1)), ((12, 20, 40), (1, 0, 1)),
                ((37, 19, 70), (0, 1, 0)), ((6, 4, 2), (1, 1, 1)), ((4, 6, 10), (0, 0, 0)),
                ((20, 30, 44), (0, 0, 0)), ((18, 4, 4), (0, 0, 1)), ((9, 26, 100), (0, 0, 1))]

# Shapes with nx % 4 == 0, even ny and no wrap in x and y, where the s = 2, 3
# kernel can stage planes by tensor-map box copies (staging = "tma"): ragged x
# and y tiles, a level narrower than the x halo, a periodic z axis (z
# reflections and wraps), several z chunks per tile column.
TMA_SHAPES = [((20, 12, 36), (0, 0, 0)), ((20, 30, 44), (0, 0, 0)), ((18, 4, 4), (0, 0, 1)),
              ((9, 26, 100), (0, 0, 1)), ((168, 160, 160), (0, 0, 0)), ((160, 162, 164), (0, 0, 1))]


@pytest.mark.parametrize("shape,bc", TMA_SHAPES)
@pytest.mark.parametrize("order,s", [(2, 3), (1, 2)])
@pytest.mark.parametrize("zero", [False, True])
def test_tma_staging_matches_oracle_and_copy_staging(shape, bc, order, s, zero):
    g, h, _ = make_grid(shape, bc, "mixed")
    u = np.zeros(shape) if zero else W.random_field(shape, 40)
    rhs = 50.0 * W.random_field(shape, 41)
    outs = {}
    for staging in ("cp_async", "tma"):
        g.set_options(staging=staging)
        out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        g.op_superstep(0, order, s, 0.9, None if zero else dev(u, torch.float32), dev(rhs, torch.float32), out,
                       homogeneous=True)
        torch.cuda.synchronize()
        outs[staging] = out
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.rkl_superstep(u32, r32, h, bc, None, order, s, 0.9)
    assert torch.isfinite(outs["tma"]).all()
    assert relerr(outs["tma"].double(), ref) < 5e-5
    # the same arithmetic on the same staged values: identical to the last bit
    assert torch.equal(outs["tma"], outs["cp_async"])


def test_tma_staging_solve_equals_copy_staging():
    # 176^3: level 0 (5.5 M cells) runs the fused super-step (levels of 2^22 cells and more)
    p = W.sphere(176)
    sg = pytest.importorskip("paper_2306_05332_gb300")
    phis = {}
    for staging in ("cp_async", "tma"):
        g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed")
        g.set_boundary(p.faces)
        g.set_density(p.rho, 1.0)
        g.set_options(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, staging=staging)
        info = g.solve(tol=1e-8, levels=4)
        assert info["rel_residual"] <= 1e-8
        phis[staging] = g.potential()
    np.testing.assert_array_equal(phis["tma"], phis["cp_async"])


@pytest.mark.parametrize("shape,bc", FUSED_SHAPES)
@pytest.mark.parametrize("order,s", [(1, 2), (1, 5), (2, 2), (2, 3), (2, 4), (2, 6), (1, 6)])
@pytest.mark.parametrize("zero", [False, True])
def test_fused_superstep_matches_oracle(shape, bc, order, s, zero):
    g, h, _ = make_grid(shape, bc, "mixed")
    assert g.options().fused == 1
    c = 0.9
    u = np.zeros(shape) if zero else W.random_field(shape, 20)
    rhs = 50.0 * W.random_field(shape, 21)
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    g.op_superstep(0, order, s, c, None if zero else dev(u, torch.float32), dev(rhs, torch.float32), out,
                   homogeneous=True)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.rkl_superstep(u32, r32, h, bc, None, order, s, c)
    assert torch.isfinite(out).all()
    assert relerr(out.double(), ref) < 5e-5


# The plane-streaming super-step at sizes where it runs several z chunks per
# tile column: ragged tiles in y and z, and an x extent that is not a multiple
# of four (scalar plane loads).
LEAN_SHAPES = [((168, 160, 160), (0, 0, 0)), ((170, 160, 162), (1, 0, 1))]


@pytest.mark.parametrize("shape,bc", LEAN_SHAPES)
@pytest.mark.parametrize("order,s", [(2, 3), (1, 2)])
@pytest.mark.parametrize("zero", [False, True])
def test_plane_streaming_superstep_matches_oracle(shape, bc, order, s, zero):
    assert shape[0] * shape[1] * shape[2] >= 1 << 22
    g, h, _ = make_grid(shape, bc, "mixed")
    c = 1.0
    u = np.zeros(shape) if zero else W.random_field(shape, 30)
    rhs = 50.0 * W.random_field(shape, 31)
    out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
    g.op_superstep(0, order, s, c, None if zero else dev(u, torch.float32), dev(rhs, torch.float32), out,
                   homogeneous=True)
    torch.cuda.synchronize()
    u32 = u.astype(np.float32).astype(np.float64)
    r32 = rhs.astype(np.float32).astype(np.float64)
    ref = O.rkl_superstep(u32, r32, h, bc, None, order, s, c)
    assert torch.isfinite(out).all()
    assert relerr(out.double(), ref) < 5e-5


def test_fused_equals_unfused_fp32():
    shape, bc = (64, 48, 80), (0, 0, 0)
    g, h, _ = make_grid(shape, bc, "mixed")
    u = dev(W.random_field(shape, 22), torch.float32)
    rhs = dev(W.random_field(shape, 23), torch.float32)
    a = torch.empty(shape, dtype=torch.float32, device="cuda")
    b = torch.empty(shape, dtype=torch.float32, device="cuda")
    g.set_options(fused=1)
    g.op_superstep(1 - 1, 2, 3, 1.0, u, rhs, a, homogeneous=True)
    g.set_options(fused=0)
    g.op_superstep(0, 2, 3, 1.0, u, rhs, b, homogeneous=True)
    torch.cuda.synchronize()
    assert relerr(a.double(), b.double().cpu().numpy()) < 1e-5


@pytest.mark.parametrize("fused", [0, 1])
def test_mixed_solve_fused_and_unfused_agree(fused):
    p = W.sphere(64)
    sg = pytest.importorskip("paper_2306_05332_gb300")
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed")
    g.set_boundary(p.faces)
    g.set_density(p.rho, 1.0)
    g.set_options(fused=fused)
    info = g.solve(tol=1e-11, levels=4)
    ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-13, levels=4)
    assert np.linalg.norm(g.potential() - ref) / np.linalg.norm(ref) < 1e-8
    _, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-11, levels=4)
    assert abs(info["cycles"] - rinfo.cycles) <= 1


def test_fused_option_change_takes_effect_on_the_same_grid():
    # the cycle graph is cached per option set: switching the fused super-step
    # off and on must re-capture (level 0 of 176^3 has 5.5 M cells, above the
    # fused size of 2^22 cells; the levels below run one launch per stage)
    p = W.sphere(176)
    sg = pytest.importorskip("paper_2306_05332_gb300")
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed")
    g.set_boundary(p.faces)
    g.set_options(rkl_order=2, s_smooth=3, fused=1, fixed_cycles=2)
    counts = {}
    for fused in (1, 0, 1):
        g.set_options(fused=fused)
        g.set_density(p.rho, 1.0)
        g.set_profiling(True)
        g.solve(tol=0.0, levels=4)
        counts.setdefault(fused, []).append(g.kernel_stats()["rkl_stage_l0"]["launches"])
        g.set_profiling(False)
    # fused: one launch per super-step (3 per cycle); unfused: one per stage
    assert counts[1] == [2 * 3, 2 * 3]
    assert counts[0] == [2 * 3 * 3]


def test_operator_wrappers_check_shapes():
    # every operator argument must have its level's shape (coarse arrays the
    # next level's); a mismatch raises before anything is launched
    g, _, _ = make_grid((16, 24, 8), (1, 1, 1), "fp64")
    u = torch.zeros((16, 24, 8), dtype=torch.float64, device="cuda")
    rhs = torch.zeros_like(u)
    out = torch.zeros_like(u)
    bad = torch.zeros((16, 24, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        g.op_superstep(0, 2, 3, 1.0, u, bad, out)
    with pytest.raises(ValueError):
        g.op_superstep(1, 2, 3, 1.0, u, rhs, out)            # level-0 arrays at level 1
    with pytest.raises(ValueError):
        g.op_residual_restrict(0, u, rhs, torch.zeros((8, 12, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(ValueError):
        g.op_prolong_correct(0, bad, out)
    with pytest.raises(ValueError):
        g.op_gsrb_sweep(0, bad, rhs)
    with pytest.raises(ValueError):
        g.op_coarse_solve(0, bad, out)
    with pytest.raises(TypeError):
        g.op_superstep(0, 2, 3, 1.0, u.float(), rhs, out)
