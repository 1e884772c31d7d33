"""GPU parity of whole solves (sg_solve / sg_backward / sg_solve_batch) with
the FP64 oracle.

* FP64 path: same cycle count and options as the oracle, coarsest solve with a
  fixed super-step count, potential within 1e-12 relative L2 of the oracle.
* Mixed path (FP32 V-cycle inside FP64 defect correction): solved to a tight
  residual, potential within 1e-8 relative L2 of the oracle's converged FP64
  solution.
* Full size (256^3 sphere, five levels): the residual of the GPU potential,
  recomputed by the oracle on the CPU in FP64, meets the tolerance.
"""

import math

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def grid_for(p, precision, **opts):
    sg = _sg()
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision=precision)
    if p.faces is not None:
        g.set_boundary(p.faces)
    g.set_density(p.rho, p.four_pi_G)
    if opts:
        g.set_options(**opts)
    return g


def test_sinusoid_single_level_rkl1_closed_form():
    # 32^3 sinusoid, single-level RKL1, s = 24 from dt_par = h^2/6, to 1e-10.
    p = W.sinusoid(32)
    g = grid_for(p, "fp64", single_tau_frac=1.0)
    info = g.solve(tol=1e-10, s=24, levels=1)
    phi = g.potential()
    assert info["cycles"] == 3
    opts = O.Options(single_s=24, single_tau_frac=1.0)
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, None, 1.0, tol=1e-10, levels=1, opts=opts)
    assert rinfo.cycles == 3
    assert rel_l2(phi, ref) < 1e-12
    h = 1.0 / 32
    lam = -(12.0 / h ** 2) * math.sin(math.pi * h / 2) ** 2
    exact = p.rho / lam
    g24 = float(O.legendre(24, math.cos(math.pi / 32)))
    np.testing.assert_allclose(phi - exact, -(g24 ** 3) * exact, atol=1e-13 * np.abs(exact).max())
    # relative residuals agree to rounding of the FP64 residual (~1e-15 of r0)
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)


@pytest.mark.parametrize("single_s", [0, -1])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_level_accelerated_rkl_matches_oracle(single_s, precision):
    # App. A.5 (single_s = 0: the Legendre-zero schedule, k = N/2 .. 1 with
    # repeats skipped, then s_1,opt) and App. A.4 (single_s = -1: the global
    # s_opt every super-step), single-level, a fixed count of super-steps
    p = W.smooth_sphere(32)
    steps = 24
    g = grid_for(p, precision, single_s=single_s, fixed_cycles=steps)
    info = g.solve(tol=0.0, levels=1)
    phi = g.potential()
    opts = O.Options(single_s=single_s)
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, p.four_pi_G, levels=1, opts=opts, cycles=steps)
    assert info["cycles"] == rinfo.cycles == steps
    if precision == "fp64":
        assert rel_l2(phi, ref) < 1e-12
        np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)
    else:
        # FP32 super-steps on the error equation, FP64 update: FP32 rounding of
        # each correction, relative to the potential
        assert rel_l2(phi, ref) < 1e-5
    if single_s == -1:
        sg = _sg()
        assert sg.plan_s_opt(32) == O.s_opt_global(32)


def test_single_level_accelerated_rkl_anisotropic_to_tolerance():
    # the schedule of the largest extent on a 24 x 40 x 32 box with mixed walls
    shape, lo, hi, bc = (24, 40, 32), (0.0, 0.0, 0.0), (1.0, 1.25, 0.75), (0, 1, 0)
    rho = W.random_field(shape, 81)
    faces = W.random_faces(shape, 82)
    p = W.Problem(rho=rho, lo=lo, hi=hi, bc=bc, faces=faces, four_pi_G=1.0)
    g = grid_for(p, "fp64")
    info = g.solve(tol=1e-9, levels=1)
    phi = g.potential()
    ref, rinfo = O.solve(rho, lo, hi, bc, faces, 1.0, tol=1e-9, levels=1)
    assert info["cycles"] == rinfo.cycles
    assert rel_l2(phi, ref) < 1e-12


@pytest.mark.parametrize("order,s,c", [(2, 3, 1.0), (1, 2, 0.75)])
def test_sphere_fp64_fixed_cycles_match_oracle(order, s, c):
    p = W.sphere(64)
    kw = dict(rkl_order=order, s_smooth=s, tau_frac=c, coarse_tol=0.0, coarse_max_ss=12, fixed_cycles=5)
    g = grid_for(p, "fp64", **kw)
    info = g.solve(tol=0.0, levels=4)
    phi = g.potential()
    opts = O.Options(rkl_order=order, s_smooth=s, tau_frac=c, coarse_tol=0.0, coarse_max_ss=12)
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, levels=4, opts=opts, cycles=5)
    assert info["cycles"] == 5 and info["levels"] == 4
    assert rel_l2(phi, ref) < 1e-12
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)


def test_sphere_fp64_tolerance_stop_matches_oracle():
    p = W.sphere(64)
    g = grid_for(p, "fp64")
    info = g.solve(tol=1e-9, levels=4)
    phi = g.potential()
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-9, levels=4, opts=O.Options())
    assert info["cycles"] == rinfo.cycles
    assert info["coarse_ss"] == rinfo.coarse_ss
    assert rel_l2(phi, ref) < 1e-12


@pytest.mark.parametrize("order,s,c", [(2, 3, 1.0), (1, 2, 0.75)])
def test_sphere_mixed_refined_matches_oracle(order, s, c):
    p = W.sphere(64)
    g = grid_for(p, "mixed", rkl_order=order, s_smooth=s, tau_frac=c)
    info = g.solve(tol=1e-11, levels=4)
    phi = g.potential()
    assert info["rel_residual"] <= 1e-11
    opts = O.Options(rkl_order=order, s_smooth=s, tau_frac=c)
    ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-13, levels=4, opts=opts)
    assert rel_l2(phi, ref) < 1e-8
    # the oracle's own residual of the GPU potential
    h = O.spacing(p.shape, p.lo, p.hi)
    r = O.residual(phi, O.source(p.rho, 1.0, p.bc), h, p.bc, p.faces)
    r0 = O.l2norm(O.residual(np.zeros(p.shape), O.source(p.rho, 1.0, p.bc), h, p.bc, p.faces))
    assert O.l2norm(r) / r0 <= 1.01e-11


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_periodic_grf(precision):
    p = W.grf(32, seed=4)
    p.rho = p.rho + 1.5
    if precision == "fp64":
        g = grid_for(p, precision, coarse_tol=0.0, coarse_max_ss=10, fixed_cycles=6)
        g.solve(tol=0.0)
        phi = g.potential()
        ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, None, 1.0, opts=O.Options(coarse_tol=0.0, coarse_max_ss=10),
                         cycles=6)
        assert rel_l2(phi, ref) < 1e-12
    else:
        g = grid_for(p, precision)
        g.solve(tol=1e-11)
        phi = g.potential()
        ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, None, 1.0, tol=1e-13)
        assert rel_l2(phi, ref) < 1e-8
    assert abs(phi.mean()) < 1e-12 * np.abs(phi).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_anisotropic_mixed_boundaries(precision):
    shape, lo, hi, bc = (16, 32, 24), (0.0, 0.0, 0.0), (1.5, 2.0, 1.0), (1, 0, 0)
    rho = W.random_field(shape, 51)
    faces = W.random_faces(shape, 52)
    p = W.Problem(rho=rho, lo=lo, hi=hi, bc=bc, faces=faces, four_pi_G=2.0)
    g = grid_for(p, precision)
    info = g.solve(tol=1e-11)
    phi = g.potential()
    ref, rinfo = O.solve(rho, lo, hi, bc, faces, 2.0, tol=1e-13)
    assert info["levels"] == rinfo.levels == 3
    assert rel_l2(phi, ref) < (1e-10 if precision == "fp64" else 1e-8)


def _bench_settings():
    import json
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    with open(os.path.join(root, "tests", "golden", "oracle_cycles_sphere256.json")) as f:
        return bench.SOLVER, json.load(f)["cycles"]


@pytest.mark.parametrize("settings", ["defaults", "bench"])
def test_full_size_sphere_256_mixed_five_levels(settings):
    p = W.sphere(256)
    g = grid_for(p, "mixed")
    if settings == "bench":
        # the configuration bench.py times; the oracle's own cycle count on this
        # workload with the same settings is stored by tests/golden/make_oracle_cycles.py
        solver, oracle_cycles = _bench_settings()
        g.set_options(**solver)
    info = g.solve(tol=1e-8, levels=5)
    phi = g.potential()
    assert info["levels"] == 5 and info["rel_residual"] <= 1e-8
    if settings == "bench":
        assert info["cycles"] == oracle_cycles
    h = O.spacing(p.shape, p.lo, p.hi)
    f = O.source(p.rho, 1.0, p.bc)
    r = O.residual(phi, f, h, p.bc, p.faces)
    r0 = O.l2norm(O.residual(np.zeros(p.shape), f, h, p.bc, p.faces))
    assert O.l2norm(r) / r0 <= 1.01e-8
    # second-order discretisation error against the analytic sphere, away from the surface
    X, Y, Z = W.mesh(p.shape, p.lo, p.hi)
    rr = np.sqrt(X * X + Y * Y + Z * Z)
    far = rr > 0.5
    assert np.max(np.abs(phi - p.exact)[far]) < 2e-3 * np.max(np.abs(p.exact))


def test_adjoint_matches_oracle_and_finite_differences():
    shape, lo, hi, bc = (16, 16, 16), (0, 0, 0), (1, 1, 1), (0, 0, 0)
    rho = W.random_field(shape, 61)
    faces = W.random_faces(shape, 62)
    w = W.loss_weights(shape, 63)
    p = W.Problem(rho=rho, lo=lo, hi=hi, bc=bc, faces=faces, four_pi_G=3.0)
    g = grid_for(p, "fp64")
    g.solve(tol=1e-13)
    grad, info = g.backward(w, tol=1e-13)
    ref, _ = O.adjoint(w, lo, hi, bc, four_pi_G=3.0, tol=1e-13)
    assert rel_l2(grad, ref) < 1e-10
    eps = 1e-3
    for cell in W.sample_cells(shape, 4, 64):
        vals = []
        for sgn in (1, -1):
            r2 = rho.copy()
            r2[cell] += sgn * eps
            g.set_density(r2, 3.0)
            g.solve(tol=1e-13)
            vals.append(np.sum(w * g.potential()))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - grad[cell]) <= 1e-7 * max(1.0, abs(fd))


def test_autograd_function():
    shape, lo, hi = (16, 16, 16), (0, 0, 0), (1, 1, 1)
    sg = _sg()
    g = sg.Grid(shape, lo, hi, (0, 0, 0), precision="mixed")
    g.set_boundary(W.random_faces(shape, 71))
    g.four_pi_G = 1.0
    rho = torch.tensor(W.random_field(shape, 72), device="cuda", requires_grad=True)
    w = torch.tensor(W.loss_weights(shape, 73), device="cuda")
    phi = sg.solve(rho, g, 1e-11)
    (w * phi).sum().backward()
    ref, _ = O.adjoint(w.cpu().numpy(), lo, hi, (0, 0, 0), four_pi_G=1.0, tol=1e-13)
    assert rel_l2(rho.grad.cpu().numpy(), ref) < 1e-8


def test_batch_equals_individual_solves():
    sg = _sg()
    probs = [W.blobs(n, np.random.default_rng(n)) for n in (32, 64, 32)]
    grids = [grid_for(p, "mixed") for p in probs]
    infos = sg.solve_batch(grids, tol=1e-10)
    for p, g, info in zip(probs, grids, infos):
        assert info["rel_residual"] <= 1e-10
        ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-13)
        assert rel_l2(g.potential(), ref) < 1e-8


def test_errors_are_reported():
    sg = _sg()
    p = W.sphere(32)
    g = grid_for(p, "fp64")
    with pytest.raises(sg.SGError) as e:
        g.solve(tol=1e-8, levels=g.max_levels + 1)
    assert e.value.status == 1
    g.set_options(max_cycles=2)
    info = g.solve(tol=1e-14, check=False)
    assert info["status"] == "SG_ERR_NOT_CONVERGED" and info["cycles"] == 2
    bad = p.rho.copy()
    bad[3, 3, 3] = np.nan
    g.set_density(bad, 1.0)
    info = g.solve(tol=1e-8, check=False)
    assert info["status"] == "SG_ERR_NONFINITE"
    g2 = sg.Grid((8, 8, 8), precision="mixed")
    with pytest.raises(sg.SGError) as e:
        g2.potential()
    assert e.value.status == 7


def test_kernel_profile_counts_every_class():
    p = W.sphere(64)
    g = grid_for(p, "mixed")
    g.set_profiling(True)
    info = g.solve(tol=1e-8, levels=4)
    st = g.kernel_stats()
    g.set_profiling(False)
    for name in ("rkl_stage_l0", "rkl_stage_coarse", "residual_l0", "residual_restrict",
                 "prolong_correct", "bottom_levels", "update_residual"):
        assert st[name]["launches"] > 0 and st[name]["ms"] > 0, name
    # mixed precision: the true FP64 residual at the start and once to confirm
    # convergence; the recurrence update after every cycle; of the three
    # restrictions per cycle (4 levels) the last one runs inside the cluster
    # launch of the two coarsest levels (16^3 and 8^3), which also holds the
    # coarse solve
    assert st["residual_l0"]["launches"] == 2
    assert st["update_residual"]["launches"] == info["cycles"]
    assert st["bottom_levels"]["launches"] == info["cycles"]
    assert st["residual_restrict"]["launches"] == 2 * info["cycles"]
    assert st["coarse_solve"]["launches"] == 0
    # the start (phi = 0: f and the face terms, 20 B/cell) and the confirmation (28 B/cell)
    assert st["residual_l0"]["bytes"] == (20.0 + 28.0) * 64 ** 3
    assert st["update_residual"]["bytes"] == 40.0 * 64 ** 3 * info["cycles"]


def test_batch_graph_matches_individual_solves_exactly():
    # every branch of the batch graph runs the same kernels on the same data as a
    # single solve: results agree to the last bit, cycle counts are equal
    sg = _sg()
    probs = [W.blobs(32, np.random.default_rng(5)), W.blobs(64, np.random.default_rng(6))]
    gp = W.grf(32, seed=7)
    probs.append(gp)
    sin = W.sinusoid(16)
    probs.append(sin)
    anis = W.Problem(rho=W.random_field((8, 4, 6), 8), lo=(0, 0, 0), hi=(1, 1, 1), bc=(0, 0, 0),
                     faces=W.random_faces((8, 4, 6), 9))          # one level: solved on its own
    probs.append(anis)
    precs = ["mixed", "mixed", "mixed", "fp64", "fp64"]
    batch = [grid_for(p, pr) for p, pr in zip(probs, precs)]
    single = [grid_for(p, pr) for p, pr in zip(probs, precs)]
    infos = sg.solve_batch(batch, tol=1e-9)
    for gb, gs, ib in zip(batch, single, infos):
        isg = gs.solve(tol=1e-9)
        assert ib["cycles"] == isg["cycles"]
        np.testing.assert_array_equal(gb.potential(), gs.potential())
    ref, _ = O.solve(gp.rho, gp.lo, gp.hi, gp.bc, None, 1.0, tol=1e-12)
    assert rel_l2(batch[2].potential(), ref) < 1e-8


def test_autotune_keeps_order_and_converges():
    p = W.sphere(64)
    g = grid_for(p, "mixed")
    opts, table = g.autotune(levels=4, keep_order=True)
    assert len(table) > 0 and all(t["rkl_order"] == 2 for t in table)
    best = min(table, key=lambda t: t["ms_per_decade"])
    assert opts["s_smooth"] == best["s_smooth"] and opts["rkl_order"] == 2
    assert (opts["n_pre"], opts["n_post"]) == (best["n_pre"], best["n_post"])
    assert {(t["n_pre"], t["n_post"]) for t in table} == {(2, 1), (3, 2), (4, 3), (5, 3)}
    assert all(0 < t["factor"] <= 1 + 1e-9 for t in table)
    # RKL2 with even s at tau_max does not damp the checkerboard mode, which
    # the coarse grid cannot see: such candidates never converge and score last
    for t in table:
        if t["s_smooth"] % 2 == 0 and t["tau_frac"] == 1.0:
            assert t["factor"] > 0.999
    assert not (opts["s_smooth"] % 2 == 0 and opts["tau_frac"] == 1.0)
    g.set_density(p.rho, 1.0)
    info = g.solve(tol=1e-9, levels=4)
    ref, _ = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-12, levels=4)
    assert rel_l2(g.potential(), ref) < 1e-7
    assert info["rel_residual"] <= 1e-9


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_device_loop_host_loop_and_direct_launches_agree(precision):
    # use_graph = 1: the cycle loop in the solve graph's WHILE nodes; 2: one graph
    # per cycle, the loop on the host; 0: no graph.  Same kernels, same order:
    # identical potentials, cycle counts, histories and coarse super-step counts.
    p = W.sphere(64)
    out = {}
    for mode in (1, 2, 0):
        g = grid_for(p, precision, use_graph=mode)
        info = g.solve(tol=1e-9, levels=4)
        out[mode] = (g.potential(), info)
    for mode in (2, 0):
        np.testing.assert_array_equal(out[mode][0], out[1][0])
        for k in ("cycles", "history", "coarse_ss", "rel_residual", "stage_cell_updates"):
            assert out[mode][1][k] == out[1][1][k], (mode, k)
    assert out[1][1]["rel_residual"] <= 1e-9


def test_device_loop_reports_the_cycle_cap_and_fixed_counts():
    p = W.sphere(32)
    g = grid_for(p, "mixed", max_cycles=3)
    info = g.solve(tol=1e-14, levels=4, check=False)
    assert info["status"] == "SG_ERR_NOT_CONVERGED" and info["cycles"] == 3
    g.set_options(max_cycles=100, fixed_cycles=5)
    g.set_density(p.rho, 1.0)
    info = g.solve(tol=0.0, levels=4)
    assert info["status"] == "SG_OK" and info["cycles"] == 5 and len(info["history"]) == 6


@pytest.mark.parametrize("inner", [(2, 1), (0, 1)])
def test_inner_level_smoothing_counts_match_oracle(inner):
    # levels 1 .. L-2 smooth inner_n_pre / inner_n_post times (level 0 keeps
    # N_pre / N_post): the FP64 solve against the oracle for the same cycles
    p = W.sphere(64)
    kw = dict(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, coarse_tol=0.0, coarse_max_ss=12,
              fixed_cycles=4, inner_n_pre=inner[0], inner_n_post=inner[1])
    g = grid_for(p, "fp64", **kw)
    info = g.solve(tol=0.0, levels=4)
    opts = O.Options(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, coarse_tol=0.0, coarse_max_ss=12,
                     inner_n_pre=inner[0], inner_n_post=inner[1])
    ref, rinfo = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, levels=4, opts=opts, cycles=4)
    assert info["cycles"] == 4
    assert rel_l2(g.potential(), ref) < 1e-12
    np.testing.assert_allclose(info["history"], rinfo.history, rtol=1e-9, atol=1e-14)
    # mixed precision with the cluster launch of the two coarsest levels (level
    # B smooths with the inner counts there too): the oracle's cycle count
    gm = grid_for(p, "mixed", rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3,
                  inner_n_pre=inner[0], inner_n_post=inner[1])
    im = gm.solve(tol=1e-9, levels=4)
    opts_m = O.Options(rkl_order=2, s_smooth=3, tau_frac=0.9, n_pre=5, n_post=3, inner_n_pre=inner[0],
                       inner_n_post=inner[1])
    _, rm = O.solve(p.rho, p.lo, p.hi, p.bc, p.faces, 1.0, tol=1e-9, levels=4, opts=opts_m)
    assert abs(im["cycles"] - rm.cycles) <= 1


@pytest.mark.parametrize("shape", [(48, 40, 36), (33, 21, 17)])
def test_pinned_host_buffers_move_over_the_link_bit_exactly(shape):
    # pinned (mapped) host buffers moved by copy engines (the default) or read
    # and written by kernels over the CPU-GPU link (host_copy = "kernel");
    # pageable ones by copy-engine transfers: the same bits (an odd cell
    # count takes the kernels' scalar path)
    sg = _sg()
    rng = np.random.default_rng(7)
    rho = rng.standard_normal(shape)
    faces = W.random_faces(shape, 8)
    out = {}
    for kind in ("pageable", "pinned", "pinned_engine"):
        g = sg.Grid(shape, (0, 0, 0), (1, 1, 1), (0, 0, 0), precision="mixed")
        g.set_options(host_copy="kernel" if kind == "pinned" else "engine")
        assert g.options().host_copy == (1 if kind == "pinned" else 0)
        g.set_boundary(faces)
        src = rho if kind == "pageable" else torch.from_numpy(rho).pin_memory()
        g.set_density(src, 3.0)
        info = g.solve(tol=1e-9)
        assert info["rel_residual"] <= 1e-9
        phi = np.empty(shape) if kind == "pageable" else torch.empty(shape, dtype=torch.float64).pin_memory()
        g.potential(phi)
        grav = np.empty((3,) + shape) if kind == "pageable" else torch.empty((3,) + shape, dtype=torch.float64).pin_memory()
        g.gravity(out=grav)
        out[kind] = (np.asarray(phi).copy(), np.asarray(grav).copy(), info["cycles"])
        del g
    for kind in ("pinned", "pinned_engine"):
        assert out[kind][2] == out["pageable"][2]
        assert np.array_equal(out[kind][0], out["pageable"][0])
        assert np.array_equal(out[kind][1], out["pageable"][1])
    assert np.abs(out["pinned"][0]).max() > 0


def test_grids_solved_from_several_threads_match_one_at_a_time():
    # independent grids, each created on its own stream and driven by its own
    # host thread (the library's calls release the interpreter lock; shapes
    # whose plans no other test made, so the threads fill the plan cache), give
    # the same bits as the same solves one at a time
    import threading
    sg = _sg()
    shapes = [(40, 48, 36), (56, 40, 44), (36, 52, 60), (44, 36, 52)]
    rng = np.random.default_rng(31)
    rhos = [rng.standard_normal(s) for s in shapes]

    def run(i, out):
        st = torch.cuda.Stream()
        g = sg.Grid(shapes[i], (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (0, 0, 0), precision="mixed",
                    stream=st.cuda_stream)
        g.set_options(rkl_order=2, s_smooth=3, n_pre=5, n_post=3)
        g.set_density(rhos[i], 1.0)
        info = g.solve(tol=1e-9)
        out[i] = (g.potential(), info["cycles"], info["rel_residual"])

    together = {}
    threads = [threading.Thread(target=run, args=(i, together)) for i in range(len(shapes))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    alone = {}
    for i in range(len(shapes)):
        run(i, alone)
    for i in range(len(shapes)):
        assert together[i][1] == alone[i][1] and together[i][2] <= 1e-9
        assert np.array_equal(together[i][0], alone[i][0])
