"""The two coarsest levels of the FP32 V-cycle in one cluster launch against
the level-by-level kernels (the `fused` option switches between them), on
every boundary mix and on the cluster sizes the planner picks (16 where the
device schedules clusters of 16, else 8; 8, 4 and 2 CTAs; level B of 32^3,
32 x 16 x 16, 16^3, 8^3, 24^3 and 24 x 16 x 12 cells; a valid
hierarchy has an even coarsest level, so level B always splits in two), and
the fallback to the level-by-level kernels where the coarsest level's x extent
is not a multiple of four.

Both paths evaluate the same formulas in the same order (RKL stages, residual,
8-child restriction, periodic mean, accelerated RKL1 coarse solve with its
tolerance stop, 27/9/3/1 prolongation), so after two cycles the potentials
agree to FP32 rounding (tolerance 1e-5 relative; a wrong ghost or coefficient
gives differences of 1e-3 and more).  The solve with the cluster launch is
also checked against the FP64 oracle's solution.
"""

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


LO, HI = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)

# (shape (nz, ny, nx), bc, levels): level B = levels - 2
CASES = [
    ((128, 128, 128), (0, 0, 0), 4),   # B 32^3, 16 CTAs of 2 planes (the benchmark's level B)
    ((128, 64, 64), (1, 1, 1), 4),     # B 32 x 16 x 16, 16 CTAs, the z wrap between the end CTAs
    ((64, 64, 64), (0, 0, 0), 4),      # B 16^3, 8 CTAs of 2 planes
    ((32, 32, 32), (1, 1, 1), 4),      # B 8^3, 4 CTAs, coarse mean removed
    ((48, 48, 48), (1, 0, 1), 3),      # B 24^3, 4 CTAs, 3 strips per coarse row
    ((24, 32, 48), (0, 1, 0), 3),      # B 12 x 16 x 24 (z, y, x), 2 CTAs of 6 planes
]


def _run(shape, bc, levels, fused, opts, cycles=2, prof=False):
    sg = _sg()
    g = sg.Grid(shape, LO, HI, bc, precision="mixed")
    if any(b == 0 for b in bc):
        g.set_boundary(W.random_faces(shape, 3))
    rho = W.random_field(shape, 4)
    if all(b == 1 for b in bc):
        rho = rho - rho.mean()
    g.set_density(rho, 1.0)
    g.set_options(fused=fused, fixed_cycles=cycles, **opts)
    if prof:
        g.set_profiling(True)
    info = g.solve(tol=0.0, levels=levels, check=False)
    stats = g.kernel_stats() if prof else None
    return g.potential(), info, stats


@pytest.mark.parametrize("shape,bc,levels", CASES)
@pytest.mark.parametrize("opts", [dict(rkl_order=2, s_smooth=3),
                                  dict(rkl_order=1, s_smooth=2, tau_frac=0.75, n_pre=1, n_post=2)])
def test_cluster_launch_matches_level_by_level(shape, bc, levels, opts):
    a, ia, st = _run(shape, bc, levels, 1, opts, prof=True)
    b, ib, _ = _run(shape, bc, levels, 0, opts)
    assert st["bottom_levels"]["launches"] == 2
    assert st["coarse_solve"]["launches"] == 0
    assert np.all(np.isfinite(a))
    if all(x == 1 for x in bc):
        a, b = a - a.mean(), b - b.mean()
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5
    assert ia["coarse_ss"] == ib["coarse_ss"]


def test_unsupported_shape_falls_back_to_level_by_level():
    # level C of 10 x 6 x 18 (x extent not a multiple of four)
    shape, bc, levels = (40, 24, 72), (0, 1, 0), 3
    opts = dict(rkl_order=2, s_smooth=3)
    a, _, st = _run(shape, bc, levels, 1, opts, prof=True)
    b, _, _ = _run(shape, bc, levels, 0, opts)
    assert st["bottom_levels"]["launches"] == 0
    assert st["coarse_solve"]["launches"] == 2
    assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-5


def test_cluster_path_solve_matches_oracle():
    sg = _sg()
    shape, bc, levels = (64, 64, 64), (0, 1, 0), 4
    faces = W.random_faces(shape, 7)
    rho = W.random_field(shape, 8)
    g = sg.Grid(shape, LO, HI, bc, precision="mixed")
    g.set_boundary(faces)
    g.set_density(rho, 1.0)
    g.set_profiling(True)
    info = g.solve(tol=1e-11, levels=levels)
    assert g.kernel_stats()["bottom_levels"]["launches"] == info["cycles"]
    ref, _ = O.solve(rho, LO, HI, bc, faces, 1.0, tol=1e-13, levels=levels)
    assert np.linalg.norm(g.potential() - ref) / np.linalg.norm(ref) < 1e-8
