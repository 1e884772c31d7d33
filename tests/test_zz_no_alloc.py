"""The allocation-free residual entry point (sg_residual_restrict_noalloc)
against the grid-based sg_op_residual_restrict on the same inputs.

Both run the same residual / residual-restrict and norm-fold kernels; the
allocation-free one keeps the per-block partial norms in a static device
array instead of the grid's buffers.  Calls in a row must each match, so a
call is not disturbed by what the previous one left in the shared array.
This file is collected last so that it also runs after every other GPU test
in one process; it passes alone in a fresh process as well.

Tolerances are those of the operator tests: 1e-12 relative for FP64, 2e-5
for FP32 (same kernels, so in practice the results are identical).
"""

import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-12, "mixed": 2e-5}
LO, HI = (0.0, -0.5, 0.25), (1.3, 0.2, 1.35)


def _sg():
    import paper_2306_05332_gb300 as sg
    return sg


def _case(shape, bc, precision, seed):
    sg = _sg()
    dt = torch.float64 if precision == "fp64" else torch.float32
    g = sg.Grid(shape, LO, HI, bc, precision=precision)
    faces_dev = None
    if any(b == 0 for b in bc):
        faces = W.random_faces(shape, seed)
        g.set_boundary(faces)
        faces_dev = [torch.as_tensor(np.ascontiguousarray(f), dtype=torch.float64, device="cuda") for f in faces]
    u = torch.as_tensor(W.random_field(shape, seed + 1), dtype=dt, device="cuda")
    rhs = torch.as_tensor(50.0 * W.random_field(shape, seed + 2), dtype=dt, device="cuda")
    return g, faces_dev, u, rhs, dt


def _relerr(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _compare_once(shape, bc, precision, with_coarse, seed):
    sg = _sg()
    g, faces_dev, u, rhs, dt = _case(shape, bc, precision, seed)
    cshape = tuple(n // 2 for n in shape)
    ca = torch.full(cshape, float("nan"), dtype=dt, device="cuda") if with_coarse else None
    cb = torch.full(cshape, float("nan"), dtype=dt, device="cuda") if with_coarse else None
    na = g.op_residual_restrict(0, u, rhs, ca)
    nb = sg.residual_restrict_noalloc(shape, LO, HI, bc, u, rhs, cb, faces=faces_dev)
    torch.cuda.synchronize()
    tol = TOL[precision]
    assert abs(nb[0] - na[0]) <= tol * abs(na[0])
    assert abs(nb[1] - na[1]) <= tol * abs(na[1])
    if with_coarse:
        assert torch.isfinite(cb).all()
        assert _relerr(cb, ca) <= tol
    # and against the oracle's definition (r = rhs - L u, 8-cell mean)
    h = O.spacing(shape, LO, HI)
    faces_np = None if faces_dev is None else [f.cpu().numpy() for f in faces_dev]
    r = -O.residual(u.double().cpu().numpy(), rhs.double().cpu().numpy(), h, bc, faces_np)
    assert abs(nb[0] - np.sum(r ** 2)) <= (1e-12 if precision == "fp64" else 1e-4) * np.sum(r ** 2)
    return nb


@pytest.mark.gpu
def test_two_calls_in_a_row_match_the_grid_entry_point():
    # first: FP64, Dirichlet faces, restriction + norms; second: FP32, periodic,
    # another shape, norms only; third: FP32 with faces and restriction
    _compare_once((20, 12, 36), (0, 0, 0), "fp64", True, 40)
    _compare_once((16, 24, 8), (1, 1, 1), "mixed", False, 50)
    _compare_once((12, 20, 40), (1, 0, 1), "mixed", True, 60)


@pytest.mark.gpu
def test_repeated_call_matches_and_allocates_nothing():
    sg = _sg()
    shape, bc = (64, 48, 80), (0, 0, 0)
    first = _compare_once(shape, bc, "fp64", True, 70)
    g, faces_dev, u, rhs, dt = _case(shape, bc, "fp64", 70)
    coarse = torch.empty(tuple(n // 2 for n in shape), dtype=dt, device="cuda")
    sg.residual_restrict_noalloc(shape, LO, HI, bc, u, rhs, coarse, faces=faces_dev)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = sg.residual_restrict_noalloc(shape, LO, HI, bc, u, rhs, coarse, faces=faces_dev)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert again == first


@pytest.mark.gpu
def test_full_size_256_cube():
    # the 256^3 sphere workload's level 0 (2560 of the 8192 block slots)
    sg = _sg()
    p = W.sphere(256)
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="fp64")
    g.set_boundary(p.faces)
    faces_dev = [torch.as_tensor(np.ascontiguousarray(f), device="cuda") for f in p.faces]
    u = torch.zeros(p.shape, dtype=torch.float64, device="cuda")
    rhs = torch.as_tensor(p.rho, device="cuda")
    ca = torch.empty(tuple(n // 2 for n in p.shape), dtype=torch.float64, device="cuda")
    cb = torch.empty_like(ca)
    na = g.op_residual_restrict(0, u, rhs, ca)
    nb = sg.residual_restrict_noalloc(p.shape, p.lo, p.hi, p.bc, u, rhs, cb, faces=faces_dev)
    assert abs(nb[0] - na[0]) <= 1e-12 * na[0] and nb[1] == na[1]
    assert _relerr(cb, ca) <= 1e-12


# Argument errors return before any CUDA call (the fake pointers below are
# never dereferenced), so these run without a GPU.
def _raw(shape, coarse=True, norms=True, dtype=0, bc=(0, 0, 0)):
    sg = _sg()
    nz, ny, nx = shape
    D3, I3 = ctypes.c_double * 3, ctypes.c_int * 3
    out = (ctypes.c_double * 2)() if norms else None
    fake = ctypes.c_void_p(256)
    return sg.lib().sg_residual_restrict_noalloc(nx, ny, nz, D3(0, 0, 0), D3(1, 1, 1), I3(*bc), None, dtype,
                                                 fake, fake, fake if coarse else None, out, None)


def test_rejects_grids_beyond_the_static_scratch():
    sg = _sg()
    # 4096 x 1024 x 2: ceil(4096/32) * ceil(1024/8) = 16384 blocks > 8192 slots
    assert _raw((2, 1024, 4096)) == 1
    msg = sg.lib().sg_last_error().decode()
    assert "16384" in msg and "8192" in msg


def test_rejects_bad_arguments():
    assert _raw((8, 8, 7)) == 1                      # restriction of an odd size
    assert _raw((8, 8, 8), coarse=False, norms=False) == 1
    assert _raw((8, 8, 8), dtype=2) == 1
    assert _raw((8, 8, 1)) == 1
    assert _raw((8, 8, 8), bc=(0, 3, 0)) == 1


@pytest.mark.gpu
def test_binding_rejects_arrays_of_the_wrong_shape():
    # the kernels take bare pointers: the binding checks every array against the
    # stated shape before the call, so a short buffer is never written past
    sg = _sg()
    shape, bc = (8, 8, 8), (0, 0, 0)
    u = torch.zeros(shape, dtype=torch.float64, device="cuda")
    rhs = torch.zeros(shape, dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        sg.residual_restrict_noalloc((8, 8, 16), LO, HI, bc, u, rhs, None)
    with pytest.raises(ValueError):
        sg.residual_restrict_noalloc(shape, LO, HI, bc, u, rhs, torch.zeros((4, 4, 2), dtype=torch.float64,
                                                                            device="cuda"))
    faces = [torch.zeros((8, 8), dtype=torch.float64, device="cuda") for _ in range(6)]
    faces[4] = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        sg.residual_restrict_noalloc(shape, LO, HI, bc, u, rhs, None, faces=faces)
