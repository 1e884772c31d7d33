"""GB300-native RKL-multigrid Poisson solver (thin Python binding).

Every step of the solve runs in the CUDA kernels of ``lib/libsg.so`` (built
from ``csrc/`` by ``python -m paper_2306_05332_gb300.build``); this module only
marshals arguments to the C ABI declared in ``include/sg.h``.  There is no CPU
fallback: if the library is missing, importing the binding's entry points
raises.

Arrays are C-contiguous float64 ``[nz][ny][nx]``.  A numpy array (or a CPU
tensor) is passed as host memory; a CUDA tensor as device memory on the grid's
stream (by default ``torch.cuda.current_stream()``).

>>> g = Grid((256, 256, 256), lo=(-1, -1, -1), hi=(1, 1, 1), precision="mixed")
>>> g.set_boundary(faces); g.set_density(rho, four_pi_G=1.0)
>>> info = g.solve(tol=1e-8, levels=5)
>>> phi = g.potential()
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as LIB_PATH

__all__ = ["Grid", "Grid2D", "SGError", "Options", "SolveInfo", "lib", "solve", "PoissonSolve",
           "DIRICHLET", "PERIODIC", "FP64", "MIXED", "default_options", "exported_symbols"]

DIRICHLET, PERIODIC = 0, 1
FP64, MIXED = 0, 1
SG_MAX_HISTORY = 256

STATUS = {0: "SG_OK", 1: "SG_ERR_ARG", 2: "SG_ERR_CUDA", 3: "SG_ERR_OOM", 4: "SG_ERR_NOT_CONVERGED",
          5: "SG_ERR_TIMEOUT", 6: "SG_ERR_NONFINITE", 7: "SG_ERR_STATE"}


class Options(ctypes.Structure):
    _fields_ = [("rkl_order", ctypes.c_int), ("s_smooth", ctypes.c_int), ("tau_frac", ctypes.c_double),
                ("n_pre", ctypes.c_int), ("n_post", ctypes.c_int), ("coarse_tol", ctypes.c_double),
                ("coarse_max_ss", ctypes.c_int), ("coarse_tau_frac", ctypes.c_double),
                ("max_cycles", ctypes.c_int), ("single_s", ctypes.c_int),
                ("single_tau_frac", ctypes.c_double), ("fixed_cycles", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("fused", ctypes.c_int), ("smoother", ctypes.c_int),
                ("omega", ctypes.c_double), ("max_residual_tol", ctypes.c_double), ("tile_rows", ctypes.c_int),
                ("inner_n_pre", ctypes.c_int), ("inner_n_post", ctypes.c_int), ("staging", ctypes.c_int),
                ("host_copy", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("cycles", ctypes.c_int), ("levels", ctypes.c_int),
                ("s_smooth", ctypes.c_int), ("rkl_order", ctypes.c_int), ("precision", ctypes.c_int),
                ("r0", ctypes.c_double), ("rel_residual", ctypes.c_double),
                ("max_residual", ctypes.c_double), ("history", ctypes.c_double * SG_MAX_HISTORY),
                ("coarse_ss", ctypes.c_int * SG_MAX_HISTORY), ("elapsed_ms", ctypes.c_double),
                ("stage_cell_updates", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong)]

    def as_dict(self):
        n = self.cycles
        return {"status": STATUS.get(self.status, self.status), "cycles": n, "levels": self.levels,
                "s_smooth": self.s_smooth, "rkl_order": self.rkl_order, "precision": self.precision,
                "r0": self.r0, "rel_residual": self.rel_residual, "max_residual": self.max_residual,
                "history": list(self.history[:min(n + 1, SG_MAX_HISTORY)]),
                "coarse_ss": list(self.coarse_ss[:min(n, SG_MAX_HISTORY)]),
                "elapsed_ms": self.elapsed_ms, "stage_cell_updates": self.stage_cell_updates,
                "kernel_launches": self.kernel_launches}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double)]


SG_KERNEL_CLASSES = 11
SMOOTHERS = {"rkl": 0, "gsrb": 1}
STAGINGS = {"cp_async": 0, "tma": 1}
HOST_COPIES = {"engine": 0, "kernel": 1}     # sg_host_copy


class TuneEntry(ctypes.Structure):
    _fields_ = [("rkl_order", ctypes.c_int), ("s_smooth", ctypes.c_int), ("fused", ctypes.c_int),
                ("tau_frac", ctypes.c_double), ("ms_per_cycle", ctypes.c_double), ("factor", ctypes.c_double),
                ("ms_per_decade", ctypes.c_double), ("n_pre", ctypes.c_int), ("n_post", ctypes.c_int),
                ("tile_rows", ctypes.c_int), ("inner_n_pre", ctypes.c_int), ("inner_n_post", ctypes.c_int)]


class SGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_LIB = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "sg_default_options": ([ctypes.POINTER(Options)], _I),
    "sg_create_grid": ([_I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I), _I, _P,
                        ctypes.POINTER(_P)], _I),
    "sg_create_grid_2d": ([_I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I), _I, _P,
                           ctypes.POINTER(_P)], _I),
    "sg_set_options": ([_P, ctypes.POINTER(Options)], _I),
    "sg_get_options": ([_P, ctypes.POINTER(Options)], _I),
    "sg_set_boundary": ([_P, ctypes.POINTER(_P), _I], _I),
    "sg_set_density": ([_P, _P, _I, _D], _I),
    "sg_set_potential_guess": ([_P, _P, _I], _I),
    "sg_solve": ([_P, _D, _I, _I, ctypes.POINTER(SolveInfo)], _I),
    "sg_potential": ([_P, _P, _I], _I),
    "sg_gravity": ([_P, _P, _P, _I], _I),
    "sg_backward": ([_P, _P, _P, _I, _D, ctypes.POINTER(SolveInfo)], _I),
    "sg_solve_batch": ([ctypes.POINTER(_P), _I, _D, ctypes.POINTER(SolveInfo)], _I),
    "sg_destroy": ([_P], None),
    "sg_last_error": ([], ctypes.c_char_p),
    "sg_max_levels": ([_P], _I),
    "sg_op_superstep": ([_P, _I, _I, _I, _I, _D, _I, _P, _P, _P], _I),
    "sg_op_gsrb_sweep": ([_P, _I, _I, _I, _D, _P, _P], _I),
    "sg_op_residual_restrict": ([_P, _I, _I, _I, _P, _P, _P, ctypes.POINTER(_D)], _I),
    "sg_op_residual_exact": ([_P, _I, _P, _P, _P, _P, ctypes.POINTER(_D)], _I),
    "sg_op_prolong_correct": ([_P, _I, _I, _P, _P], _I),
    "sg_op_coarse_solve": ([_P, _I, _I, _P, _P, ctypes.POINTER(_I)], _I),
    "sg_set_profiling": ([_P, _I], _I),
    "sg_kernel_stats": ([_P, ctypes.POINTER(KernelStat)], _I),
    "sg_autotune": ([_P, _I, _I, ctypes.POINTER(TuneEntry), _I, ctypes.POINTER(_I)], _I),
    "sg_plan_schedule": ([_I, _I, ctypes.POINTER(_I)], _I),
    "sg_plan_stage_coefficients": ([_I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                    ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "sg_plan_levels": ([_I, _I, _I], _I),
    "sg_plan_s_opt": ([_I, ctypes.POINTER(_I)], _I),
    "sg_measure_fp64_rate": ([ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "sg_plan_sor_omega": ([_I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D)], _I),
    "sg_residual_restrict_noalloc": ([_I, _I, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_I),
                                      ctypes.POINTER(_P), _I, _P, _P, _P, ctypes.POINTER(_D), _P], _I),
}


def exported_symbols():
    """Names of the C ABI entry points this binding declares."""
    return sorted(_SIGS)


def lib():
    """Load libsg.so (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2306_05332_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(status):
    if status != 0:
        raise SGError(status, lib().sg_last_error().decode())


def default_options():
    o = Options()
    _check(lib().sg_default_options(ctypes.byref(o)))
    return o


def _torch():
    try:
        import torch
        return torch
    except ImportError:        # pragma: no cover - torch is optional for host arrays
        return None


def _ptr(a, dtype=np.float64):
    """(pointer, on_device, keepalive) of a contiguous array / tensor."""
    torch = _torch()
    if torch is not None and isinstance(a, torch.Tensor):
        want = torch.float64 if dtype == np.float64 else torch.float32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return ctypes.c_void_p(a.data_ptr()), int(a.is_cuda), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), 0, arr


def _require_writable(out):
    if isinstance(out, np.ndarray) and (out.dtype != np.float64 or not out.flags.c_contiguous):
        raise TypeError("out must be a C-contiguous float64 array")


def _dev_ptr(t, dtype, shape=None, device=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype code
    (0: float64, 1: float32).  With `shape` / `device` the tensor must have
    exactly that shape and sit on that device: the kernels take bare pointers
    and would read or write past a smaller buffer."""
    torch = _torch()
    if torch is None or not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("operator entry points take CUDA tensors")
    want = torch.float64 if dtype == 0 else torch.float32
    if t.dtype != want or not t.is_contiguous():
        raise TypeError(f"tensor must be contiguous {want}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"tensor has shape {tuple(t.shape)}, expected {tuple(shape)}")
    if device is not None and t.device != device:
        raise ValueError(f"tensor is on {t.device}, expected {device}")
    return ctypes.c_void_p(t.data_ptr())


class Grid:
    """One solver grid: shape (nz, ny, nx) on the box [lo, hi] (x, y, z order)."""

    def __init__(self, shape, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), bc=(DIRICHLET,) * 3,
                 precision="mixed", stream=None):
        nz, ny, nx = (int(v) for v in shape)
        self.shape = (nz, ny, nx)
        self.lo, self.hi, self.bc = tuple(lo), tuple(hi), tuple(int(b) for b in bc)
        self.precision = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}[precision]
        if stream is None:
            torch = _torch()
            stream = torch.cuda.current_stream().cuda_stream if (torch and torch.cuda.is_available()) else 0
        self.stream = int(stream)
        torch = _torch()
        self.device = (torch.device("cuda", torch.cuda.current_device())
                       if (torch and torch.cuda.is_available()) else None)
        h = ctypes.c_void_p()
        _check(lib().sg_create_grid(nx, ny, nz, (_D * 3)(*self.lo), (_D * 3)(*self.hi), (_I * 3)(*self.bc),
                                    self.precision, ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self._h = h
        self.four_pi_G = 1.0

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _LIB is not None:
            _LIB.sg_destroy(h)
            self._h = None

    close = __del__

    @property
    def handle(self):
        return self._h

    @property
    def max_levels(self):
        return lib().sg_max_levels(self._h)

    def options(self):
        o = Options()
        _check(lib().sg_get_options(self._h, ctypes.byref(o)))
        return o

    def set_options(self, **kw):
        o = self.options()
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            if k == "smoother" and isinstance(v, str):
                v = SMOOTHERS[v]
            if k == "staging" and isinstance(v, str):
                v = STAGINGS[v]
            if k == "host_copy" and isinstance(v, str):
                v = HOST_COPIES[v]
            setattr(o, k, v)
        _check(lib().sg_set_options(self._h, ctypes.byref(o)))
        return o

    def set_boundary(self, faces):
        ptrs, keep, on_dev = [], [], 0
        for f in faces:
            if f is None:
                ptrs.append(None)
                continue
            p, d, k = _ptr(f)
            ptrs.append(p.value)
            keep.append(k)
            on_dev = d
        arr = (ctypes.c_void_p * 6)(*ptrs)
        _check(lib().sg_set_boundary(self._h, arr, on_dev))

    def set_density(self, rho, four_pi_G=1.0):
        p, d, keep = _ptr(rho)
        _check(lib().sg_set_density(self._h, p, d, float(four_pi_G)))
        self.four_pi_G = float(four_pi_G)

    def set_guess(self, phi):
        p, d, keep = _ptr(phi)
        _check(lib().sg_set_potential_guess(self._h, p, d))

    def solve(self, tol=1e-10, s=0, levels=0, check=True):
        info = SolveInfo()
        st = lib().sg_solve(self._h, float(tol), int(s), int(levels), ctypes.byref(info))
        if check and st not in (0,):
            _check(st)
        return info.as_dict()

    def gravity(self, out=None, phi=None):
        """g = -grad phi to fourth order (Sec. 3) as an array (3, nz, ny, nx):
        of the last solve's potential, or of `phi`.  `out` (numpy float64 or a
        CUDA float64 tensor of that shape) receives it when given; with a CUDA
        `out`, `phi` (if any) must be a CUDA tensor too."""
        if out is None:
            out = np.empty((3,) + tuple(self.shape), dtype=np.float64)
        _require_writable(out)
        po, do, keep_o = _ptr(out)
        pp, keep_p = None, None
        if phi is not None:
            pp, dp, keep_p = _ptr(phi)
            if dp != do:
                raise TypeError("phi and out must both be host arrays or both CUDA tensors")
        _check(lib().sg_gravity(self._h, pp, po, do))
        return out

    def potential(self, out=None):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        _require_writable(out)
        p, d, keep = _ptr(out)
        _check(lib().sg_potential(self._h, p, d))
        return out

    def backward(self, dL_dphi, out=None, tol=1e-10, check=True):
        if out is None:
            out = np.empty(self.shape, dtype=np.float64)
        _require_writable(out)
        pi, di, ki = _ptr(dL_dphi)
        po, do, ko = _ptr(out)
        if di != do:
            raise TypeError("dL_dphi and out must both be host or both be device memory")
        info = SolveInfo()
        st = lib().sg_backward(self._h, pi, po, di, float(tol), ctypes.byref(info))
        if check and st != 0:
            _check(st)
        return out, info.as_dict()

    def set_profiling(self, on=True):
        _check(lib().sg_set_profiling(self._h, int(bool(on))))

    def autotune(self, levels=0, keep_order=True):
        """Measure the smoother candidates and keep the fastest per residual decade."""
        cap = 1024
        arr = (TuneEntry * cap)()
        n = ctypes.c_int(0)
        _check(lib().sg_autotune(self._h, int(levels), int(bool(keep_order)), arr, cap, ctypes.byref(n)))
        table = [{k: getattr(arr[i], k) for k, _ in TuneEntry._fields_} for i in range(min(n.value, cap))]
        return self.options().as_dict(), table

    def kernel_stats(self):
        arr = (KernelStat * SG_KERNEL_CLASSES)()
        _check(lib().sg_kernel_stats(self._h, arr))
        return {a.name.decode(): {"launches": a.launches, "ms": a.ms, "bytes": a.bytes} for a in arr}

    # ---- single operators (CUDA tensors of the grid's working precision) ----
    @property
    def dtype_code(self):
        return 0 if self.precision == FP64 else 1

    def level_shape(self, level):
        """(nz, ny, nx) of multigrid level `level` (each axis halved per level)."""
        if not 0 <= int(level) < self.max_levels:
            raise ValueError(f"level {level} out of range [0, {self.max_levels})")
        return tuple(n >> int(level) for n in self.shape)

    def _op(self, t, level):
        """Pointer of an operator argument: the level's shape, the grid's dtype and device."""
        return _dev_ptr(t, self.dtype_code, self.level_shape(level), self.device)

    def op_superstep(self, level, order, s, tau_frac, u, rhs, out, homogeneous=False):
        """out = one RKL super-step from u (None: u = 0, fused FP32 path only)."""
        dt = self.dtype_code
        with _device_of(self.device):
            _check(lib().sg_op_superstep(self._h, level, dt, order, s, float(tau_frac), int(homogeneous),
                                         self._op(u, level) if u is not None else None, self._op(rhs, level),
                                         self._op(out, level)))

    def op_gsrb_sweep(self, level, u, rhs, omega=1.0, homogeneous=False):
        """One red-black Gauss-Seidel / SOR sweep of L u = rhs, in place on u."""
        dt = self.dtype_code
        with _device_of(self.device):
            _check(lib().sg_op_gsrb_sweep(self._h, level, dt, int(homogeneous), float(omega),
                                          self._op(u, level), self._op(rhs, level)))

    def op_residual_restrict(self, level, u, rhs, coarse_out=None, homogeneous=False):
        dt = self.dtype_code
        norms = (_D * 2)()
        cp = None
        if coarse_out is not None:
            cshape = tuple(n // 2 for n in self.level_shape(level))
            cp = _dev_ptr(coarse_out, dt, cshape, self.device)
        with _device_of(self.device):
            _check(lib().sg_op_residual_restrict(self._h, level, dt, int(homogeneous), self._op(u, level),
                                                 self._op(rhs, level), cp, norms))
        return norms[0], norms[1]

    def op_residual_exact(self, u, rhs, r_out, r32_out, homogeneous=False):
        """FP64 residual of level 0 with the neighbour sum in exact fixed point (FP64 u, rhs, r_out; FP32 r32_out)."""
        shape = self.level_shape(0)
        norms = (_D * 2)()
        with _device_of(self.device):
            _check(lib().sg_op_residual_exact(self._h, int(homogeneous), _dev_ptr(u, 0, shape, self.device),
                                              _dev_ptr(rhs, 0, shape, self.device),
                                              _dev_ptr(r_out, 0, shape, self.device),
                                              _dev_ptr(r32_out, 1, shape, self.device), norms))
        return norms[0], norms[1]

    def op_prolong_correct(self, level, coarse, fine):
        dt = self.dtype_code
        with _device_of(self.device):
            _check(lib().sg_op_prolong_correct(self._h, level, dt, self._op(coarse, level + 1),
                                               self._op(fine, level)))

    def op_coarse_solve(self, level, rhs, out):
        dt = self.dtype_code
        done = ctypes.c_int(0)
        with _device_of(self.device):
            _check(lib().sg_op_coarse_solve(self._h, level, dt, self._op(rhs, level), self._op(out, level),
                                            ctypes.byref(done)))
        return done.value


class Grid2D(Grid):
    """A two-dimensional grid (Sec. 2.2's 2D variants: five-point operator,
    4-cell restriction, 9/3/3/1 prolongation): shape (ny, nx) on the rectangle
    [lo, hi] (x, y order), bc = (x, y).  Arrays are (ny, nx); set_boundary takes
    the four faces -x, +x (length ny) and -y, +y (length nx); gravity returns
    (3, ny, nx) with a zero z component."""

    def __init__(self, shape, lo=(0.0, 0.0), hi=(1.0, 1.0), bc=(DIRICHLET, DIRICHLET), precision="mixed",
                 stream=None):
        ny, nx = (int(v) for v in shape)
        self.shape = (ny, nx)
        self.lo, self.hi, self.bc = tuple(lo), tuple(hi), tuple(int(b) for b in bc)
        self.precision = {"fp64": FP64, "mixed": MIXED, FP64: FP64, MIXED: MIXED}[precision]
        torch = _torch()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream if (torch and torch.cuda.is_available()) else 0
        self.stream = int(stream)
        self.device = (torch.device("cuda", torch.cuda.current_device())
                       if (torch and torch.cuda.is_available()) else None)
        h = ctypes.c_void_p()
        _check(lib().sg_create_grid_2d(nx, ny, (_D * 2)(*self.lo), (_D * 2)(*self.hi), (_I * 2)(*self.bc),
                                       self.precision, ctypes.c_void_p(self.stream), ctypes.byref(h)))
        self._h = h
        self.four_pi_G = 1.0

    def set_boundary(self, faces):
        faces = list(faces)
        if len(faces) != 4:
            raise ValueError("a 2D grid takes four faces: -x, +x, -y, +y")
        ny, nx = self.shape
        for f, n in zip(faces, (ny, ny, nx, nx)):
            if f is not None and np.asarray(f).size != n:
                raise ValueError(f"face of {np.asarray(f).size} values, expected {n}")
        super().set_boundary(faces + [None, None])

    def level_shape(self, level):
        if not 0 <= int(level) < self.max_levels:
            raise ValueError(f"level {level} out of range [0, {self.max_levels})")
        return tuple(n >> int(level) for n in self.shape)


class _NoDevice:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def _device_of(device):
    """Context that makes `device` current for the duration of a call."""
    torch = _torch()
    if device is None or torch is None:
        return _NoDevice()
    return torch.cuda.device(device)


def residual_restrict_noalloc(shape, lo, hi, bc, u, rhs, coarse_out=None, faces=None, norms=True,
                              stream=None):
    """Residual r = rhs - L u of the CUDA tensors u, rhs (shape (nz, ny, nx) on
    the box [lo, hi], boundary kinds bc, all in x, y, z order) without a Grid
    and without allocating device memory: its 8-cell mean into coarse_out (or
    None) and, when norms is true, returns (sum r^2, max |r|).  faces: None
    (homogeneous ghosts) or six CUDA float64 face tensors (None entries are
    zero faces).  Runs on `stream` (a cudaStream_t as int; default: torch's
    current stream).  Calls on one device must not overlap: they share one
    scratch array."""
    torch = _torch()
    if torch is None or not isinstance(u, torch.Tensor) or not u.is_cuda:
        raise TypeError("u must be a CUDA tensor")
    dt = 0 if u.dtype == torch.float64 else 1
    nz, ny, nx = (int(v) for v in shape)
    dev = u.device
    # the kernels take bare pointers: every array must have the stated shape and
    # sit on u's device, whose scratch array the call uses
    up = _dev_ptr(u, dt, (nz, ny, nx), dev)
    rp = _dev_ptr(rhs, dt, (nz, ny, nx), dev)
    cp = None
    if coarse_out is not None:
        cp = _dev_ptr(coarse_out, dt, (nz // 2, ny // 2, nx // 2), dev)
    fp = None
    if faces is not None:
        if len(faces) != 6:
            raise ValueError("faces: six entries (-x, +x, -y, +y, -z, +z)")
        fshape = [(nz, ny)] * 2 + [(nz, nx)] * 2 + [(ny, nx)] * 2
        fp = (_P * 6)(*[None if f is None else _dev_ptr(f, 0, fs, dev).value for f, fs in zip(faces, fshape)])
    out = (_D * 2)() if norms else None
    if stream is None:
        stream = torch.cuda.current_stream(dev).cuda_stream
    with torch.cuda.device(dev):
        _check(lib().sg_residual_restrict_noalloc(nx, ny, nz, (_D * 3)(*lo), (_D * 3)(*hi), (_I * 3)(*bc), fp, dt,
                                                  up, rp, cp, out, stream))
    return (out[0], out[1]) if norms else None


def plan_schedule(N, count):
    """The Legendre-zero schedule of App. A.5 the solver runs (host only)."""
    out = (_I * max(1, count))()
    _check(lib().sg_plan_schedule(int(N), int(count), out))
    return list(out[:count])


def plan_stage_coefficients(order, s):
    """{mu, nu, mut, gt: lists of s + 1, tau_max_over_dtpar} of one super-step (host only)."""
    arrs = [(_D * (s + 1))() for _ in range(4)]
    t = _D(0.0)
    _check(lib().sg_plan_stage_coefficients(int(order), int(s), *arrs, ctypes.byref(t)))
    return {"mu": list(arrs[0]), "nu": list(arrs[1]), "mut": list(arrs[2]), "gt": list(arrs[3]),
            "tau_max_over_dtpar": t.value}


def plan_s_opt(N):
    """App. A.4's global s_opt for a level of largest extent N (host only)."""
    out = _I(0)
    _check(lib().sg_plan_s_opt(int(N), ctypes.byref(out)))
    return out.value


def measure_fp64_rate():
    """(TFLOP/s, ms) of FP64 FMA chains on the current device (roofline aid)."""
    t, ms = _D(0.0), _D(0.0)
    _check(lib().sg_measure_fp64_rate(ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def plan_levels(shape):
    """Level count of the level rule for shape (nz, ny, nx) (host only)."""
    nz, ny, nx = (int(v) for v in shape)
    return lib().sg_plan_levels(nx, ny, nz)


def plan_sor_omega(shape, lo, hi):
    """App. B's SOR omega for shape (nz, ny, nx) on [lo, hi] (x, y, z order; host only)."""
    nz, ny, nx = (int(v) for v in shape)
    om = _D(0.0)
    _check(lib().sg_plan_sor_omega(nx, ny, nz, (_D * 3)(*lo), (_D * 3)(*hi), ctypes.byref(om)))
    return om.value


def solve_batch(grids, tol=1e-8):
    """Solve several prepared grids through sg_solve_batch; returns their infos."""
    n = len(grids)
    hs = (ctypes.c_void_p * n)(*[g.handle.value for g in grids])
    infos = (SolveInfo * n)()
    st = lib().sg_solve_batch(hs, n, float(tol), infos)
    _check(st)
    return [i.as_dict() for i in infos]


def _autograd():
    import torch

    class PoissonSolve(torch.autograd.Function):
        """phi = solve(rho) on a prepared grid; backward is the adjoint solve
        L_h lambda = dL/dphi with dL/drho = 4 pi G lambda (sg_backward)."""

        @staticmethod
        def forward(ctx, rho, grid, tol, levels):
            rho = rho.detach().contiguous()
            grid.set_density(rho, grid.four_pi_G)
            grid.solve(tol=tol, levels=levels)
            phi = torch.empty_like(rho)
            grid.potential(phi)
            ctx.grid, ctx.tol = grid, tol
            return phi

        @staticmethod
        def backward(ctx, gphi):
            g = torch.empty_like(gphi)
            ctx.grid.backward(gphi.detach().contiguous(), g, tol=ctx.tol)
            return g, None, None, None

    return PoissonSolve


def __getattr__(name):
    if name == "PoissonSolve":
        return _autograd()
    raise AttributeError(name)


def solve(rho, grid, tol=1e-10, levels=0):
    """Differentiable solve: phi = L_h^{-1}(4 pi G rho) on `grid` (a Grid whose
    boundary and four_pi_G are set), usable inside torch autograd."""
    return _autograd().apply(rho, grid, tol, levels)
