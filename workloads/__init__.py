"""Seeded synthetic inputs for the RKL-multigrid Poisson solver.

This module only builds inputs: densities, Dirichlet face values taken from
analytic potentials, loss weights and random sample positions.  It holds none
of the solver's arithmetic, so the CPU oracle (``oracle/``) and the CUDA path
(``paper_2306_05332_gb300``) can both draw their inputs from it without sharing
any of the method.

Array layout everywhere: C order ``[nz][ny][nx]`` (x fastest), float64, cell
centres at ``lo + (i + 1/2) h``.  Dirichlet face arrays come in the order
``-x, +x, -y, +y, -z, +z``; the x faces are ``[nz][ny]``, the y faces
``[nz][nx]`` and the z faces ``[ny][nx]``, each sampled at the centres of the
boundary faces of the cells.

Workloads (sizes as used by the tests and the benchmark):

* ``sinusoid``   -- rho = sin(pi x) sin(pi y) sin(pi z) on [0,1]^3, phi = 0 on the
                    boundary, 4 pi G = 1 (32^3 single-level RKL1 case).
* ``sphere``     -- uniform sphere rho = 1, R = 0.25, centred in [-1,1]^3, faces
                    from the exterior potential (256^3 multigrid case).
* ``grf``        -- periodic Gaussian random field with P(k) ~ k^-3, zero mean,
                    unit rms (512^3 mixed-precision case).
* ``blobs``      -- 1-4 Gaussian blobs on the unit cube with monopole faces
                    (64-instance batched case, N in {32, 64, 96, 128}).
* ``noisy_sphere`` -- sphere plus 0.1 N(0,1) noise, and loss weights U[0,1]
                    (256^3 differentiable case).
* ``smooth_sphere`` -- the model problem of Sec. 4.1 (Eq. source_3D) with its
                    analytic potential (Eq. phi_3D), for accuracy tests.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
PERIODIC = 1


@dataclass
class Problem:
    """One Poisson problem: grad^2 phi = four_pi_G * rho on a box."""

    rho: np.ndarray                      # [nz][ny][nx] float64
    lo: tuple                            # (x, y, z)
    hi: tuple
    bc: tuple                            # per axis (x, y, z): DIRICHLET / PERIODIC
    faces: list | None = None            # 6 Dirichlet face arrays or None (all zero)
    four_pi_G: float = 1.0
    exact: np.ndarray | None = None      # analytic potential at cell centres, if any
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.rho.shape            # (nz, ny, nx)


def centres(n, lo, hi):
    h = (hi - lo) / n
    return lo + (np.arange(n, dtype=np.float64) + 0.5) * h


def mesh(shape, lo, hi):
    """Cell-centre coordinates X, Y, Z, each [nz][ny][nx]."""
    nz, ny, nx = shape
    x = centres(nx, lo[0], hi[0])
    y = centres(ny, lo[1], hi[1])
    z = centres(nz, lo[2], hi[2])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def faces_from_function(fn, shape, lo, hi):
    """Sample fn(x, y, z) at the boundary face centres, order -x,+x,-y,+y,-z,+z."""
    nz, ny, nx = shape
    x = centres(nx, lo[0], hi[0])
    y = centres(ny, lo[1], hi[1])
    z = centres(nz, lo[2], hi[2])
    zz, yy = np.meshgrid(z, y, indexing="ij")        # [nz][ny]
    zx, xz = np.meshgrid(z, x, indexing="ij")        # [nz][nx]
    yx, xy = np.meshgrid(y, x, indexing="ij")        # [ny][nx]
    return [
        np.ascontiguousarray(fn(np.full_like(zz, lo[0]), yy, zz)),
        np.ascontiguousarray(fn(np.full_like(zz, hi[0]), yy, zz)),
        np.ascontiguousarray(fn(xz, np.full_like(zx, lo[1]), zx)),
        np.ascontiguousarray(fn(xz, np.full_like(zx, hi[1]), zx)),
        np.ascontiguousarray(fn(xy, yx, np.full_like(yx, lo[2]))),
        np.ascontiguousarray(fn(xy, yx, np.full_like(yx, hi[2]))),
    ]


# --------------------------------------------------------------------------
# Analytic potentials (textbook closed forms, used for boundary values only)
# --------------------------------------------------------------------------

def sphere_potential(r, R, rho0, four_pi_G):
    """Potential of a uniform sphere solving grad^2 phi = four_pi_G rho."""
    r = np.asarray(r, dtype=np.float64)
    inside = four_pi_G * rho0 * (r * r - 3.0 * R * R) / 6.0
    with np.errstate(divide="ignore"):
        outside = -four_pi_G * rho0 * R ** 3 / (3.0 * np.maximum(r, 1e-300))
    return np.where(r <= R, inside, outside)


def smooth_sphere_potential(r, rho0=1.0, r0=0.25):
    """Eq. phi_3D of Sec. 4.1 (G = 1, so four_pi_G = 4 pi)."""
    r = np.asarray(r, dtype=np.float64)
    M = 32.0 * math.pi * rho0 * r0 ** 3 / 105.0
    inside = (-2.0 / 3.0 * math.pi * rho0 * r0 ** 2
              + 4.0 * math.pi * rho0 * (r ** 2 / 6.0 - r ** 4 / (10.0 * r0 ** 2)
                                        + r ** 6 / (42.0 * r0 ** 4)))
    with np.errstate(divide="ignore"):
        outside = -M / np.maximum(r, 1e-300)
    return np.where(r <= r0, inside, outside)


# --------------------------------------------------------------------------
# Workloads
# --------------------------------------------------------------------------

def sinusoid(n=32, four_pi_G=1.0):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    X, Y, Z = mesh((n, n, n), lo, hi)
    rho = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    exact = -four_pi_G * rho / (3.0 * np.pi ** 2)
    return Problem(rho=rho, lo=lo, hi=hi, bc=(DIRICHLET,) * 3, faces=None,
                   four_pi_G=four_pi_G, exact=exact, name=f"sinusoid{n}")


def sphere(n=256, R=0.25, rho0=1.0, four_pi_G=1.0, shape=None):
    shape = shape or (n, n, n)
    lo, hi = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0)
    X, Y, Z = mesh(shape, lo, hi)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    rho = np.where(r <= R, rho0, 0.0).astype(np.float64)
    pot = lambda x, y, z: sphere_potential(np.sqrt(x * x + y * y + z * z), R, rho0, four_pi_G)
    faces = faces_from_function(pot, shape, lo, hi)
    return Problem(rho=rho, lo=lo, hi=hi, bc=(DIRICHLET,) * 3, faces=faces,
                   four_pi_G=four_pi_G, exact=pot(X, Y, Z), name=f"sphere{shape[2]}")


def smooth_sphere(n=32):
    """Sec. 4.1 model problem on [-0.5, 0.5]^3, G = 1, faces from Eq. phi_3D."""
    lo, hi = (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5)
    shape = (n, n, n)
    X, Y, Z = mesh(shape, lo, hi)
    r = np.sqrt(X * X + Y * Y + Z * Z)
    r0 = 0.25
    rho = np.where(r <= r0, (1.0 - r * r / r0 ** 2) ** 2, 0.0)
    pot = lambda x, y, z: smooth_sphere_potential(np.sqrt(x * x + y * y + z * z))
    faces = faces_from_function(pot, shape, lo, hi)
    return Problem(rho=rho, lo=lo, hi=hi, bc=(DIRICHLET,) * 3, faces=faces,
                   four_pi_G=4.0 * math.pi, exact=pot(X, Y, Z), name=f"smooth{n}")


def grf(n=512, seed=0, slope=-3.0, shape=None):
    """Periodic Gaussian random field, P(k) ~ |k|^slope, k = 0 removed, unit rms."""
    shape = shape or (n, n, n)
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    white = rng.standard_normal(shape)
    wk = np.fft.rfftn(white)
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k = np.sqrt(KX * KX + KY * KY + KZ * KZ)
    amp = np.zeros_like(k)
    nz_mask = k > 0
    amp[nz_mask] = k[nz_mask] ** (slope / 2.0)
    rho = np.fft.irfftn(wk * amp, s=shape, axes=(0, 1, 2))
    rho -= rho.mean()
    rho /= np.sqrt(np.mean(rho * rho))
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    return Problem(rho=np.ascontiguousarray(rho), lo=lo, hi=hi, bc=(PERIODIC,) * 3,
                   faces=None, four_pi_G=1.0, name=f"grf{nx}", meta={"seed": seed})


def monopole_faces(rho, lo, hi, four_pi_G):
    """Dirichlet faces of the monopole -four_pi_G M / (4 pi |x - x_cm|)."""
    shape = rho.shape
    X, Y, Z = mesh(shape, lo, hi)
    dV = np.prod([(hi[d] - lo[d]) / shape[2 - d] for d in range(3)])
    M = rho.sum() * dV
    xc = (rho * X).sum() / rho.sum()
    yc = (rho * Y).sum() / rho.sum()
    zc = (rho * Z).sum() / rho.sum()
    pot = lambda x, y, z: -four_pi_G * M / (4.0 * math.pi * np.sqrt(
        (x - xc) ** 2 + (y - yc) ** 2 + (z - zc) ** 2))
    return faces_from_function(pot, shape, lo, hi)


def blobs(n, rng, four_pi_G=1.0):
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    shape = (n, n, n)
    X, Y, Z = mesh(shape, lo, hi)
    nb = int(rng.integers(1, 5))
    rho = np.zeros(shape)
    for _ in range(nb):
        c = rng.uniform(0.25, 0.75, size=3)
        sig = rng.uniform(0.05, 0.2)
        A = rng.uniform(0.5, 2.0)
        rho += A * np.exp(-((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2) / (2 * sig * sig))
    faces = monopole_faces(rho, lo, hi, four_pi_G)
    return Problem(rho=rho, lo=lo, hi=hi, bc=(DIRICHLET,) * 3, faces=faces,
                   four_pi_G=four_pi_G, name=f"blobs{n}", meta={"n_blobs": nb})


def blob_batch(count=64, seed=0, sizes=(32, 64, 96, 128)):
    """Batched workload: grid sizes uniform over `sizes`, 1-4 Gaussian blobs each."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    return [blobs(int(n), rng) for n in ns]


def batch_sizes(count=64, seed=0, sizes=(32, 64, 96, 128)):
    """The grid sizes `blob_batch` would draw, without building the densities."""
    rng = np.random.default_rng(seed)
    return [int(n) for n in rng.choice(np.asarray(sizes), size=count)]


def noisy_sphere(n=256, seed=0, noise=0.1):
    base = sphere(n)
    rng = np.random.default_rng(seed)
    base.rho = base.rho + noise * rng.standard_normal(base.rho.shape)
    base.exact = None
    base.name = f"noisy_sphere{n}"
    return base


def loss_weights(shape, seed=1):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=shape)


def sample_cells(shape, count=16, seed=2):
    rng = np.random.default_rng(seed)
    flat = rng.choice(int(np.prod(shape)), size=count, replace=False)
    return [tuple(int(v) for v in np.unravel_index(f, shape)) for f in flat]


def random_field(shape, seed, scale=1.0):
    """Plain N(0, scale^2) field, for operator-level parity cases."""
    return scale * np.random.default_rng(seed).standard_normal(shape)


def random_faces(shape, seed, scale=1.0):
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    dims = [(nz, ny), (nz, ny), (nz, nx), (nz, nx), (ny, nx), (ny, nx)]
    return [scale * rng.standard_normal(d) for d in dims]
