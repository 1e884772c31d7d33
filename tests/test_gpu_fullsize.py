"""Full-size parity of the configurations other than the 256^3 benchmark:

* the 512^3 periodic Gaussian random field (P(k) ~ k^-3, mean removed), mixed
  precision to a relative residual of 1e-8: the residual of the returned
  potential is recomputed on the CPU in FP64 from the definition of the
  periodic 7-point Laplacian (np.roll), and the potential has zero mean;
* the 256^3 differentiable solve (uniform sphere plus 10% seeded noise, loss
  L = sum w phi with w ~ U[0, 1]): the adjoint gradient dL/drho on 16 seeded
  cells against central differences of the forward solve.  phi is linear in
  rho, so central differences are exact up to the solver's tolerance; a large
  step (100) keeps that tolerance far below the differences.
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


def periodic_residual(phi, f, h):
    """L phi - f for the periodic 7-point Laplacian, by its definition."""
    hx, hy, hz = h
    lap = (-2.0 * (1.0 / hx ** 2 + 1.0 / hy ** 2 + 1.0 / hz ** 2)) * phi
    for axis, hd in ((2, hx), (1, hy), (0, hz)):
        lap += (np.roll(phi, 1, axis) + np.roll(phi, -1, axis)) * (1.0 / hd ** 2)
    lap -= f
    return lap


def test_grf_512_periodic_mixed_reaches_tolerance():
    sg = _sg()
    p = W.grf(512, seed=0)
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="mixed")
    g.set_density(p.rho, p.four_pi_G)
    info = g.solve(tol=1e-8)
    assert info["rel_residual"] <= 1e-8
    phi = g.potential()
    del g
    f = p.four_pi_G * (p.rho - p.rho.mean())            # Eq. source_modification
    h = O.spacing(p.shape, p.lo, p.hi)
    r = periodic_residual(phi, f, h)
    rel = np.sqrt(np.mean(r * r)) / np.sqrt(np.mean(f * f))
    assert rel <= 1.01e-8
    assert abs(phi.mean()) <= 1e-10 * np.abs(phi).max()


def test_adjoint_256_noisy_sphere_against_central_differences():
    sg = _sg()
    p = W.noisy_sphere(256, seed=0, noise=0.1)
    w = W.loss_weights(p.shape, seed=1)
    g = sg.Grid(p.shape, p.lo, p.hi, p.bc, precision="fp64")
    g.set_boundary(p.faces)
    g.set_density(p.rho, 1.0)
    g.solve(tol=1e-11, levels=5)
    grad, _ = g.backward(w, tol=1e-11)
    eps = 100.0
    for cell in W.sample_cells(p.shape, 16, seed=2):
        vals = []
        for sgn in (1.0, -1.0):
            r2 = p.rho.copy()
            r2[cell] += sgn * eps
            g.set_density(r2, 1.0)
            g.solve(tol=1e-11, levels=5)
            vals.append(float(np.sum(w * g.potential())))
        fd = (vals[0] - vals[1]) / (2.0 * eps)
        assert abs(fd - grad[cell]) <= 1e-5 * abs(fd) + 1e-7, (cell, fd, grad[cell])
