"""Pins of the oracle's mass-spring cloth energy (Sec. 7.1: implicit-Euler
inertia with a lumped mass matrix, per-edge springs, gravity) to facts
outside it:

* gradient and Hessian are the derivatives of the energy (Richardson
  central differences);
* a uniform stretch by s of the flat n x n grid, with the inertial target
  at the stretched state and no gravity, has the closed-form energy
  h^2 k/2 (s^2 - 1)^2 sum_e l_e^2, where sum_e l_e^2 is counted from the
  grid's geometry (2 n (n-1) axis edges of length a, (n-1)^2 diagonals of
  length a sqrt 2, a = 1 / (n-1));
* the lumped masses sum to rho times the area of the unit square;
* a rigid lift by z0 of the resting cloth costs rho z0^2 / 2 - h^2 rho g_z z0
  (inertia plus gravity, springs at rest);
* the springs' part of the Hessian is symmetric and annihilates
  translations."""
import numpy as np
import pytest

import oracle
import synth

P = [2.0e3, 0.02, 1.5, 0.1, -0.2, -9.81]


def problem(n=6, seed=6):
    c = synth.cloth_grid(n, sigma=0.3, seed=seed)
    rp, col = oracle.pattern(c.nV, c.faces)
    return c, rp, col


def test_gradient_is_derivative_of_energy():
    c, _, _ = problem()
    x0 = c.x.copy()
    g = oracle.cloth_assemble(c.rest, c.faces, x0, c.xhat, P)["grad"]
    rng = np.random.default_rng(1)
    v = rng.normal(size=x0.shape)

    def f(t):
        return oracle.cloth_assemble(c.rest, c.faces, x0 + t * v, c.xhat, P)["energy"]

    h = 1e-4

    def d(hh):
        return (f(hh) - f(-hh)) / (2 * hh)

    fd = (4 * d(h / 2) - d(h)) / 3
    assert abs(fd - np.vdot(g, v)) <= 1e-7 * abs(fd)


def test_hessian_is_derivative_of_gradient():
    c, rp, col = problem()
    x0 = c.x.copy()
    out = oracle.cloth_assemble(c.rest, c.faces, x0, c.xhat, P, rp, col)
    Hd = oracle.bsr_to_dense(c.nV, 3, rp, col, out["vals"])
    v = np.random.default_rng(2).normal(size=x0.shape)

    def g(t):
        return oracle.cloth_assemble(c.rest, c.faces, x0 + t * v, c.xhat, P)["grad"]

    h = 1e-4
    d = lambda hh: (g(hh) - g(-hh)) / (2 * hh)  # noqa: E731
    fd = (4 * d(h / 2) - d(h)) / 3
    hv = (Hd @ v.reshape(-1)).reshape(-1, 3)
    assert np.linalg.norm(fd - hv) <= 1e-7 * np.linalg.norm(hv)
    assert np.abs(Hd - Hd.T).max() <= 1e-12 * np.abs(Hd).max()


@pytest.mark.parametrize("n,s", [(4, 1.3), (7, 0.8)])
def test_uniform_stretch_closed_form(n, s):
    c = synth.cloth_grid(n)
    x = s * c.rest
    a = 1.0 / (n - 1)
    sum_l2 = 2 * n * (n - 1) * a * a + (n - 1) ** 2 * 2 * a * a
    k, h = 3.0e3, 0.05
    e = oracle.cloth_assemble(c.rest, c.faces, x, x, [k, h, 1.0, 0.0, 0.0, 0.0])["energy"]
    want = h * h * k / 2 * (s * s - 1) ** 2 * sum_l2
    assert abs(e - want) <= 1e-12 * want


def test_mass_total_and_rigid_lift():
    c = synth.cloth_grid(9)
    rho = 2.5
    assert abs(oracle.lumped_mass(c.rest, c.faces, rho).sum() - rho) <= 1e-12
    z0, h, gz = 0.3, 0.1, -9.81
    x = c.rest + np.array([0.0, 0.0, z0])
    e = oracle.cloth_assemble(c.rest, c.faces, x, c.rest, [1e3, h, rho, 0.0, 0.0, gz])["energy"]
    want = 0.5 * rho * z0 * z0 - h * h * rho * gz * z0
    assert abs(e - want) <= 1e-12 * abs(want)


def test_spring_hessian_annihilates_translations():
    c, rp, col = problem(seed=7)
    no_inertia = [P[0], P[1], 0.0, 0.0, 0.0, 0.0]   # rho = 0: springs only
    out = oracle.cloth_assemble(c.rest, c.faces, c.x, c.xhat, no_inertia, rp, col)
    Hd = oracle.bsr_to_dense(c.nV, 3, rp, col, out["vals"])
    t = np.tile([1.0, -2.0, 0.5], c.nV)
    assert np.abs(Hd @ t).max() <= 1e-12 * np.abs(Hd).max()
