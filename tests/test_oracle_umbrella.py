"""Pins of the oracle's per-vertex one-ring term (uniform-Laplacian
smoothing, w/2 |x_v - mean of its neighbours|^2) and of its block pattern:

* gradient and Hessian are the derivatives of the energy (Richardson
  central differences);
* the energy is quadratic: its Hessian does not depend on x, E(s x) =
  s^2 E(x), and translations cost nothing;
* on the flat regular grid every interior vertex is the mean of its six
  neighbours (they come in opposite pairs), so with x affine in the rest
  position only boundary vertices contribute;
* the pattern is the set of vertex pairs within two edges, computed here
  independently as the nonzeros of I + A + A^2 of the adjacency matrix A."""
import numpy as np
import pytest

import oracle
import synth

W = 1.7


def cases():
    V, F = synth.icosphere(1)
    g = synth.grid_uv(n=6, sigma=0.3, seed=3)
    return [("sphere3d", F, synth.perturb(V, 5e-2, 4)), ("grid2d", g.faces, g.x)]


@pytest.mark.parametrize("name,F,x", cases(), ids=["sphere3d", "grid2d"])
def test_derivatives(name, F, x):
    nV, vd = x.shape
    rp, col = oracle.ring_pattern(nV, F)
    out = oracle.umbrella_assemble(F, x, W, rp, col)
    v = np.random.default_rng(2).normal(size=x.shape)

    def e(t):
        return oracle.umbrella_assemble(F, x + t * v, W)["energy"]

    def g(t):
        return oracle.umbrella_assemble(F, x + t * v, W)["grad"]

    h = 1e-3
    d = lambda fn, hh: (fn(hh) - fn(-hh)) / (2 * hh)  # noqa: E731
    fd_e = (4 * d(e, h / 2) - d(e, h)) / 3
    assert abs(fd_e - np.vdot(out["grad"], v)) <= 1e-9 * abs(fd_e)
    fd_g = (4 * d(g, h / 2) - d(g, h)) / 3
    Hd = oracle.bsr_to_dense(nV, vd, rp, col, out["vals"])
    assert np.abs(fd_g.reshape(-1) - Hd @ v.reshape(-1)).max() <= 1e-9 * np.abs(fd_g).max()


@pytest.mark.parametrize("name,F,x", cases(), ids=["sphere3d", "grid2d"])
def test_quadratic_invariances(name, F, x):
    nV, vd = x.shape
    rp, col = oracle.ring_pattern(nV, F)
    a = oracle.umbrella_assemble(F, x, W, rp, col)
    b = oracle.umbrella_assemble(F, 2.5 * x + 0.3, W, rp, col)
    assert np.abs(a["vals"] - b["vals"]).max() <= 1e-14 * np.abs(a["vals"]).max()
    assert abs(oracle.umbrella_assemble(F, 2.5 * x, W)["energy"] - 6.25 * a["energy"]) <= 1e-12 * a["energy"]
    assert abs(oracle.umbrella_assemble(F, x + 0.3, W)["energy"] - a["energy"]) <= 1e-12 * a["energy"]


def test_affine_grid_interior_is_free():
    g = synth.grid_uv(n=7)
    x = g.rest[:, :2] @ np.array([[1.3, 0.2], [-0.4, 0.9]]) + 0.5
    total = oracle.umbrella_assemble(g.faces, x, W)["energy"]
    n = 7
    boundary = [i for i in range(n * n) if i % n in (0, n - 1) or i // n in (0, n - 1)]
    rings = oracle.vertex_rings(n * n, g.faces)
    part = sum(0.5 * W * np.sum((x[v] - x[rings[v]].mean(0)) ** 2) for v in boundary)
    assert total > 0 and abs(total - part) <= 1e-12 * total


def test_pattern_is_two_ring():
    V, F = synth.icosphere(1)
    nV = len(V)
    A = np.zeros((nV, nV), dtype=np.int64)
    for f in F:
        for c in range(3):
            A[f[c], f[(c + 1) % 3]] = A[f[(c + 1) % 3], f[c]] = 1
    M = np.eye(nV, dtype=np.int64) + A + A @ A
    rp, col = oracle.ring_pattern(nV, F)
    for r in range(nV):
        assert list(col[rp[r]:rp[r + 1]]) == list(np.nonzero(M[r])[0])
