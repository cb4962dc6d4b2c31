"""Pins of the oracle's matrix-free Hessian-vector product (Sec. 5.5,
Sec. 6.2; used by the CG solver of Sec. 7.2) to facts outside it:

* hv is the directional derivative of the gradient, checked by
  Richardson-extrapolated central differences of the oracle's gradient
  along v (which also catches a transposed block or a wrong gather);
* the Hessian is symmetric: u.(H v) = v.(H u);
* every energy here is invariant under translation, so H t = 0 for a
  uniform translation t at any x."""
import numpy as np
import pytest

import oracle
import synth

SHELL_P = [1.0e5, 0.3, 1.0e-3]


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def cases():
    grid = synth.grid_uv(n=7, sigma=0.05, seed=11)
    V, F = synth.icosphere(1)
    xs = synth.perturb(V, sigma=2e-2, seed=12)
    out = [("symdir", oracle.Problem(grid.rest, grid.faces, oracle.SYMDIR, 2), grid.x)]
    for name, e in [("stvk", oracle.STVK), ("nh", oracle.NH), ("hinge", oracle.HINGE), ("shell", oracle.SHELL)]:
        out.append((name, oracle.Problem(V, F, e, 3, [0.5, 1.0] if e == oracle.HINGE else SHELL_P), xs))
    return out


CASES = cases()


@pytest.mark.parametrize("name,P,x", CASES, ids=[c[0] for c in CASES])
def test_hvp_is_directional_derivative_of_gradient(name, P, x):
    rng = np.random.default_rng(3)
    v = rng.normal(size=x.shape)
    hv = P.hvp(x, v)["hv"]

    def g(y):
        return P.assemble(y, hessian=False)["grad"]

    def d(h):
        return (g(x + h * v) - g(x - h * v)) / (2 * h)

    h = 1e-4 * np.abs(x).max()
    fd = (4 * d(h / 2) - d(h)) / 3
    assert rel(fd, hv) < 1e-6


@pytest.mark.parametrize("name,P,x", CASES, ids=[c[0] for c in CASES])
def test_hvp_symmetric(name, P, x):
    rng = np.random.default_rng(4)
    u = rng.normal(size=x.shape)
    v = rng.normal(size=x.shape)
    a = np.vdot(u, P.hvp(x, v)["hv"])
    b = np.vdot(v, P.hvp(x, u)["hv"])
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))


@pytest.mark.parametrize("name,P,x", CASES, ids=[c[0] for c in CASES])
def test_hvp_translation_null(name, P, x):
    t = np.tile(np.arange(1.0, x.shape[1] + 1), (x.shape[0], 1))
    hv = P.hvp(x, t)["hv"]
    scale = np.abs(P.assemble(x)["vals"]).max() * np.abs(t).max()
    assert np.abs(hv).max() <= 1e-10 * scale
