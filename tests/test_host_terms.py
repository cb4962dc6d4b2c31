"""The device's per-element forward mode (terms.cuh: sparse hyper-duals
composed through invariants, differentiated in edge vectors, expanded to
vertex coordinates by the accessors the kernels write their chunks with),
compiled for the host, against the FP64 oracle's dense hyper-dual route
(route 0, the paper's ActiveT form): energy, gradient and local Hessian of
StVK and Neo-Hookean membrane triangles and dihedral hinges on a deformed
icosphere, and of the 2D symmetric Dirichlet term on the perturbed grid.

Bars: FP64 1e-12 relative (per element; the gradient and Hessian in the
Frobenius norm), FP32 2e-5 (inputs rounded to float; the host's FP32 math).
A hinge's energy and gradient carry theta - thetabar, which cancels near the
rest angle: a rounding d of theta (about 1e-16 pi in FP64, 1e-7 pi in FP32,
either route) moves them by up to 2 w |theta - thetabar| d and 2 w d
|grad theta|, with |grad theta| about sqrt(|H| / 2w) near rest; their bars
add that floor.  A membrane density near rest is a difference of terms of
size mu t A; its energy bar adds a few roundings of that size."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from paper_2509_00406_gb300 import _build

E_, NU, THICK = 1.0e5, 0.3, 1.0e-3
KB, HH = 0.5, 1.0        # hinge stiffness and h of the oracle's HINGE energy: w = kb abar / 3 h^2
TOL = {0: 1e-12, 1: 2e-5}
THETA_ROUND = {0: 4e-16 * np.pi, 1: 4e-7 * np.pi}   # a few roundings of theta, per precision
FLOOR = {0: 1e-15, 1: 1e-6}                         # a few roundings of a membrane density's terms
DP = np.ctypeslib.ndpointer(np.float64)


@pytest.fixture(scope="module")
def L():
    lib = C.CDLL(_build.build_host())
    lib.adm_host_tri_local.argtypes = [C.c_int32, C.c_int32, DP, DP, C.c_double, C.c_double, C.c_double, C.c_double,
                                       DP, DP, DP]
    lib.adm_host_hinge_local.argtypes = [C.c_int32, DP, C.c_double, C.c_double, DP, DP, DP]
    return lib


@pytest.fixture(scope="module")
def case():
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=3e-2, seed=17)
    return oracle.Problem(V, F, oracle.SHELL, 3, params=[E_, NU, THICK]), x


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


def rounded(a, prec):
    a = np.ascontiguousarray(a, dtype=np.float64).ravel()
    return a.astype(np.float32).astype(np.float64) if prec == 1 else a


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kind,energy", [(0, oracle.STVK), (1, oracle.NH)])
def test_membrane_triangles_match_oracle(L, case, prec, kind, energy):
    P, x = case
    for t in range(P.nT):
        vid = P.F[t]
        xl = rounded(x[vid], prec)
        ref = oracle.local(energy, xl, 3, P.Dinv[t], P.area[t], params=[E_, NU, THICK], route=0)
        f, g, H = np.zeros(1), np.zeros(9), np.zeros(81)
        Di = rounded(P.Dinv[t], prec)
        assert L.adm_host_tri_local(kind, prec, xl, Di, float(P.area[t]), E_, NU, THICK, f, g, H) == 0
        # near rest the density is a difference of terms of size mu t A
        scale = E_ / (2 * (1 + NU)) * THICK * P.area[t]
        assert abs(f[0] - ref["f"]) <= TOL[prec] * abs(ref["f"]) + FLOOR[prec] * scale, t
        assert rel(g, ref["g"]) <= TOL[prec], t
        assert rel(H.reshape(9, 9), ref["H"]) <= TOL[prec], t


@pytest.mark.parametrize("prec", [0, 1])
def test_symmetric_dirichlet_matches_oracle(L, prec):
    """The 2D symmetric Dirichlet term on the perturbed 33 x 33 grid of the
    unit square (the FP64 workload), per triangle."""
    g0 = synth.grid_uv()
    P = oracle.Problem(g0.rest, g0.faces, oracle.SYMDIR, 2)
    for t in range(0, P.nT, 5):
        vid = P.F[t]
        xl = rounded(g0.x[vid], prec)
        ref = oracle.local(oracle.SYMDIR, xl, 2, P.Dinv[t], P.area[t], route=0)
        f, g, H = np.zeros(1), np.zeros(6), np.zeros(36)
        Di = rounded(P.Dinv[t], prec)
        assert L.adm_host_tri_local(2, prec, xl, Di, float(P.area[t]), E_, NU, THICK, f, g, H) == 0
        assert abs(f[0] - ref["f"]) <= TOL[prec] * abs(ref["f"]), t
        assert np.linalg.norm(g - ref["g"]) <= TOL[prec] * np.linalg.norm(ref["H"]), t   # g vanishes near the identity
        assert rel(H.reshape(6, 6), ref["H"]) <= TOL[prec], t


@pytest.mark.parametrize("prec", [0, 1])
def test_hinges_match_oracle(L, case, prec):
    P, x = case
    for h in range(0, P.nH, 2):
        vid = P.H[h]
        xl = rounded(x[vid], prec)
        ref = oracle.local(oracle.HINGE, xl, 3, thetabar=P.thetabar[h], abar=P.abar[h], params=[KB, HH], route=0)
        w = KB * P.abar[h] / 3.0 * HH * HH
        f, g, H = np.zeros(1), np.zeros(12), np.zeros(144)
        assert L.adm_host_hinge_local(prec, xl, float(P.thetabar[h]), float(w), f, g, H) == 0
        d = THETA_ROUND[prec]
        nH = np.linalg.norm(ref["H"])
        dth = abs(float(np.sqrt(max(ref["f"], 0.0) / w)))                # |theta - thetabar|
        assert abs(f[0] - ref["f"]) <= TOL[prec] * abs(ref["f"]) + 2 * w * dth * d, h
        assert np.linalg.norm(g - ref["g"]) <= TOL[prec] * np.linalg.norm(ref["g"]) + 2 * w * d * np.sqrt(nH / (2 * w)), h
        assert rel(H.reshape(12, 12), ref["H"]) <= TOL[prec], h
