"""The per-term Hessian filtering of the filtered passes (Sec. 7.1: a term's
negative local eigenvalues set to eps), the device code of spd.cuh compiled
for the host, against the FP64 oracle's projection (numpy eigh of the
vertex-DOF local Hessian with the translations kept null, oracle.spd_project).

The device filter works on the term's Hessian in its edge vectors He
(H = D^T He D for the edge map D): its edge-metric transform, shifted-Cholesky
test and round-robin Jacobi share nothing with the oracle but the definition.
He is recovered from the oracle's H as (D D^T)^-1 D H D^T (D D^T)^-1.

Local Hessians come from the oracle on a deformed icosphere (5e-2 of the
radius), where most hinge and many triangle Hessians are indefinite.  Bars:
FP64 1e-10 relative Frobenius per term; FP32 (He rounded to float, the
device's FP32 threshold tau = 1e-5 on both sides) 2e-5."""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth
from paper_2509_00406_gb300 import _build

SHELL_P = [1.0e5, 0.3, 1.0e-3]
HINGE_C = [[-1, -1, 0], [1, 0, -1], [0, 1, 0], [0, 0, 1]]   # vertex a, edge p: e = x1-x0, u = xa-x0, v = xb-x1
TRI_C = [[-1, -1], [1, 0], [0, 1]]                          # u = x1-x0, w = x2-x0


@pytest.fixture(scope="module")
def H():
    L = C.CDLL(_build.build_host())
    L.adm_host_project_edges.argtypes = [C.c_int32, C.c_int32, np.ctypeslib.ndpointer(np.float64), C.c_double]
    return L


def edge_map(coef):
    nv, ne = len(coef), len(coef[0])
    D = np.zeros((ne * 3, nv * 3))
    for a in range(nv):
        for p in range(ne):
            D[3 * p:3 * p + 3, 3 * a:3 * a + 3] = coef[a][p] * np.eye(3)
    return D


def packed(M):
    n = M.shape[0]
    return np.array([M[i, j] for j in range(n) for i in range(j + 1)])


def unpacked(v, n):
    M = np.zeros((n, n))
    k = 0
    for j in range(n):
        for i in range(j + 1):
            M[i, j] = M[j, i] = v[k]
            k += 1
    return M


def filtered(H, kind, prec, Hv, coef, eps):
    D = edge_map(coef)
    Mi = np.linalg.inv(D @ D.T)
    He = Mi @ D @ Hv @ D.T @ Mi
    v = np.ascontiguousarray(packed(0.5 * (He + He.T)))
    assert H.adm_host_project_edges(kind, prec, v, eps) == 0
    return D.T @ unpacked(v, D.shape[0]) @ D


def problem():
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=5e-2, seed=31)
    return oracle.Problem(V, F, oracle.SHELL, 3, params=SHELL_P), x


# FP32 at eps = 0: an eigenvalue that FP32 round-off puts on the other side
# of the threshold -tau max|lambda| than FP64 moves the result by about
# tau max|lambda|, within the bar; with an eps comparable to the Hessian's
# norm (1e-3 here is about 60 % of it) the same flip moves it by eps
@pytest.mark.parametrize("prec,eps", [(0, 0.0), (0, 1e-3), (1, 0.0)])
def test_hinge_filter_matches_oracle_projection(H, prec, eps):
    P, x = problem()
    ph = oracle._shell_hinge_params(SHELL_P)
    tol, tau = (1e-10, oracle.SPD_TAU) if prec == 0 else (2e-5, 1e-5)
    clamped = 0
    for h in range(0, P.nH, 3):
        vid = P.H[h]
        Hv = oracle.local(oracle.HINGE, x[vid], 3, thetabar=P.thetabar[h], abar=P.abar[h], params=ph)["H"]
        Hv = 0.5 * (Hv + Hv.T)
        want = oracle.spd_project(Hv, eps, oracle.translations(4, 3), tau=tau)
        got = filtered(H, 0, prec, Hv, HINGE_C, eps)
        clamped += np.abs(want - Hv).max() > 1e-8 * np.abs(Hv).max()
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), h
    assert clamped > 0.5 * len(range(0, P.nH, 3))        # most of them indefinite


@pytest.mark.parametrize("prec", [0, 1])
def test_triangle_filter_matches_oracle_projection(H, prec):
    P, x = problem()
    tol, tau = (1e-10, oracle.SPD_TAU) if prec == 0 else (2e-5, 1e-5)
    clamped = 0
    for t in range(P.nT):
        vid = P.F[t]
        Hv = oracle.local(oracle.STVK, x[vid], 3, P.Dinv[t], P.area[t], params=SHELL_P)["H"]
        Hv = 0.5 * (Hv + Hv.T)
        want = oracle.spd_project(Hv, 0.0, oracle.translations(3, 3), tau=tau)
        got = filtered(H, 1, prec, Hv, TRI_C, 0.0)
        clamped += np.abs(want - Hv).max() > 1e-8 * np.abs(Hv).max()
        assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want), t
    assert clamped > 0


def test_bad_kind_is_refused(H):
    v = np.zeros(45)
    assert H.adm_host_project_edges(2, 0, v, 0.0) == 9
    assert H.adm_host_project_edges(0, 2, v, 0.0) == 9
