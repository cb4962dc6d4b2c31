"""Pins of the CPU FP64 oracle against facts that do not come from the oracle
itself: the paper's printed formulas, closed forms, hand-enumerated
fixtures (tests/golden), finite differences, invariances and brute force.

A plausible slip anywhere in the oracle (a dropped term, a flipped sign, a
transposed operand, a wrong index) makes at least one of these fail."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(1234)

E, NU, T = 1.0e5, 0.3, 1.0e-3
MU = E / (2 * (1 + NU))
LAM = E * NU / (1 - NU * NU)


# --------------------------------------------------------------------------
# helpers
# --------------------------------------------------------------------------
def fd_grad(fun, x, h=1e-5):
    """Richardson-extrapolated central differences of a scalar function."""
    g = np.zeros_like(x)
    for i in range(x.size):
        def d(step):
            e = np.zeros_like(x)
            e.flat[i] = step
            return (fun(x + e) - fun(x - e)) / (2 * step)
        g.flat[i] = (4 * d(h / 2) - d(h)) / 3
    return g


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


def single_triangle_rest():
    """A generic rest triangle in 3D and its oracle rest data."""
    V = np.array([[0.1, -0.2, 0.3], [1.2, 0.1, 0.2], [0.3, 0.9, -0.1]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    Dinv, area = oracle.tri_rest(V, F)
    return V, Dinv[0], area[0]


def local_fd_check(energy, xl, vdim, **kw):
    out = oracle.local(energy, xl, vdim=vdim, **kw)
    assert out["err"] == 0
    f = lambda y: oracle.local(energy, y, vdim=vdim, **kw)["f"]
    gfd = fd_grad(f, xl.copy())
    assert rel(out["g"], gfd) < 1e-8, (out["g"], gfd)
    gf = lambda y: oracle.local(energy, y, vdim=vdim, **kw)["g"]
    Hfd = np.stack([fd_grad(lambda y, i=i: gf(y)[i], xl.copy()) for i in range(xl.size)])
    assert rel(out["H"], Hfd) < 1e-7
    assert np.allclose(out["H"], out["H"].T, rtol=0, atol=1e-12 * np.abs(out["H"]).max())
    return out


# --------------------------------------------------------------------------
# 1. elementary hyper-dual rules (textbook derivatives)
# --------------------------------------------------------------------------
@pytest.mark.parametrize(
    "op,inputs,f,g,H",
    [
        (0, (1.7,), lambda a: 1 / a, lambda a: [-1 / a**2], lambda a: [[2 / a**3]]),
        (1, (2.3,), np.sqrt, lambda a: [0.5 / np.sqrt(a)], lambda a: [[-0.25 * a**-1.5]]),
        (2, (0.8,), np.log, lambda a: [1 / a], lambda a: [[-1 / a**2]]),
        (3, (0.9,), np.sin, lambda a: [np.cos(a)], lambda a: [[-np.sin(a)]]),
        (4, (0.9,), np.cos, lambda a: [-np.sin(a)], lambda a: [[-np.cos(a)]]),
    ],
)
def test_hd_unary_rules(op, inputs, f, g, H):
    v, gg, hh = oracle.hd_probe(op, *inputs)
    a = inputs[0]
    assert np.isclose(v, f(a), rtol=1e-15)
    assert np.allclose(gg, g(a), rtol=1e-14)
    assert np.allclose(hh, H(a), rtol=1e-14)


def test_hd_binary_rules():
    y, x = 0.7, -1.3
    v, g, H = oracle.hd_probe(5, y, x)          # atan2(y, x)
    r2 = x * x + y * y
    assert np.isclose(v, np.arctan2(y, x))
    assert np.allclose(g, [x / r2, -y / r2])
    fy = lambda z: oracle.hd_probe(5, *z)[1]
    Hfd = np.stack([fd_grad(lambda z, i=i: fy(z)[i], np.array([y, x])) for i in range(2)])
    assert np.allclose(H, Hfd, atol=1e-9)
    v, g, H = oracle.hd_probe(6, 2.0, 3.0)      # product
    assert v == 6.0 and np.allclose(g, [3, 2]) and np.allclose(H, [[0, 1], [1, 0]])
    v, g, H = oracle.hd_probe(7, 2.0, 4.0)      # quotient a/b
    assert np.isclose(v, 0.5)
    assert np.allclose(g, [0.25, -2 / 16])
    assert np.allclose(H, [[0, -1 / 16], [-1 / 16, 2 * 2 / 64]])


# --------------------------------------------------------------------------
# 2. rest frame
# --------------------------------------------------------------------------
def test_rest_frame_preserves_edges():
    V, Dinv, area = single_triangle_rest()
    Dm = np.linalg.inv(Dinv.reshape(2, 2))
    u, w = V[1] - V[0], V[2] - V[0]
    # Dm holds the rest edges in an orthonormal frame: lengths, angle, area kept
    assert np.isclose(np.linalg.norm(Dm[:, 0]), np.linalg.norm(u))
    assert np.isclose(np.linalg.norm(Dm[:, 1]), np.linalg.norm(w))
    assert np.isclose(Dm[:, 0] @ Dm[:, 1], u @ w)
    assert np.isclose(area, 0.5 * np.linalg.norm(np.cross(u, w)))
    assert np.isclose(np.linalg.det(Dm), 2 * area)          # counter-clockwise frame
    assert np.isclose(Dm[1, 0], 0.0, atol=1e-15)            # e1 along the first edge


# --------------------------------------------------------------------------
# 3. symmetric Dirichlet (Sec. 7.2)
# --------------------------------------------------------------------------
def test_symdir_identity_grid():
    g = synth.grid_uv(33, 0.0, 1)
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    out = P.assemble(g.rest[:, :2])
    # J is a rotation on every triangle: |J|^2 = |J^-1|^2 = 2, sum of areas = 1
    assert abs(out["energy"] - 4.0) < 1e-13
    assert np.abs(out["grad"]).max() < 1e-13
    assert out["n_domain_err"] == 0


def test_symdir_uniform_scale_closed_form():
    g = synth.grid_uv(9, 0.0, 1)
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    for s in (0.5, 1.3, 2.0):
        out = P.assemble(s * g.rest[:, :2], hessian=False)
        assert np.isclose(out["energy"], 2 * s * s + 2 / (s * s), rtol=1e-13)


def test_symdir_hessian_at_identity_closed_form():
    # rest triangle in the xy-plane with its first edge along +x: the local
    # frame is the xy frame and J = I at uv = rest_xy.  Second variation of
    # A(|J|^2 + |J^-1|^2) at J = I:  d2f[dJ, dJ] = 4A (|dJ|^2 + tr(dJ dJ)).
    V = np.array([[0.0, 0.0, 0.0], [1.3, 0.0, 0.0], [0.4, 0.8, 0.0]])
    Dinv, area = oracle.tri_rest(V, np.array([[0, 1, 2]], dtype=np.int32))
    out = oracle.local(oracle.SYMDIR, V[:, :2].ravel(), vdim=2, Dinv=Dinv[0], area=area[0])
    assert np.abs(out["g"]).max() < 1e-14
    D = np.linalg.inv(np.linalg.inv(Dinv[0].reshape(2, 2)))
    for _ in range(5):
        dx = RNG.normal(size=(3, 2))
        dJ = np.stack([dx[1] - dx[0], dx[2] - dx[0]], 1) @ D      # d(Ds) Dm^-1
        expect = 4 * area[0] * (np.sum(dJ * dJ) + np.trace(dJ @ dJ))
        assert np.isclose(dx.ravel() @ out["H"] @ dx.ravel(), expect, rtol=1e-12)


def test_symdir_routes_and_fd():
    V, Dinv, area = single_triangle_rest()
    xl = RNG.normal(scale=0.1, size=6) + np.array([0, 0, 1.0, 0.1, 0.2, 0.9])
    out = local_fd_check(oracle.SYMDIR, xl, 2, Dinv=Dinv, area=area)
    cf = oracle.local(oracle.SYMDIR, xl, vdim=2, Dinv=Dinv, area=area, route=1)
    assert np.isclose(cf["f"], out["f"], rtol=1e-14)
    assert rel(cf["g"], out["g"]) < 1e-13


def test_symdir_flip_is_domain_error():
    V, Dinv, area = single_triangle_rest()
    flipped = np.array([0, 0, 0, 1.0, 1.0, 0])          # clockwise image
    assert oracle.local(oracle.SYMDIR, flipped, vdim=2, Dinv=Dinv, area=area)["err"] == 1
    g = synth.grid_uv(33, 0.01, 1, relative=False)      # absolute sigma folds triangles
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    assert P.assemble(g.x, hessian=False)["n_domain_err"] > 0


# --------------------------------------------------------------------------
# 4. StVK membrane
# --------------------------------------------------------------------------
def test_stvk_rest_state():
    V, Dinv, area = single_triangle_rest()
    out = oracle.local(oracle.STVK, V.ravel(), Dinv=Dinv, area=area)
    assert abs(out["f"]) < 1e-20 and np.abs(out["g"]).max() < 1e-12
    ev = np.linalg.eigvalsh(out["H"])
    scale = ev.max()
    # 6-dimensional rigid-motion null space, positive otherwise
    assert np.sum(np.abs(ev) < 1e-9 * scale) == 6
    assert ev.min() > -1e-9 * scale


def test_stvk_uniaxial_closed_form():
    # rest triangle in the xy-plane with e1 = +x; stretch x by s:
    # E = diag((s^2-1)/2, 0), psi = (mu + lambda/2) (s^2 - 1)^2 / 4
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.7, 0.0]])
    Dinv, area = oracle.tri_rest(V, np.array([[0, 1, 2]], dtype=np.int32))
    for s in (0.8, 1.1, 1.4):
        x = V * np.array([s, 1.0, 1.0])
        f = oracle.local(oracle.STVK, x.ravel(), Dinv=Dinv[0], area=area[0])["f"]
        assert np.isclose(f, T * area[0] * (MU + 0.5 * LAM) * (s * s - 1) ** 2 / 4, rtol=1e-13)


def test_stvk_routes_and_fd():
    V, Dinv, area = single_triangle_rest()
    xl = V.ravel() + RNG.normal(scale=0.1, size=9)
    out = local_fd_check(oracle.STVK, xl, 3, Dinv=Dinv, area=area)
    cf = oracle.local(oracle.STVK, xl, Dinv=Dinv, area=area, route=1)
    assert np.isclose(cf["f"], out["f"], rtol=1e-14)
    assert rel(cf["g"], out["g"]) < 1e-13
    assert rel(cf["H"], out["H"]) < 1e-13


# --------------------------------------------------------------------------
# 5. Neo-Hookean membrane (invariants of C, Sec. 7.7)
# --------------------------------------------------------------------------
def test_nh_rest_and_uniaxial():
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.7, 0.0]])
    Dinv, area = oracle.tri_rest(V, np.array([[0, 1, 2]], dtype=np.int32))
    out = oracle.local(oracle.NH, V.ravel(), Dinv=Dinv[0], area=area[0])
    assert abs(out["f"]) < 1e-15 and np.abs(out["g"]).max() < 1e-12
    for s in (0.7, 1.2, 1.4):
        x = V * np.array([s, 1.0, 1.0])
        f = oracle.local(oracle.NH, x.ravel(), Dinv=Dinv[0], area=area[0])["f"]
        psi = 0.5 * MU * (s * s - 1) - MU * np.log(s) + 0.5 * LAM * np.log(s) ** 2
        assert np.isclose(f, T * area[0] * psi, rtol=1e-12)


def test_nh_routes_and_fd():
    V, Dinv, area = single_triangle_rest()
    xl = V.ravel() + RNG.normal(scale=0.1, size=9)
    out = local_fd_check(oracle.NH, xl, 3, Dinv=Dinv, area=area)
    cf = oracle.local(oracle.NH, xl, Dinv=Dinv, area=area, route=1)
    assert np.isclose(cf["f"], out["f"], rtol=1e-13)
    assert rel(cf["g"], out["g"]) < 1e-12


# --------------------------------------------------------------------------
# 6. hinge bending (Sec. 7.7)
# --------------------------------------------------------------------------
def _hinge_x(pa, pb):
    return np.array([[0, 0, 0], [1, 0, 0], [0.5, np.cos(pa), np.sin(pa)],
                     [0.5, -np.cos(pb), np.sin(pb)]], dtype=float)


def test_hinge_golden_angles():
    rows = np.loadtxt(os.path.join(GOLDEN, "hinge_angles.txt"))
    for pa, pb, theta in rows:
        # f = w (theta - 0)^2 with w = k_b A/3 h^2; k_b = 3, A = 1, h = 1 -> f = theta^2
        out = oracle.local(oracle.HINGE, _hinge_x(pa, pb).ravel(), thetabar=0.0, abar=1.0,
                           params=[3.0, 1.0])
        assert np.isclose(out["f"], theta**2, rtol=1e-12, atol=1e-24)
        # the signed angle itself: f with thetabar = theta vanishes
        out2 = oracle.local(oracle.HINGE, _hinge_x(pa, pb).ravel(), thetabar=theta, abar=1.0,
                            params=[3.0, 1.0])
        assert abs(out2["f"]) < 1e-24


def test_hinge_rigid_invariance_and_rest_rank1():
    x = _hinge_x(0.3, 0.5) + RNG.normal(scale=0.05, size=(4, 3))
    rest = oracle.hinge_rest(np.array([[0, 1, 2, 3]], dtype=np.int32), x)
    th = rest[0][0]
    Q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    xr = x @ Q.T + np.array([0.3, -1.0, 2.0])
    assert np.isclose(oracle.hinge_rest(np.array([[0, 1, 2, 3]], dtype=np.int32), xr)[0][0], th)
    out = oracle.local(oracle.HINGE, x.ravel(), thetabar=th, abar=0.7, params=[2.0, 1.0])
    assert abs(out["f"]) < 1e-28 and np.abs(out["g"]).max() < 1e-14
    ev = np.linalg.eigvalsh(out["H"])
    assert np.sum(np.abs(ev) > 1e-10 * np.abs(ev).max()) == 1     # rank one, 2 w dth dth^T
    cf = oracle.local(oracle.HINGE, x.ravel(), thetabar=th - 1e-3, abar=0.7, params=[2.0, 1.0],
                      route=1)
    w = 2.0 * 0.7 / 3.0
    dth = cf["g"] / (2 * w * 1e-3)
    assert rel(out["H"], 2 * w * np.outer(dth, dth)) < 1e-8


def test_hinge_routes_fd_invariances():
    x = _hinge_x(0.2, -0.4) + RNG.normal(scale=0.05, size=(4, 3))
    out = local_fd_check(oracle.HINGE, x.ravel(), 3, thetabar=0.1, abar=0.6, params=[1.5, 0.5])
    cf = oracle.local(oracle.HINGE, x.ravel(), thetabar=0.1, abar=0.6, params=[1.5, 0.5], route=1)
    assert np.isclose(cf["f"], out["f"], rtol=1e-14)
    assert rel(cf["g"], out["g"]) < 1e-12
    g = out["g"].reshape(4, 3)
    assert np.abs(g.sum(0)).max() < 1e-12 * np.abs(g).max()
    assert np.abs(np.cross(x, g).sum(0)).max() < 1e-12 * np.abs(g).max()


@pytest.mark.parametrize("pa,pb", [(0.2, -0.4), (0.9, 0.7), (-1.3, 0.4), (2.6, -2.5)])
def test_hinge_closed_form_hessian(pa, pb):
    """The closed-form hinge Hessian (product rule on the discrete-shells
    gradient) against the hyper-dual route and against Richardson
    differences of the closed-form gradient; symmetric, translations in its
    null space; at rest it is 2 w dtheta dtheta^T."""
    x = _hinge_x(pa, pb) + RNG.normal(scale=0.05, size=(4, 3))
    kw = dict(thetabar=0.35, abar=0.6, params=[1.5, 0.5])
    cf = oracle.local(oracle.HINGE, x.ravel(), route=1, **kw)
    hd = oracle.local(oracle.HINGE, x.ravel(), route=0, **kw)
    assert rel(cf["H"], hd["H"]) < 1e-11
    assert rel(cf["H"], cf["H"].T) < 1e-13
    fdH = np.stack([fd_grad(lambda y: oracle.local(oracle.HINGE, y, route=1, **kw)["g"][i], x.ravel(), h=1e-4)
                    for i in range(12)])
    assert rel(cf["H"], fdH) < 1e-8
    for d in range(3):
        t = np.zeros((4, 3))
        t[:, d] = 1.0
        assert np.abs(cf["H"] @ t.ravel()).max() < 1e-11 * np.abs(cf["H"]).max()
    rest = oracle.hinge_rest(np.array([[0, 1, 2, 3]], dtype=np.int32), x)
    at = oracle.local(oracle.HINGE, x.ravel(), thetabar=rest[0][0], abar=0.6, params=[1.5, 0.5], route=1)
    w = 1.5 * 0.6 / 3.0 * 0.5 ** 2
    near = oracle.local(oracle.HINGE, x.ravel(), thetabar=rest[0][0] - 1e-3, abar=0.6, params=[1.5, 0.5], route=1)
    dth = near["g"] / (2 * w * 1e-3)
    assert rel(at["H"], 2 * w * np.outer(dth, dth)) < 1e-10


def test_shell_closed_form_route_assembles_hyperdual_result():
    """Route 1 of the whole shell (closed-form StVK and hinge Hessians)
    assembles the same gradient and BSR Hessian as route 0."""
    sh = synth.icosphere_shell(2, sigma=2e-2, seed=3)
    P = oracle.Problem(sh.rest, sh.faces, oracle.SHELL, 3, params=[E, NU, T])
    a = P.assemble(sh.x, route=0)
    b = P.assemble(sh.x, route=1)
    assert np.isclose(a["energy"], b["energy"], rtol=1e-12)
    assert rel(b["grad"], a["grad"]) < 1e-12
    assert rel(b["vals"], a["vals"]) < 1e-12
    Pb = oracle.Problem(sh.rest, sh.faces, oracle.HINGE, 3, params=[0.7, 1.0])
    a = Pb.assemble(sh.x, route=0)
    b = Pb.assemble(sh.x, route=1)
    assert rel(b["vals"], a["vals"]) < 1e-11


# --------------------------------------------------------------------------
# 7. area (Sec. 7.6, gradient printed in the paper)
# --------------------------------------------------------------------------
def test_area_paper_gradient():
    row = np.loadtxt(os.path.join(GOLDEN, "area_gradient.txt"))
    x, a, g = row[:9], row[9], row[10:]
    cf = oracle.local(oracle.AREA, x, route=1)
    hd = oracle.local(oracle.AREA, x, route=0)
    assert np.isclose(cf["f"], a) and np.allclose(cf["g"], g, atol=1e-15)
    assert np.isclose(hd["f"], a) and np.allclose(hd["g"], g, atol=1e-15)
    xl = RNG.normal(size=9)
    out = local_fd_check(oracle.AREA, xl, 3)
    assert rel(oracle.local(oracle.AREA, xl, route=1)["g"], out["g"]) < 1e-13


# --------------------------------------------------------------------------
# 8. ARAP-style residual (vector-valued term, Eq. 3)
# --------------------------------------------------------------------------
def _arap_one(uv, V):
    F = np.array([[0, 1, 2]], dtype=np.int32)
    P = oracle.Problem(V, F, oracle.ARAP, 2)
    return P, P.arap_jacobian(uv)


def test_arap_rotation_and_scaled_rotation():
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.3, 0.8, 0.0]])
    for phi in (0.0, 0.7, -2.5):
        R = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
        for s in (1.0, 1.7):
            uv = (s * V[:, :2]) @ R.T
            P, out = _arap_one(uv, V)
            expect = np.sqrt(P.area[0]) * (s - 1) * R.ravel()
            assert np.allclose(out["r"], expect, atol=1e-14)


def test_arap_closest_rotation_is_polar_factor():
    V, _, _ = single_triangle_rest()
    uv = RNG.normal(size=(3, 2))
    d1, d2 = uv[1] - uv[0], uv[2] - uv[0]
    if d1[0] * d2[1] - d1[1] * d2[0] < 0:
        uv[[1, 2]] = uv[[2, 1]]
    P, out = _arap_one(uv, V)
    Dm = np.linalg.inv(P.Dinv[0].reshape(2, 2))
    J = np.stack([uv[1] - uv[0], uv[2] - uv[0]], 1) @ np.linalg.inv(Dm)
    U, _, Vt = np.linalg.svd(J)
    R = U @ Vt                                     # polar factor of J (det J > 0)
    assert np.allclose(out["r"], np.sqrt(P.area[0]) * (J - R).ravel(), atol=1e-14)


def test_arap_jacobian_fd():
    V, _, _ = single_triangle_rest()
    uv = np.array([[0.0, 0.1], [1.1, 0.0], [0.2, 0.9]])
    P, out = _arap_one(uv, V)
    Jd = np.zeros((4, 6))
    for p in range(24):
        Jd[p // 6, out["col"][p]] = out["val"][p]
    for r in range(4):
        Jfd = fd_grad(lambda y: _arap_one(y.reshape(3, 2), V)[1]["r"][r], uv.ravel().copy())
        assert rel(Jd[r], Jfd) < 1e-9


# --------------------------------------------------------------------------
# 9. connectivity (hand-enumerated fixtures, icosphere counts)
# --------------------------------------------------------------------------
def _golden_connectivity():
    hinges, nnzb, absent = {}, {}, []
    for line in open(os.path.join(GOLDEN, "connectivity.txt")):
        p = line.split()
        if not p or p[0].startswith("#"):
            continue
        if p[0] == "hinges":
            hinges.setdefault(p[1], []).append([int(v) for v in p[2:]])
        elif p[0] == "nnzb":
            nnzb[(p[1], p[2])] = int(p[3])
        elif p[0] == "absent":
            absent.append((p[1], p[2], int(p[3]), int(p[4])))
    return hinges, nnzb, absent


def test_connectivity_golden():
    tiny = synth.tiny_meshes()
    hinges, nnzb, absent = _golden_connectivity()
    for name, H in hinges.items():
        V, F = tiny[name]
        assert oracle.hinges(V.shape[0], F).tolist() == H
    for (name, kind), n in nnzb.items():
        V, F = tiny[name]
        H = oracle.hinges(V.shape[0], F) if kind == "shell" else None
        rp, col = oracle.pattern(V.shape[0], F, H)
        assert col.shape[0] == n
    for name, kind, i, j in absent:
        V, F = tiny[name]
        rp, col = oracle.pattern(V.shape[0], F)
        assert j not in col[rp[i]:rp[i + 1]]


@pytest.mark.parametrize("level", [0, 1, 2, 3, 4])
def test_icosphere_counts(level):
    V, F = synth.icosphere(level)
    nV, nT = V.shape[0], F.shape[0]
    H = oracle.hinges(nV, F)
    assert nV - 3 * nT // 2 + nT == 2                 # Euler characteristic of S^2
    assert H.shape[0] == 3 * nT // 2                  # closed: every edge interior
    rp, col = oracle.pattern(nV, F)
    assert col.shape[0] == nV + 2 * H.shape[0]        # diagonal + both edge blocks
    if level >= 1:
        rp, col = oracle.pattern(nV, F, H)
        assert col.shape[0] == nV + 4 * H.shape[0]    # + both wing-pair blocks
    for i in range(nV):
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)


def test_hinge_rejects_nonmanifold():
    F = np.array([[0, 1, 2], [1, 0, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.hinges(5, F)
    F = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)     # inconsistent orientation
    with pytest.raises(ValueError):
        oracle.hinges(4, F)


# --------------------------------------------------------------------------
# 10. assembly (Eq. 2): brute-force dense S_j^T H_j S_j, FD, invariances
# --------------------------------------------------------------------------
def _dense_bruteforce(P, x):
    vd = P.vdim
    n = P.nV * vd
    Hd = np.zeros((n, n))
    gd = np.zeros(n)
    f = 0.0
    elems = []
    p = None if P.params is None else list(P.params)
    tri_p = p[:3] if (p is not None and P.energy == oracle.SHELL) else p
    hinge_p = p[3:5] if (p is not None and P.energy == oracle.SHELL) else p
    if P.energy in (oracle.SYMDIR, oracle.STVK, oracle.SHELL, oracle.NH, oracle.AREA):
        te = oracle.STVK if P.energy == oracle.SHELL else P.energy
        for t in range(P.nT):
            elems.append((P.F[t], dict(energy=te, Dinv=P.Dinv[t], area=P.area[t], params=tri_p)))
    if P.energy in (oracle.HINGE, oracle.SHELL):
        for h in range(P.nH):
            elems.append((P.H[h], dict(energy=oracle.HINGE, thetabar=P.thetabar[h],
                                       abar=P.abar[h], params=hinge_p)))
    for vid, kw in elems:
        k = len(vid) * vd
        S = np.zeros((k, n))
        for a, v in enumerate(vid):
            for d in range(vd):
                S[a * vd + d, v * vd + d] = 1.0
        en = kw.pop("energy")
        out = oracle.local(en, S @ x.ravel(), vdim=vd, **kw)
        f += out["f"]
        gd += S.T @ out["g"]
        Hd += S.T @ out["H"] @ S
    return f, gd, Hd


@pytest.mark.parametrize(
    "mesh,energy,vd",
    [("two_triangles", oracle.SYMDIR, 2), ("grid3", oracle.SYMDIR, 2),
     ("tetrahedron", oracle.SHELL, 3), ("icosphere0", oracle.SHELL, 3),
     ("icosphere0", oracle.NH, 3), ("two_triangles", oracle.HINGE, 3),
     ("tetrahedron", oracle.AREA, 3)],
)
def test_assembly_matches_bruteforce(mesh, energy, vd):
    V, F = synth.tiny_meshes()[mesh]
    P = oracle.Problem(V, F, energy, vd, params=[1.0e3, 0.3, 0.01, 2.0, 1.0] if energy == oracle.SHELL else None)
    x = (V[:, :vd] if vd == 2 else V) + RNG.normal(scale=0.03, size=(V.shape[0], vd))
    out = P.assemble(x)
    f, g, Hd = _dense_bruteforce(P, x)
    assert np.isclose(out["energy"], f, rtol=1e-13)
    assert rel(out["grad"].ravel(), g) < 1e-13
    Hb = oracle.bsr_to_dense(P.nV, vd, P.row_ptr, P.col, out["vals"])
    assert rel(Hb, Hd) < 1e-13
    # every structural nonzero of the dense matrix is inside the pattern
    mask = oracle.bsr_to_dense(P.nV, vd, P.row_ptr, P.col, np.ones_like(out["vals"]))
    assert np.all((np.abs(Hd) > 0) <= (mask > 0))


def test_assembled_fd_and_invariances_shell():
    V, F = synth.icosphere(1)
    P = oracle.Problem(V, F, oracle.SHELL, 3, params=[1.0e3, 0.3, 0.01, 0.5, 1.0])
    x = V + RNG.normal(scale=0.02, size=V.shape)
    out = P.assemble(x)
    g = out["grad"]
    Hd = oracle.bsr_to_dense(P.nV, 3, P.row_ptr, P.col, out["vals"])
    energy = lambda y: P.assemble(y.reshape(-1, 3), hessian=False)["energy"]
    idx = RNG.choice(x.size, 12, replace=False)
    for i in idx:
        def fi(s):
            y = x.copy().ravel()
            y[i] += s
            return energy(y)
        h = 1e-5
        d = lambda s: (fi(s) - fi(-s)) / (2 * s)
        assert np.isclose(g.ravel()[i], (4 * d(h / 2) - d(h)) / 3, rtol=1e-7, atol=1e-9)
        def gi(s):
            y = x.copy().ravel()
            y[i] += s
            return P.assemble(y.reshape(-1, 3), hessian=False)["grad"].ravel()
        col_fd = (4 * (gi(h / 4) - gi(-h / 4)) / (h / 2) - (gi(h / 2) - gi(-h / 2)) / h) / 3
        assert rel(Hd[:, i], col_fd) < 1e-6
    assert np.allclose(Hd, Hd.T, atol=1e-12 * np.abs(Hd).max())
    # translation invariance: gradient sums to zero, H annihilates translations
    assert np.abs(g.sum(0)).max() < 1e-12 * np.abs(g).max()
    for d in range(3):
        t = np.zeros_like(x)
        t[:, d] = 1.0
        assert np.abs(Hd @ t.ravel()).max() < 1e-10 * np.abs(Hd).max()
    # rotation invariance: sum of x_v cross g_v vanishes
    assert np.abs(np.cross(x, g).sum(0)).max() < 1e-12 * np.abs(g).max()


def test_symdir_assembled_translation_invariance():
    g = synth.grid_uv()
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    out = P.assemble(g.x)
    assert out["n_domain_err"] == 0
    assert np.abs(out["grad"].sum(0)).max() < 1e-12 * np.abs(out["grad"]).max()
    Hd = oracle.bsr_to_dense(P.nV, 2, P.row_ptr, P.col, out["vals"])
    for d in range(2):
        t = np.zeros((P.nV, 2))
        t[:, d] = 1.0
        assert np.abs(Hd @ t.ravel()).max() < 1e-10 * np.abs(Hd).max()
