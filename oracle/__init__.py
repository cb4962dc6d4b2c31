"""CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never calls it and
shares no code with it (see ``oracle.c`` for what it computes and the paper
passages each function follows).

The C source is compiled on first use with the system C compiler into
``oracle/_build/liboracle.so`` (plain ``-O2``, IEEE arithmetic).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# energy identifiers of the public interface
SYMDIR, STVK, HINGE, SHELL, NH, MLP, AREA, ARAP = 1, 2, 3, 4, 5, 6, 7, 16

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i64, i32, vp = C.c_int64, C.c_int, C.c_void_p
            L.orc_hinges.restype = i64
            L.orc_hinges.argtypes = [i64, i64, _ip, vp]
            L.orc_pattern.restype = i64
            L.orc_pattern.argtypes = [i64, i64, _ip, i64, vp, vp, vp]
            L.orc_tri_rest.restype = None
            L.orc_tri_rest.argtypes = [i64, _dp, _ip, _dp, _dp]
            L.orc_hinge_rest.restype = None
            L.orc_hinge_rest.argtypes = [i64, vp, _dp, vp, vp]
            L.orc_assemble.restype = i64
            L.orc_assemble.argtypes = [
                i32, vp, i32, i32, i64, i32, i64, _ip, _dp, _dp, i64, vp, vp, vp, _dp, _ip, _ip,
                vp, _dp, vp, vp, vp,
            ]
            L.orc_local.restype = i32
            L.orc_local.argtypes = [i32, i32, vp, i32, _dp, i32, _dp, C.c_double, C.c_double,
                                    C.c_double, _dp, _dp, _dp]
            L.orc_hd_flops.restype = i64
            L.orc_hd_flops.argtypes = [i32]
            L.orc_hd_probe.restype = None
            L.orc_hd_probe.argtypes = [i32, _dp, i32, _dp]
            L.orc_invariants_from_F.restype = None
            L.orc_invariants_from_F.argtypes = [i64, _dp, _dp]
            L.orc_nh_targets.restype = None
            L.orc_nh_targets.argtypes = [i64, _dp, vp, i32, _dp, _dp]
            L.orc_mlp_eval.restype = None
            L.orc_mlp_eval.argtypes = [_dp, _dp, i64, _dp, _dp]
            L.orc_mlp_loss.restype = C.c_double
            L.orc_mlp_loss.argtypes = [_dp, _dp, i64, _dp, _dp, _dp, C.c_double, vp]
            L.orc_mlp_set.restype = None
            L.orc_mlp_set.argtypes = [_dp, _dp]
            L.orc_arap_jacobian.restype = i64
            L.orc_arap_jacobian.argtypes = [i64, _ip, _dp, _dp, _dp, _dp, _ip, _ip, _dp]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _params(p):
    return None if p is None or len(p) == 0 else np.ascontiguousarray(p, dtype=np.float64)


# --------------------------------------------------------------------------
# connectivity and rest data
# --------------------------------------------------------------------------
def hinges(nV: int, F: np.ndarray) -> np.ndarray:
    """Canonical hinges (nH, 4) int32: (e0, e1, a, b), e0 < e1, sorted."""
    F = np.ascontiguousarray(F, dtype=np.int32)
    L = lib()
    n = L.orc_hinges(nV, F.shape[0], F, None)
    if n < 0:
        raise ValueError("non-manifold or inconsistently oriented edge")
    H = np.zeros((max(n, 1), 4), dtype=np.int32)
    L.orc_hinges(nV, F.shape[0], F, _ptr(H))
    return H[:n]


def pattern(nV: int, F: np.ndarray, H: np.ndarray | None = None):
    """Brute-force block pattern of the triangle (and hinge) stencils."""
    F = np.ascontiguousarray(F, dtype=np.int32)
    nH = 0 if H is None else int(H.shape[0])
    Hc = None if H is None else np.ascontiguousarray(H, dtype=np.int32)
    L = lib()
    nnzb = L.orc_pattern(nV, F.shape[0], F, nH, _ptr(Hc), None, None)
    row_ptr = np.zeros(nV + 1, dtype=np.int32)
    col = np.zeros(max(nnzb, 1), dtype=np.int32)
    L.orc_pattern(nV, F.shape[0], F, nH, _ptr(Hc), _ptr(row_ptr), _ptr(col))
    return row_ptr, col[:nnzb]


def tri_rest(V: np.ndarray, F: np.ndarray):
    V = np.ascontiguousarray(V, dtype=np.float64)
    F = np.ascontiguousarray(F, dtype=np.int32)
    nT = F.shape[0]
    Dinv = np.zeros((max(nT, 1), 4))
    area = np.zeros(max(nT, 1))
    lib().orc_tri_rest(nT, V, F, Dinv, area)
    return Dinv[:nT], area[:nT]


def hinge_rest(H: np.ndarray, V: np.ndarray):
    V = np.ascontiguousarray(V, dtype=np.float64)
    Hc = np.ascontiguousarray(H, dtype=np.int32)
    n = Hc.shape[0]
    tb = np.zeros(max(n, 1))
    ab = np.zeros(max(n, 1))
    lib().orc_hinge_rest(n, _ptr(Hc), V, _ptr(tb), _ptr(ab))
    return tb[:n], ab[:n]


class Problem:
    """Connectivity, pattern and rest data of one (batched) mesh for one
    energy, built by the oracle's own routines."""

    def __init__(self, rest: np.ndarray, F: np.ndarray, energy: int, vdim: int, params=None):
        self.rest = np.ascontiguousarray(rest, dtype=np.float64)
        self.F = np.ascontiguousarray(F, dtype=np.int32)
        self.nV = int(self.rest.shape[0])
        self.nT = int(self.F.shape[0])
        self.energy = energy
        self.vdim = vdim
        self.params = _params(params)
        self.Dinv, self.area = tri_rest(self.rest, self.F)
        if energy in (HINGE, SHELL):
            self.H = hinges(self.nV, self.F)
            self.thetabar, self.abar = hinge_rest(self.H, self.rest)
        else:
            self.H = np.zeros((0, 4), dtype=np.int32)
            self.thetabar = np.zeros(0)
            self.abar = np.zeros(0)
        self.row_ptr, self.col = pattern(self.nV, self.F, self.H if energy in (HINGE, SHELL) else None)

    @property
    def nH(self) -> int:
        return int(self.H.shape[0])

    @property
    def nnzb(self) -> int:
        return int(self.col.shape[0])

    def n_elements(self) -> int:
        if self.energy == SHELL:
            return self.nT + self.nH
        if self.energy == HINGE:
            return self.nH
        return self.nT

    def assemble(self, x: np.ndarray, route: int = 0, rows: np.ndarray | None = None,
                 hessian: bool = True, per_element: bool = False):
        """Energy, gradient (nV, vdim) and BSR values (nnzb, vdim, vdim).

        rows: optional vertex ids; only those block rows (and gradient rows)
        are assembled, from every element touching them."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.nV, self.vdim)
        vd = self.vdim
        grad = np.zeros((self.nV, vd))
        vals = np.zeros((self.nnzb, vd, vd)) if hessian else None
        mask = None
        if rows is not None:
            mask = np.zeros(self.nV, dtype=np.uint8)
            mask[np.asarray(rows)] = 1
        e = np.zeros(1)
        elem = np.zeros(max(self.n_elements(), 1)) if per_element else None
        nerr = lib().orc_assemble(
            self.energy, _ptr(self.params), 0 if self.params is None else len(self.params), route,
            self.nV, vd, self.nT, self.F, self.Dinv, self.area, self.nH, _ptr(self.H),
            _ptr(self.thetabar), _ptr(self.abar), x, self.row_ptr, self.col, _ptr(mask), e,
            _ptr(grad), _ptr(vals), _ptr(elem))
        if nerr < 0:
            raise RuntimeError(f"oracle assembly error {nerr}")
        out = {"energy": float(e[0]), "grad": grad, "vals": vals, "n_domain_err": int(nerr)}
        if per_element:
            out["elem_energy"] = elem[: self.n_elements()]
        return out

    def hvp(self, x: np.ndarray, v: np.ndarray, route: int = 0):
        """Matrix-free mode (Sec. 5.5 and Sec. 6.2: each element's local
        Hessian applied to its gathered part of v, the products accumulated;
        the CG solver of Sec. 7.2 uses it).  That sum, sum_j S_j^T H_j S_j v,
        is the assembled Hessian of Eq. 2 applied to v, which is what this
        computes: the oracle's BSR values times v, block by block.  Returns
        the energy, the gradient and hv, both (nV, vdim)."""
        out = self.assemble(x, route=route)
        vd = self.vdim
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(self.nV, vd)
        rows = np.repeat(np.arange(self.nV), np.diff(self.row_ptr))
        hv = np.zeros((self.nV, vd))
        np.add.at(hv, rows, np.einsum("bij,bj->bi", out["vals"], v[self.col]))
        return {"energy": out["energy"], "grad": out["grad"], "hv": hv, "n_domain_err": out["n_domain_err"]}

    def assemble_projected(self, x: np.ndarray, eps: float = 0.0):
        """Hessian filtering (Sec. 7.1, after Teran et al. 2005): the local
        Hessian of every element term has its negative eigenvalues set to
        eps (>= 0) before Eq. 2 assembles it; energy and gradient are those
        of assemble().  For the shell, the membrane triangle and the hinge
        are separate terms.  Reading: the term's rigid translations are exact
        zeros of its Hessian, not negative eigenvalues, and stay zero.  A
        Python loop over elements: small meshes only."""
        vd = self.vdim
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(self.nV, vd)
        base = self.assemble(x, hessian=False)
        vals = np.zeros((self.nnzb, vd, vd))

        def scatter(vid, Hl):
            for a, va in enumerate(vid):
                lo, hi = self.row_ptr[va], self.row_ptr[va + 1]
                for b, vb in enumerate(vid):
                    k = lo + int(np.searchsorted(self.col[lo:hi], vb))
                    vals[k] += Hl[a * vd:(a + 1) * vd, b * vd:(b + 1) * vd]

        p = [] if self.params is None else list(self.params)
        if self.energy != HINGE:
            te = STVK if self.energy == SHELL else self.energy
            for t in range(self.nT):
                vid = self.F[t]
                loc = local(te, x[vid], vd, self.Dinv[t], self.area[t], params=p[:3] or None)
                scatter(vid, spd_project(loc["H"], eps, translations(3, vd)))
        if self.energy in (HINGE, SHELL):
            ph = _shell_hinge_params(p) if self.energy == SHELL else (p or None)
            for h in range(self.nH):
                vid = self.H[h]
                loc = local(HINGE, x[vid], 3, thetabar=self.thetabar[h], abar=self.abar[h], params=ph)
                scatter(vid, spd_project(loc["H"], eps, translations(4, 3)))
        return {"energy": base["energy"], "grad": base["grad"], "vals": vals, "n_domain_err": base["n_domain_err"]}

    def arap_jacobian(self, uv: np.ndarray):
        """Residual r (4 nT), CSR Jacobian (row_ptr, col, val)."""
        uv = np.ascontiguousarray(uv, dtype=np.float64).reshape(self.nV, 2)
        nT = self.nT
        r = np.zeros(4 * nT)
        rp = np.zeros(4 * nT + 1, dtype=np.int32)
        jc = np.zeros(24 * nT, dtype=np.int32)
        jv = np.zeros(24 * nT)
        nerr = lib().orc_arap_jacobian(nT, self.F, self.Dinv, self.area, uv, r, rp, jc, jv)
        return {"r": r, "row_ptr": rp, "col": jc, "val": jv, "n_domain_err": int(nerr)}


def local(energy: int, xl, vdim: int = 3, Dinv=None, area: float = 0.0, thetabar: float = 0.0,
          abar: float = 0.0, params=None, route: int = 0):
    """Local f, gradient (k), Hessian (k, k) of one element."""
    xl = np.ascontiguousarray(xl, dtype=np.float64).ravel()
    k = xl.shape[0]
    f = np.zeros(1)
    g = np.zeros(k)
    H = np.zeros(k * k)
    Dinv = np.ascontiguousarray(np.zeros(4) if Dinv is None else Dinv, dtype=np.float64).ravel()
    p = _params(params)
    err = lib().orc_local(energy, route, _ptr(p), 0 if p is None else len(p), xl, vdim, Dinv,
                          float(area), float(thetabar), float(abar), f, g, H)
    if err < 0:
        raise ValueError(f"no route {route} for energy {energy}")
    return {"f": float(f[0]), "g": g, "H": H.reshape(k, k), "err": int(err)}


def dense_flops(energy: int, xl, vdim: int = 3, Dinv=None, area: float = 0.0, thetabar: float = 0.0,
                abar: float = 0.0, params=None) -> int:
    """Scalar floating-point operations of one element's energy, gradient and
    Hessian by dense forward mode (route 0: the paper's ActiveT form, a
    k-gradient and a k x k Hessian carried through every operation), counted
    by the oracle's hyper-dual rules."""
    lib().orc_hd_flops(1)
    local(energy, xl, vdim, Dinv, area, thetabar, abar, params, route=0)
    return int(lib().orc_hd_flops(1))


MLP_NPARAM = 4481


def invariants_from_F(F):
    """(I1, I2, I3) of C3 = diag(F^T F, 1) for F of shape (n, 3, 2)."""
    F = np.ascontiguousarray(F, dtype=np.float64).reshape(-1, 6)
    out = np.zeros((F.shape[0], 3))
    lib().orc_invariants_from_F(F.shape[0], F, out)
    return out


def nh_targets(I, params=None):
    """Neo-Hookean density and its gradient in the invariants."""
    I = np.ascontiguousarray(I, dtype=np.float64).reshape(-1, 3)
    psi = np.zeros(I.shape[0])
    g = np.zeros((I.shape[0], 3))
    p = _params(params)
    lib().orc_nh_targets(I.shape[0], I, _ptr(p), 0 if p is None else len(p), psi, g)
    return psi, g


def mlp_eval(theta, norm, I):
    """(n, 10): psi, dpsi/dI (3), upper Hessian (I1I1, I1I2, I2I2, I1I3, I2I3, I3I3)."""
    I = np.ascontiguousarray(I, dtype=np.float64).reshape(-1, 3)
    out = np.zeros((I.shape[0], 10))
    lib().orc_mlp_eval(np.ascontiguousarray(theta, dtype=np.float64), np.ascontiguousarray(norm, dtype=np.float64),
                       I.shape[0], I, out)
    return out


def mlp_set(theta, norm):
    """Network of the MLP membrane mesh energy (energy id MLP)."""
    lib().orc_mlp_set(np.ascontiguousarray(theta, dtype=np.float64), np.ascontiguousarray(norm, dtype=np.float64))


def mlp_loss(theta, norm, I, psi_t, g_t, beta=1.0, grad=True):
    """Sobolev loss and (optionally) its gradient in theta."""
    I = np.ascontiguousarray(I, dtype=np.float64).reshape(-1, 3)
    gbuf = np.zeros(MLP_NPARAM) if grad else None
    L = lib().orc_mlp_loss(np.ascontiguousarray(theta, dtype=np.float64), np.ascontiguousarray(norm, dtype=np.float64),
                           I.shape[0], I, np.ascontiguousarray(psi_t, dtype=np.float64),
                           np.ascontiguousarray(g_t, dtype=np.float64).reshape(-1), float(beta), _ptr(gbuf))
    return (L, gbuf) if grad else L


def hd_probe(op: int, *inputs):
    n = len(inputs)
    out = np.zeros(1 + n + n * n)
    lib().orc_hd_probe(op, np.asarray(inputs, dtype=np.float64), n, out)
    return out[0], out[1:1 + n], out[1 + n:].reshape(n, n)


SPD_TAU = 1e-10  # an eigenvalue is negative below -SPD_TAU * max |eigenvalue|


def spd_project(H: np.ndarray, eps: float = 0.0, keep=None, tau: float = SPD_TAU) -> np.ndarray:
    """A symmetric matrix with its negative eigenvalues set to eps (the
    per-term Hessian filtering of Sec. 7.1): Q max'(L) Q^T from eigh.

    An eigenvalue counts as negative below -tau max|lambda| (reading: a
    term's structural zeros, which round-off puts on either side of zero,
    are not negative; every hinge term has one besides its translations).

    keep: optional (n, m) orthonormal columns spanning exact null directions
    of H that must stay null (a term's translations).  The spectrum is then
    taken on their orthogonal complement only, so round-off in those exact
    zeros cannot turn them into clamped 'negative' eigenvalues."""
    Hs = 0.5 * (H + H.T)
    if keep is None:
        lam, Q = np.linalg.eigh(Hs)
        lam = np.where(lam < -tau * np.abs(lam).max(), eps, lam)
        return (Q * lam) @ Q.T
    n = Hs.shape[0]
    U, _, _ = np.linalg.svd(keep, full_matrices=True)
    B = U[:, keep.shape[1]:]                      # orthonormal complement
    lam, Q = np.linalg.eigh(B.T @ Hs @ B)
    lam = np.where(lam < -tau * np.abs(lam).max(), eps, lam)
    W = B @ Q
    return (W * lam) @ W.T


def translations(nv: int, vd: int) -> np.ndarray:
    """Orthonormal basis (nv vd, vd) of rigid translations of nv vertices."""
    T = np.zeros((nv * vd, vd))
    for d in range(vd):
        T[d::vd, d] = 1.0 / np.sqrt(nv)
    return T


def _shell_hinge_params(p):
    """Hinge parameters {k_b, h} of a shell parameter list {E, nu, t, k_b, h}
    (the same defaults as the membrane: k_b = E t^3 / (12 (1 - nu^2)), h = 1)."""
    E = p[0] if len(p) > 0 else 1.0e5
    nu = p[1] if len(p) > 1 else 0.3
    t = p[2] if len(p) > 2 else 1.0e-3
    kb = p[3] if len(p) > 3 and p[3] >= 0 else E * t ** 3 / (12.0 * (1.0 - nu * nu))
    h = p[4] if len(p) > 4 else 1.0
    return [kb, h]


def bsr_to_dense(nV: int, vd: int, row_ptr, col, vals) -> np.ndarray:
    """Dense (nV*vd)^2 matrix of a BSR matrix (tiny meshes only)."""
    Hd = np.zeros((nV * vd, nV * vd))
    for i in range(nV):
        for p in range(row_ptr[i], row_ptr[i + 1]):
            j = col[p]
            Hd[i * vd:(i + 1) * vd, j * vd:(j + 1) * vd] += vals[p]
    return Hd


# --------------------------------------------------------------------------
# mass-spring cloth (Sec. 7.1): per-edge springs, per-vertex inertia and
# gravity, written out from their definitions with numpy
# --------------------------------------------------------------------------
CLOTH = 8


def mesh_edges(F: np.ndarray) -> np.ndarray:
    """Unique undirected edges (min, max) of a triangle list, sorted."""
    F = np.asarray(F, dtype=np.int64)
    e = np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]])
    e.sort(axis=1)
    return np.unique(e, axis=0)


def lumped_mass(rest: np.ndarray, F: np.ndarray, rho: float) -> np.ndarray:
    """Lumped (diagonal) mass: each vertex gets a third of the rest area of
    every triangle around it, times the areal density rho."""
    rest = np.asarray(rest, dtype=np.float64)
    F = np.asarray(F, dtype=np.int64)
    a = 0.5 * np.linalg.norm(np.cross(rest[F[:, 1]] - rest[F[:, 0]], rest[F[:, 2]] - rest[F[:, 0]]), axis=1)
    m = np.zeros(rest.shape[0])
    for c in range(3):
        np.add.at(m, F[:, c], rho * a / 3.0)
    return m


def cloth_params(p=None):
    """{k, h, rho, gx, gy, gz}: spring stiffness, time step, areal density,
    gravity; defaults 1e4, 1/60, 1, (0, 0, -9.81)."""
    d = [1.0e4, 1.0 / 60.0, 1.0, 0.0, 0.0, -9.81]
    p = [] if p is None else list(p)
    return [p[i] if i < len(p) else d[i] for i in range(6)]


def cloth_assemble(rest, F, x, xhat, params=None, row_ptr=None, col=None, project=False, eps=0.0):
    """Implicit-Euler cloth energy of Sec. 7.1 and its derivatives:
        E(x) = sum_v m_v/2 |x_v - xhat_v|^2 + h^2 ( sum_e P_e(x) - sum_v m_v g.x_v ),
        P_e = l^2 k/2 (|x_i - x_j|^2 / l^2 - 1)^2  (edge e = (i, j), rest length l).
    Returns energy, gradient (nV, 3) and, given the block pattern, the BSR
    values of the Hessian (3x3 blocks).  With project, every spring's
    local Hessian is filtered as in Problem.assemble_projected (the vertex
    terms' m_v I needs none)."""
    k, h, rho = cloth_params(params)[:3]
    g = np.asarray(cloth_params(params)[3:6])
    rest = np.asarray(rest, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    xhat = np.asarray(xhat, dtype=np.float64).reshape(-1, 3)
    nV = x.shape[0]
    E = mesh_edges(F)
    m = lumped_mass(rest, F, rho)
    i, j = E[:, 0], E[:, 1]
    l2 = np.sum((rest[i] - rest[j]) ** 2, axis=1)
    d = x[i] - x[j]
    s = np.sum(d * d, axis=1) / l2
    energy = np.sum(0.5 * m * np.sum((x - xhat) ** 2, axis=1)) \
        + h * h * (np.sum(0.5 * k * l2 * (s - 1.0) ** 2) - np.sum(m * (x @ g)))
    gs = (h * h * 2.0 * k * (s - 1.0))[:, None] * d
    grad = m[:, None] * (x - xhat) - h * h * m[:, None] * g[None, :]
    np.add.at(grad, i, gs)
    np.add.at(grad, j, -gs)
    out = {"energy": float(energy), "grad": grad}
    if row_ptr is None:
        return out
    I3 = np.eye(3)
    A = h * h * (2.0 * k * (s - 1.0))[:, None, None] * I3 + h * h * (4.0 * k / l2)[:, None, None] * \
        d[:, :, None] * d[:, None, :]
    if project:
        T = translations(2, 3)
        loc = np.zeros((len(E), 6, 6))
        for q in range(len(E)):
            L = np.block([[A[q], -A[q]], [-A[q], A[q]]])
            loc[q] = spd_project(L, eps, T)
        Aii, Ajj, Aij = loc[:, :3, :3], loc[:, 3:, 3:], loc[:, :3, 3:]
    else:
        Aii, Ajj, Aij = A, A, -A
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    keys = np.repeat(np.arange(nV), np.diff(row_ptr)) * nV + col

    def blk(r, c):
        return np.searchsorted(keys, np.asarray(r) * nV + np.asarray(c))

    vals = np.zeros((col.shape[0], 3, 3))
    np.add.at(vals, blk(np.arange(nV), np.arange(nV)), m[:, None, None] * I3)
    np.add.at(vals, blk(i, i), Aii)
    np.add.at(vals, blk(j, j), Ajj)
    np.add.at(vals, blk(i, j), Aij)
    np.add.at(vals, blk(j, i), np.transpose(Aij, (0, 2, 1)))
    out["vals"] = vals
    return out


# --------------------------------------------------------------------------
# interaction terms over vertex pairs (Sec. 4.3; the contact barrier of
# Sec. 7.7) and the pattern they extend (Sec. 6.3, Alg. 1)
# --------------------------------------------------------------------------
def contact_vv(xi, xj, kappa: float, dhat: float, area: float, h: float):
    """Vertex-vertex barrier of Sec. 7.7:
        E(d) = kappa/2 dhat A_c (s - 1) ln(s) h^2,  s = d / dhat,  for d < dhat,
    0 otherwise, d = |x_i - x_j|.  Returns f, gradient (6) and Hessian (6, 6)
    over (x_i, x_j), from the scalar derivatives of E in d and the chain rule
    through d = |x_i - x_j|."""
    xi = np.asarray(xi, dtype=np.float64)
    xj = np.asarray(xj, dtype=np.float64)
    r = xi - xj
    d = float(np.linalg.norm(r))
    g = np.zeros(6)
    H = np.zeros((6, 6))
    if not (d < dhat) or d == 0.0:
        return 0.0, g, H
    c = 0.5 * kappa * area * h * h
    s = d / dhat
    f = c * dhat * (s - 1.0) * np.log(s)
    e1 = c * (np.log(s) + (s - 1.0) / s)               # dE/dd
    e2 = c / dhat * (1.0 / s + 1.0 / (s * s))          # d2E/dd2
    u = r / d
    gd = e1 * u
    Hd = e2 * np.outer(u, u) + (e1 / d) * (np.eye(3) - np.outer(u, u))
    g[:3], g[3:] = gd, -gd
    H[:3, :3], H[3:, 3:], H[:3, 3:], H[3:, :3] = Hd, Hd, -Hd, -Hd
    return f, g, H


def quad_pairs(quads) -> np.ndarray:
    """The six unordered vertex pairs of every vertex-face element (p, a, b, c):
    the off-diagonal blocks its Hessian touches."""
    q = np.asarray(quads, dtype=np.int64).reshape(-1, 4)
    return np.asarray([(t[i], t[j]) for t in q for i in range(4) for j in range(i + 1, 4)],
                      dtype=np.int64).reshape(-1, 2)


def extended_pattern(row_ptr, col, pairs, quads=()):
    """Block pattern with the blocks of interaction terms added (Alg. 1 inserts
    the new (i, j) and (j, i) entries): per row, the original columns in their
    order, then the new columns ascending, each once.  The blocks are those of
    the vertex pairs and of the six vertex pairs of every vertex-face element;
    blocks already in the pattern add nothing.  Returns (row_ptr, col)."""
    nV = len(row_ptr) - 1
    rows = [list(col[row_ptr[r]:row_ptr[r + 1]]) for r in range(nV)]
    extra = [set() for _ in range(nV)]
    allp = np.concatenate([np.asarray(pairs, dtype=np.int64).reshape(-1, 2), quad_pairs(quads)])
    for i, j in allp:
        if j not in rows[i]:
            extra[i].add(int(j))
            extra[j].add(int(i))
    rp = [0]
    out = []
    for r in range(nV):
        out.extend(rows[r])
        out.extend(sorted(extra[r]))
        rp.append(len(out))
    return np.asarray(rp, dtype=np.int64), np.asarray(out, dtype=np.int64)


def add_interactions(base, x, pairs, kappa, dhat, area, h, row_ptr, col, quads=(), project=False, eps=0.0):
    """Energy, gradient and Hessian blocks {(row, col): 3x3} of a mesh energy
    (base: energy, grad, vals over the pattern row_ptr, col) plus a
    vertex-vertex barrier per pair and a vertex-face barrier per element
    (p, a, b, c), assembled by their plain definition.  project: each
    term's Hessian filtered first (spd_project, translations kept null)."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    energy = base["energy"]
    grad = np.array(base["grad"], dtype=np.float64)
    blocks = {}
    for r in range(len(row_ptr) - 1):
        for k in range(row_ptr[r], row_ptr[r + 1]):
            blocks[(r, int(col[k]))] = np.array(base["vals"][k])
    terms = [(contact_vv(x[i], x[j], kappa, dhat, area, h), (int(i), int(j)))
             for i, j in np.asarray(pairs, dtype=np.int64).reshape(-1, 2)]
    terms += [(contact_vf(x[t[0]], x[t[1]], x[t[2]], x[t[3]], kappa, dhat, area, h), tuple(int(v) for v in t))
              for t in np.asarray(quads, dtype=np.int64).reshape(-1, 4)]
    for (f, g, H), verts in terms:
        if project and f != 0.0:
            H = spd_project(H, eps, keep=translations(len(verts), 3))
        energy += f
        for a, va in enumerate(verts):
            grad[va] += g[3 * a:3 * a + 3]
            for b, vb in enumerate(verts):
                blk = blocks.setdefault((va, vb), np.zeros((3, 3)))
                blk += H[3 * a:3 * a + 3, 3 * b:3 * b + 3]
    return {"energy": energy, "grad": grad, "blocks": blocks}


# --------------------------------------------------------------------------
# per-vertex one-ring term: uniform-Laplacian (umbrella) smoothing
# --------------------------------------------------------------------------
UMBRELLA = 9


def vertex_rings(nV: int, F) -> list:
    """Edge-adjacent neighbours of every vertex, ascending."""
    nb = [set() for _ in range(nV)]
    for f in np.asarray(F, dtype=np.int64):
        for c in range(3):
            a, b = int(f[c]), int(f[(c + 1) % 3])
            nb[a].add(b)
            nb[b].add(a)
    return [sorted(s) for s in nb]


def ring_pattern(nV: int, F):
    """Block pattern of one-ring terms: every pair of vertices of a closed
    one-ring {v} + N(v), as (row_ptr, col) with columns ascending."""
    rings = vertex_rings(nV, F)
    rows = [set([r]) for r in range(nV)]
    for v in range(nV):
        R = [v] + rings[v]
        for a in R:
            rows[a].update(R)
    rp, col = [0], []
    for r in range(nV):
        col.extend(sorted(rows[r]))
        rp.append(len(col))
    return np.asarray(rp, dtype=np.int64), np.asarray(col, dtype=np.int64)


def umbrella_assemble(F, x, w: float = 1.0, row_ptr=None, col=None):
    """sum_v w/2 |x_v - (1/k_v) sum_{u in N(v)} x_u|^2 (k_v the valence;
    vertices without neighbours contribute nothing), its gradient and, given
    the pattern, its BSR Hessian: with c = (1, -1/k, .., -1/k) over the
    closed ring, the term's Hessian is w c c^T per coordinate."""
    x = np.asarray(x, dtype=np.float64)
    nV, vd = x.shape
    rings = vertex_rings(nV, F)
    energy = 0.0
    grad = np.zeros_like(x)
    vals = None if row_ptr is None else np.zeros((len(col), vd, vd))
    for v in range(nV):
        k = len(rings[v])
        if k == 0:
            continue
        R = [v] + rings[v]
        c = np.array([1.0] + [-1.0 / k] * k)
        L = c @ x[R]
        energy += 0.5 * w * float(L @ L)
        for a, va in enumerate(R):
            grad[va] += w * c[a] * L
        if vals is not None:
            for a, va in enumerate(R):
                lo, hi = row_ptr[va], row_ptr[va + 1]
                for b, vb in enumerate(R):
                    kk = lo + int(np.searchsorted(col[lo:hi], vb))
                    vals[kk] += w * c[a] * c[b] * np.eye(vd)
    out = {"energy": energy, "grad": grad}
    if vals is not None:
        out["vals"] = vals
    return out


# --------------------------------------------------------------------------
# vertex-face contact (the second interaction term of Sec. 7.7), on a small
# dense hyper-dual number in numpy: value, gradient and Hessian over n seeds
# --------------------------------------------------------------------------
class HD:
    """Dense second-order forward-mode number (slow; tiny cases only)."""

    def __init__(self, v, g, H):
        self.v, self.g, self.H = float(v), np.asarray(g, dtype=np.float64), np.asarray(H, dtype=np.float64)

    @staticmethod
    def var(v, i, n):
        g = np.zeros(n)
        g[i] = 1.0
        return HD(v, g, np.zeros((n, n)))

    def _wrap(self, o):
        return o if isinstance(o, HD) else HD(o, np.zeros_like(self.g), np.zeros_like(self.H))

    def __add__(self, o):
        o = self._wrap(o)
        return HD(self.v + o.v, self.g + o.g, self.H + o.H)

    __radd__ = __add__

    def __neg__(self):
        return HD(-self.v, -self.g, -self.H)

    def __sub__(self, o):
        return self + (-self._wrap(o))

    def __rsub__(self, o):
        return self._wrap(o) - self

    def __mul__(self, o):
        o = self._wrap(o)
        return HD(self.v * o.v, self.v * o.g + o.v * self.g,
                  self.v * o.H + o.v * self.H + np.outer(self.g, o.g) + np.outer(o.g, self.g))

    __rmul__ = __mul__

    def chain(self, f, f1, f2):
        return HD(f, f1 * self.g, f1 * self.H + f2 * np.outer(self.g, self.g))

    def recip(self):
        return self.chain(1.0 / self.v, -1.0 / self.v ** 2, 2.0 / self.v ** 3)

    def __truediv__(self, o):
        return self * self._wrap(o).recip()

    def sqrt(self):
        r = np.sqrt(self.v)
        return self.chain(r, 0.5 / r, -0.25 / (r * self.v))

    def log(self):
        return self.chain(np.log(self.v), 1.0 / self.v, -1.0 / self.v ** 2)


def _dot(u, w):
    return u[0] * w[0] + u[1] * w[1] + u[2] * w[2]


def _cross(u, w):
    return [u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]]


def closest_region(p, a, b, c):
    """Where on triangle (a, b, c) the point closest to p lies: ('v', k) for
    vertex k, ('e', k, l) for the edge from vertex k to vertex l, ('f',) for
    the interior; by the signs of the barycentric-style dot products of the
    standard closest-point construction (Voronoi regions of the triangle)."""
    p, a, b, c = (np.asarray(z, dtype=np.float64) for z in (p, a, b, c))
    ab, ac, ap = b - a, c - a, p - a
    d1, d2 = ab @ ap, ac @ ap
    if d1 <= 0 and d2 <= 0:
        return ("v", 0)
    bp = p - b
    d3, d4 = ab @ bp, ac @ bp
    if d3 >= 0 and d4 <= d3:
        return ("v", 1)
    vc = d1 * d4 - d3 * d2
    if vc <= 0 and d1 >= 0 and d3 <= 0:
        return ("e", 0, 1)
    cp = p - c
    d5, d6 = ab @ cp, ac @ cp
    if d6 >= 0 and d5 <= d6:
        return ("v", 2)
    vb = d5 * d2 - d1 * d6
    if vb <= 0 and d2 >= 0 and d6 <= 0:
        return ("e", 0, 2)
    va = d3 * d6 - d5 * d4
    if va <= 0 and (d4 - d3) >= 0 and (d5 - d6) >= 0:
        return ("e", 1, 2)
    return ("f",)


def contact_vf(p, a, b, c, kappa: float, dhat: float, area: float, h: float):
    """Vertex-face barrier of Sec. 7.7 on (p, a, b, c): the printed energy
    kappa/2 dhat A_c (s - 1) ln(s) h^2, s = d / dhat < 1, d the distance from
    p to the triangle, A_c the given (rest) face area.  The squared distance
    is written per closest-point region (vertex, edge, interior) and
    differentiated by the dense hyper-dual number.  Returns f, g (12), H (12, 12)."""
    X = np.concatenate([np.asarray(z, dtype=np.float64) for z in (p, a, b, c)])
    P = [HD.var(X[k], k, 12) for k in range(12)]
    pts = [P[0:3], P[3:6], P[6:9], P[9:12]]            # p, a, b, c
    reg = closest_region(p, a, b, c)
    if reg[0] == "v":
        r = [pts[0][i] - pts[1 + reg[1]][i] for i in range(3)]
        q = _dot(r, r)
    elif reg[0] == "e":
        u, w = pts[1 + reg[1]], pts[1 + reg[2]]
        r = [pts[0][i] - u[i] for i in range(3)]
        e = [w[i] - u[i] for i in range(3)]
        q = _dot(r, r) - _dot(r, e) * _dot(r, e) / _dot(e, e)
    else:
        e1 = [pts[2][i] - pts[1][i] for i in range(3)]
        e2 = [pts[3][i] - pts[1][i] for i in range(3)]
        r = [pts[0][i] - pts[1][i] for i in range(3)]
        n = _cross(e1, e2)
        q = _dot(n, r) * _dot(n, r) / _dot(n, n)
    if not (q.v < dhat * dhat) or q.v <= 0.0:
        return 0.0, np.zeros(12), np.zeros((12, 12))
    s = q.sqrt() * (1.0 / dhat)
    E = (s - 1.0) * s.log() * (0.5 * kappa * area * h * h * dhat)
    return E.v, E.g, E.H


def vf_distance(p, a, b, c) -> float:
    """Distance from p to triangle (a, b, c) by the same region formulas as
    contact_vf (plain floats)."""
    reg = closest_region(p, a, b, c)
    p, a, b, c = (np.asarray(z, dtype=np.float64) for z in (p, a, b, c))
    pts = [a, b, c]
    if reg[0] == "v":
        return float(np.linalg.norm(p - pts[reg[1]]))
    if reg[0] == "e":
        u, w = pts[reg[1]], pts[reg[2]]
        r, e = p - u, w - u
        return float(np.sqrt(max(r @ r - (r @ e) ** 2 / (e @ e), 0.0)))
    n = np.cross(b - a, c - a)
    return float(abs(n @ (p - a)) / np.linalg.norm(n))
