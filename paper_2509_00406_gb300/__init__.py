"""Python binding of libadm (C ABI in include/adm.h).

Argument marshalling only: every step of the differentiation and assembly
runs in the library's sm_103a kernels.  Device memory and streams come from
PyTorch; buffers are passed to the library as raw pointers.

The shared library is built in-tree by ``__graft_entry__.build()`` (or
``paper_2509_00406_gb300._build.build()``).  If it is missing, ``lib()``
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB_PATH = os.path.join(HERE, "_build", "libadm.so")
HEADER = os.path.join(ROOT, "include", "adm.h")

# adm_energy
SYMDIR2D, STVK_MEMBRANE, HINGE_BENDING, SHELL, NH_MEMBRANE, MLP_MEMBRANE, AREA = 1, 2, 3, 4, 5, 6, 7
ARAP2D_RESIDUAL = 16
MASS_SPRING = 8
UMBRELLA = 9
# adm_precision
FP64, FP32 = 0, 1
# adm_option
OPT_ASSEMBLER, OPT_TILE_TRIS, OPT_BLOCK_THREADS, OPT_PROFILE, OPT_GRAPH, OPT_TILE_THREADS, OPT_MLP_NET = 1, 2, 3, 4, 5, 6, 7
# adm_stage
STAGES = ["zero", "triangles", "hinges", "gnorm", "finalize", "tiled", "graph", "mlp", "pairs"]
MLP_NPARAM = 4481

STATUS = {0: "ADM_OK", -1: "ADM_ERR_ARG", -2: "ADM_ERR_MESH", -3: "ADM_ERR_DOMAIN",
          -4: "ADM_ERR_CUDA", -5: "ADM_ERR_TIMEOUT", -6: "ADM_ERR_OOM", -7: "ADM_ERR_UNSUPPORTED"}

_lib = None


class AdmError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)}")


def declared_functions() -> list[str]:
    """Names of the functions declared in include/adm.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(adm_[a-z_0-9]+)\s*\(", txt)))


def lib():
    """Load libadm.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    i32, i64, vp, dp = C.c_int32, C.c_int64, C.c_void_p, C.POINTER(C.c_double)
    pp = C.POINTER(C.c_void_p)
    sig = {
        "adm_create": (i32, [vp, i64, vp, i64, i32, pp]),
        "adm_create_batch": (i32, [vp, vp, vp, vp, i32, i32, pp]),
        "adm_set_params": (i32, [vp, i32, vp, i32]),
        "adm_set_option": (i32, [vp, i32, i64]),
        "adm_pattern": (i32, [vp, i32, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64), pp, pp]),
        "adm_jac_pattern": (i32, [vp, i32, C.POINTER(i64), C.POINTER(i64), C.POINTER(i64), pp, pp]),
        "adm_hinges": (i32, [vp, pp, C.POINTER(i64)]),
        "adm_slot_map": (i32, [vp, i32, pp, C.POINTER(i64)]),
        "adm_eval": (i32, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "adm_eval_hvp": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp]),
        "adm_set_projection": (i32, [vp, i32, C.c_double]),
        "adm_set_inertia_target": (i32, [vp, vp]),
        "adm_set_interactions": (i32, [vp, i32, vp, i64, C.c_double, C.c_double, C.c_double, C.c_double, vp]),
        "adm_set_contacts": (i32, [vp, i32, vp, i64, vp, i64, C.c_double, C.c_double, C.c_double, C.c_double, vp]),
        "adm_eval_batch": (i32, [vp, i32, i32, vp, vp, vp, vp, vp, vp]),
        "adm_eval_batch_host": (i32, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "adm_eval_jacobian": (i32, [vp, i32, i32, vp, vp, vp, vp, vp]),
        "adm_get_status": (i32, [vp]),
        "adm_profile_read": (i32, [vp, C.POINTER(C.c_float), C.POINTER(i32), i32]),
        "adm_grad_norm_noalloc": (i32, [vp, i64, i32, vp, vp]),
        "adm_check_bounded_wait": (i32, [vp]),
        "adm_autotune": (i32, [vp, i32, i32, vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_float)]),
        "adm_mlp_eval": (i32, [vp, vp, i64, vp, vp, vp]),
        "adm_mlp_workspace_size": (C.c_size_t, []),
        "adm_mlp_loss_grad": (i32, [vp, vp, i64, vp, vp, vp, C.c_float, vp, vp, vp, C.c_size_t, vp]),
        "adm_mlp_adam": (i32, [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, vp]),
        "adm_mlp_nh_targets": (i32, [i64, vp, C.c_double, C.c_double, vp, vp, vp, vp]),
        "adm_mlp_attach": (i32, [vp, vp, vp]),
        "adm_strerror": (C.c_char_p, [i32]),
        "adm_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != 0:
        raise AdmError(status, where)


def _ptr(t):
    """Raw pointer of a torch tensor / numpy array / None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return C.c_void_p(t.data_ptr())
    return t.ctypes.data_as(C.c_void_p)


class _DevView:
    """__cuda_array_interface__ view of library-owned device memory."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False),
                                         "version": 3}


def _dev_copy(ptr, n: int, typestr: str = "<i4"):
    import torch
    if n == 0:
        return torch.zeros(0, dtype=torch.int32, device="cuda")
    return torch.as_tensor(_DevView(int(ptr), int(n), typestr), device="cuda").clone()


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


class Mesh:
    """A libadm handle over one mesh or a batch of meshes."""

    def __init__(self, rest, faces, var_dim: int = 3, v_off=None, f_off=None):
        L = lib()
        rest = np.ascontiguousarray(rest, dtype=np.float64)
        faces = np.ascontiguousarray(faces, dtype=np.int32)
        self.var_dim = int(var_dim)
        self.nV = int(rest.shape[0])
        self.nT = int(faces.shape[0])
        h = C.c_void_p()
        if v_off is None:
            _check(L.adm_create(_ptr(rest), self.nV, _ptr(faces), self.nT, self.var_dim, C.byref(h)),
                   "adm_create")
            self.n_mesh = 1
        else:
            vo = np.ascontiguousarray(v_off, dtype=np.int64)
            fo = np.ascontiguousarray(f_off, dtype=np.int64)
            self.n_mesh = int(vo.shape[0] - 1)
            _check(L.adm_create_batch(_ptr(rest), _ptr(vo), _ptr(faces), _ptr(fo), self.n_mesh,
                                      self.var_dim, C.byref(h)), "adm_create_batch")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().adm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- configuration ---------------------------------------------------
    def set_params(self, energy: int, params):
        p = np.ascontiguousarray(params, dtype=np.float64)
        _check(lib().adm_set_params(self._h, energy, _ptr(p), int(p.shape[0])), "adm_set_params")

    def set_option(self, option: int, value: int):
        _check(lib().adm_set_option(self._h, option, int(value)), "adm_set_option")

    # -- patterns --------------------------------------------------------
    def pattern(self, energy: int):
        """(block, n_rows, nnzb, row_ptr, col) with row_ptr/col as int32 cuda tensors."""
        b, nr, nz = C.c_int32(), C.c_int64(), C.c_int64()
        rp, col = C.c_void_p(), C.c_void_p()
        _check(lib().adm_pattern(self._h, energy, C.byref(b), C.byref(nr), C.byref(nz), C.byref(rp),
                                 C.byref(col)), "adm_pattern")
        return (b.value, nr.value, nz.value, _dev_copy(rp.value, nr.value + 1),
                _dev_copy(col.value, nz.value))

    def jac_pattern(self, energy: int = ARAP2D_RESIDUAL):
        nr, nc, nz = C.c_int64(), C.c_int64(), C.c_int64()
        rp, col = C.c_void_p(), C.c_void_p()
        _check(lib().adm_jac_pattern(self._h, energy, C.byref(nr), C.byref(nc), C.byref(nz), C.byref(rp),
                                     C.byref(col)), "adm_jac_pattern")
        return nr.value, nc.value, nz.value, _dev_copy(rp.value, nr.value + 1), _dev_copy(col.value, nz.value)

    def hinges(self):
        p, n = C.c_void_p(), C.c_int64()
        _check(lib().adm_hinges(self._h, C.byref(p), C.byref(n)), "adm_hinges")
        return _dev_copy(p.value, 4 * n.value).reshape(-1, 4)

    def slot_map(self, energy: int):
        p, n = C.c_void_p(), C.c_int64()
        _check(lib().adm_slot_map(self._h, energy, C.byref(p), C.byref(n)), "adm_slot_map")
        return _dev_copy(p.value, n.value)

    # -- evaluation --------------------------------------------------------
    def eval(self, energy: int, prec: int, x, energy_out=None, grad=None, bsr=None, stream=None):
        _check(lib().adm_eval(self._h, energy, prec, _ptr(x), _ptr(energy_out), _ptr(grad), _ptr(bsr),
                              _stream(stream)), "adm_eval")

    def set_interactions(self, energy: int, pairs, kappa: float, dhat: float, area: float, h: float = 1.0,
                         stream=None):
        """Vertex-pair contact terms (device or host int32 (n, 2)) for the
        pattern of `energy`; n = 0 clears them.  The block pattern changes:
        query pattern() again."""
        n = 0 if pairs is None else int(pairs.shape[0])
        _check(lib().adm_set_interactions(self._h, energy, _ptr(pairs) if n else None, n, float(kappa),
                                          float(dhat), float(area), float(h), _stream(stream)),
               "adm_set_interactions")

    def set_contacts(self, energy: int, pairs, vf, kappa: float, dhat: float, area: float, h: float = 1.0,
                     stream=None):
        """Vertex-vertex (int32 (n, 2)) and vertex-face (int32 (m, 4): p, a, b,
        c) contact terms, device or host, for the pattern of `energy`; None
        or empty arrays for none.  The block pattern changes: query
        pattern() again."""
        n = 0 if pairs is None else int(pairs.shape[0])
        m = 0 if vf is None else int(vf.shape[0])
        _check(lib().adm_set_contacts(self._h, energy, _ptr(pairs) if n else None, n, _ptr(vf) if m else None, m,
                                      float(kappa), float(dhat), float(area), float(h), _stream(stream)),
               "adm_set_contacts")

    def set_inertia_target(self, xhat):
        """Inertial target of the mass-spring energy (host, (nV, 3), copied)."""
        xhat = np.ascontiguousarray(xhat, dtype=np.float64)
        _check(lib().adm_set_inertia_target(self._h, _ptr(xhat)), "adm_set_inertia_target")

    def set_projection(self, enable: bool, eps: float = 0.0):
        """Hessian filtering: negative local eigenvalues set to eps before assembly."""
        _check(lib().adm_set_projection(self._h, int(bool(enable)), float(eps)), "adm_set_projection")

    def eval_hvp(self, energy: int, prec: int, x, v, hv, energy_out=None, grad=None, stream=None):
        """Matrix-free H(x) v into hv (with the energy and, optionally, the gradient)."""
        _check(lib().adm_eval_hvp(self._h, energy, prec, _ptr(x), _ptr(v), _ptr(energy_out), _ptr(grad),
                                  _ptr(hv), _stream(stream)), "adm_eval_hvp")

    def eval_batch(self, energy: int, prec: int, x, energy_per_mesh=None, gnorm=None, grad=None,
                   bsr=None, stream=None):
        _check(lib().adm_eval_batch(self._h, energy, prec, _ptr(x), _ptr(energy_per_mesh), _ptr(gnorm),
                                    _ptr(grad), _ptr(bsr), _stream(stream)), "adm_eval_batch")

    def eval_batch_host(self, energy: int, prec: int, x_host, energy_per_mesh=None, gnorm=None,
                        grad=None, bsr=None):
        _check(lib().adm_eval_batch_host(self._h, energy, prec, _ptr(x_host), _ptr(energy_per_mesh),
                                         _ptr(gnorm), _ptr(grad), _ptr(bsr)), "adm_eval_batch_host")

    def eval_jacobian(self, energy: int, prec: int, x, r, jac_vals=None, jtj=None, stream=None):
        _check(lib().adm_eval_jacobian(self._h, energy, prec, _ptr(x), _ptr(r), _ptr(jac_vals), _ptr(jtj),
                                       _stream(stream)), "adm_eval_jacobian")

    def autotune(self, energy: int, prec: int, x):
        """(best units per tile, best threads per block, ms per pass) of the
        tiled assembler on x."""
        best, thr, ms = C.c_int32(), C.c_int32(), C.c_float()
        _check(lib().adm_autotune(self._h, energy, prec, _ptr(x), C.byref(best), C.byref(thr), C.byref(ms)),
               "adm_autotune")
        return best.value, thr.value, ms.value

    def mlp_attach(self, theta, norm):
        _check(lib().adm_mlp_attach(self._h, _ptr(theta), _ptr(norm)), "adm_mlp_attach")

    def profile_read(self) -> dict:
        """{stage: (average ms per launch, launches)} since the last read."""
        n = len(STAGES)
        ms = (C.c_float * n)()
        cnt = (C.c_int32 * n)()
        _check(lib().adm_profile_read(self._h, ms, cnt, n), "adm_profile_read")
        return {STAGES[k]: (float(ms[k]), int(cnt[k])) for k in range(n)}

    def status(self) -> int:
        return int(lib().adm_get_status(self._h))


def check_bounded_wait(stream=None) -> int:
    """Run the library's bounded device wait on a barrier nothing completes;
    returns the status (ADM_ERR_TIMEOUT, -5, when the wait gave up as it must)."""
    return int(lib().adm_check_bounded_wait(_stream(stream)))


def grad_norm_noalloc(v, prec: int, norm_out, stream=None):
    """FP64 2-norm of a device vector into norm_out (device double); the call
    allocates nothing (see adm_grad_norm_noalloc in include/adm.h)."""
    _check(lib().adm_grad_norm_noalloc(_ptr(v), int(v.numel()), prec, _ptr(norm_out), _stream(stream)),
           "adm_grad_norm_noalloc")


class MLP:
    """The learned membrane network's calls (device tensors in and out)."""

    @staticmethod
    def eval(theta, norm, I, out, stream=None):
        _check(lib().adm_mlp_eval(_ptr(theta), _ptr(norm), I.shape[0], _ptr(I), _ptr(out), _stream(stream)),
               "adm_mlp_eval")

    @staticmethod
    def workspace_size() -> int:
        return int(lib().adm_mlp_workspace_size())

    @staticmethod
    def loss_grad(theta, norm, I, psi, dpsi, beta, loss, grad, workspace, stream=None):
        _check(lib().adm_mlp_loss_grad(_ptr(theta), _ptr(norm), I.shape[0], _ptr(I), _ptr(psi), _ptr(dpsi),
                                       float(beta), _ptr(loss), _ptr(grad), _ptr(workspace),
                                       workspace.numel() * workspace.element_size(), _stream(stream)),
               "adm_mlp_loss_grad")

    @staticmethod
    def adam(theta, m, v, grad, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        _check(lib().adm_mlp_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), int(step), float(lr), float(beta1),
                                  float(beta2), float(eps), _stream(stream)), "adm_mlp_adam")

    @staticmethod
    def train(theta, norm, I, psi, dpsi, steps=20000, batch=8192, beta=4.0, lr0=3e-3, lr_end=3e-5, seed=0,
              stream=None):
        """Adam on the Sobolev loss (energy + beta * gradient) over the
        samples (I, psi, dpsi), theta updated in place: `steps` batches of
        `batch` samples drawn without replacement, reshuffled every epoch
        (seeded), learning rate decaying geometrically from lr0 to lr_end.
        Every step runs the library's kernels (adm_mlp_loss_grad,
        adm_mlp_adam); returns the first and the last batch loss."""
        import torch
        n = I.shape[0]
        m, v, grad = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
        ws = torch.zeros(MLP.workspace_size() // 4 + 1, dtype=torch.float32, device=theta.device)
        loss = torch.zeros(1, dtype=torch.float64, device=theta.device)
        gen = torch.Generator(device=theta.device).manual_seed(seed)
        perm = torch.randperm(n, device=theta.device, generator=gen)
        first = None
        for step in range(1, steps + 1):
            o = (step - 1) * batch % n
            if o + batch > n:  # a new epoch
                perm = torch.randperm(n, device=theta.device, generator=gen)
                o = 0
            idx = perm[o:o + batch]
            MLP.loss_grad(theta, norm, I[idx].contiguous(), psi[idx].contiguous(), dpsi[idx].contiguous(), beta,
                          loss, grad, ws, stream)
            MLP.adam(theta, m, v, grad, step, lr0 * (lr_end / lr0) ** (step / steps), stream=stream)
            if step == 1:
                first = loss.item()
        return first, loss.item()

    @staticmethod
    def nh_targets(F, E, nu, I, psi, dpsi, stream=None):
        _check(lib().adm_mlp_nh_targets(F.shape[0], _ptr(F), float(E), float(nu), _ptr(I), _ptr(psi), _ptr(dpsi),
                                        _stream(stream)), "adm_mlp_nh_targets")


def strerror(status: int) -> str:
    return lib().adm_strerror(status).decode()
