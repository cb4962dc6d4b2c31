"""GPU parity of per-term Hessian filtering (Sec. 7.1: negative local
eigenvalues set to eps before assembly; adm_set_projection) against the
FP64 oracle's projected assembly (numpy eigh per element, the plain
definition).  The GPU filters each term in its edge-vector coordinates with
an in-register Jacobi eigensolve; the oracle works on the full vertex-DOF
local Hessian, so the two routes share nothing but the definition.

Bars as for the plain Hessian: FP64 1e-12, FP32 2e-5 relative Frobenius.
The deformations (sigma = 5e-2 of the radius) make many local Hessians
indefinite, so the filter changes the result by 6-38 %."""
import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

TOL = {adm.FP64: 1e-12, adm.FP32: 2e-5}
NP = {adm.FP64: np.float64, adm.FP32: np.float32}
TT = {adm.FP64: torch.float64, adm.FP32: torch.float32}
ORC = {adm.SYMDIR2D: oracle.SYMDIR, adm.STVK_MEMBRANE: oracle.STVK, adm.HINGE_BENDING: oracle.HINGE,
       adm.SHELL: oracle.SHELL, adm.NH_MEMBRANE: oracle.NH}
SHELL_P = [1.0e5, 0.3, 1.0e-3]
PARAMS = {adm.HINGE_BENDING: [0.5, 1.0], adm.SYMDIR2D: None}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def gpu_hess(m, energy, prec, x):
    vd = m.var_dim
    _, nV, nnzb, _, _ = m.pattern(energy)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=NP[prec]).reshape(-1)).cuda()
    H = torch.full((nnzb * vd * vd,), float("nan"), dtype=TT[prec], device="cuda")
    g = torch.zeros(nV * vd, dtype=TT[prec], device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.eval(energy, prec, xd, e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    return H.cpu().numpy().reshape(nnzb, vd, vd), g.cpu().numpy().reshape(nV, vd), e.item()


def sphere(level=2, seed=31):
    V, F = synth.icosphere(level)
    return V, F, synth.perturb(V, sigma=5e-2, seed=seed)


def run(energy, prec, rest, faces, x, vd, eps=0.0, tile_tris=None, assembler=0):
    params = PARAMS.get(energy, SHELL_P)
    m = adm.Mesh(rest, faces, vd)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    if tile_tris is not None:
        m.set_option(adm.OPT_TILE_TRIS, tile_tris)
    if params is not None:
        m.set_params(energy, params)
    m.set_projection(True, eps)
    xr = np.asarray(x, dtype=NP[prec]).astype(np.float64)
    H, g, e = gpu_hess(m, energy, prec, xr)
    P = oracle.Problem(rest, faces, ORC[energy], vd, params=params)
    ref = P.assemble_projected(xr, eps)
    m.close()
    return H, g, e, ref, P


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
@pytest.mark.parametrize("energy", [adm.STVK_MEMBRANE, adm.NH_MEMBRANE, adm.HINGE_BENDING, adm.SHELL])
def test_projected_hessian_matches_oracle(energy, prec):
    V, F, x = sphere()
    H, g, e, ref, _ = run(energy, prec, V, F, x, 3)
    tol = TOL[prec]
    assert rel(H, ref["vals"]) <= tol, rel(H, ref["vals"])
    assert rel(g, ref["grad"]) <= tol
    assert abs(e - ref["energy"]) <= tol * abs(ref["energy"])


def test_projected_symdir_fp64():
    gr = synth.grid_uv(n=17, sigma=0.2, seed=32)
    H, _, _, ref, _ = run(adm.SYMDIR2D, adm.FP64, gr.rest, gr.faces, gr.x, 2)
    assert rel(H, ref["vals"]) <= 1e-12


def test_projected_eps_positive_fp64():
    V, F, x = sphere(seed=33)
    H, _, _, ref, P = run(adm.SHELL, adm.FP64, V, F, x, 3, eps=1.0)
    assert rel(H, ref["vals"]) <= 1e-12


def test_projected_batch_ragged_fp32_is_psd():
    b = synth.shell_batch([1, 2, 1], sigma=5e-2, seed=34)
    H, _, _, ref, P = run(adm.SHELL, adm.FP32, b.rest, b.faces, b.x, 3, tile_tris=50)
    assert rel(H, ref["vals"]) <= 2e-5
    D = oracle.bsr_to_dense(P.nV, 3, P.row_ptr, P.col, H.astype(np.float64))
    lam = np.linalg.eigvalsh(0.5 * (D + D.T))
    assert lam.min() >= -1e-5 * np.abs(lam).max()


def test_projection_under_atomic_option_and_with_hvp():
    V, F, x = sphere(level=2, seed=35)
    H, _, _, ref, P = run(adm.SHELL, adm.FP64, V, F, x, 3, assembler=1)
    assert rel(H, ref["vals"]) <= 1e-12
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_projection(True, 0.0)
    v = np.random.default_rng(9).normal(size=x.shape)
    xd = torch.from_numpy(x.reshape(-1).astype(np.float64)).cuda()
    vd = torch.from_numpy(v.reshape(-1)).cuda()
    hv = torch.zeros_like(xd)
    m.eval_hvp(adm.SHELL, adm.FP64, xd, vd, hv)
    torch.cuda.synchronize()
    rows = np.repeat(np.arange(P.nV), np.diff(P.row_ptr))
    want = np.zeros((P.nV, 3))
    np.add.at(want, rows, np.einsum("bij,bj->bi", ref["vals"], v[P.col]))
    assert rel(hv.cpu().numpy().reshape(-1, 3), want) <= 1e-12
    m.close()


def test_projection_off_restores_plain_hessian():
    V, F, x = sphere(level=1, seed=36)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_projection(True, 0.0)
    Hp, _, _ = gpu_hess(m, adm.SHELL, adm.FP64, x)
    m.set_projection(False, 0.0)
    H0, _, _ = gpu_hess(m, adm.SHELL, adm.FP64, x)
    P = oracle.Problem(V, F, oracle.SHELL, 3, params=SHELL_P)
    assert rel(H0, P.assemble(x)["vals"]) <= 1e-12
    assert rel(Hp, H0) > 1e-3
    with pytest.raises(adm.AdmError):
        m.set_projection(True, -1.0)
    m.close()
