"""GPU parity of the matrix-free Hessian-vector product (Sec. 5.5,
Sec. 6.2; the CG solver of Sec. 7.2) through the C ABI: hv = H(x) v from
the tiled kernel's per-element local Hessians, against the FP64 oracle's
assembled Hessian applied to v, with the energy and gradient of the same
pass.

Bars: FP64 relative 1e-12 (energy, gradient, hv); FP32 relative 2e-5 on
hv, the Hessian bar: each hv entry is a dot product of one Hessian row with
v, so its FP32 error is the Hessian's rounding weighted by |v|, and v is
drawn O(1) with no cancellation built in."""
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


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def gpu_hvp(m, energy, prec, x, v, grad=True):
    vd = m.var_dim
    n = x.size
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=NP[prec]).reshape(-1)).cuda()
    vv = torch.from_numpy(np.ascontiguousarray(v, dtype=NP[prec]).reshape(-1)).cuda()
    hv = torch.full((n,), float("nan"), dtype=TT[prec], device="cuda")
    g = torch.full((n,), float("nan"), dtype=TT[prec], device="cuda") if grad else None
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.eval_hvp(energy, prec, xd, vv, hv, e, g)
    torch.cuda.synchronize()
    assert m.status() == 0
    out = {"hv": hv.cpu().numpy().reshape(-1, vd), "energy": e.item()}
    if grad:
        out["grad"] = g.cpu().numpy().reshape(-1, vd)
    return out


def check(energy, prec, rest, faces, x, vd, params=None, tile_tris=None, assembler=0, seed=0):
    m = adm.Mesh(rest, faces, vd)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    if tile_tris is not None:
        m.set_option(adm.OPT_TILE_TRIS, tile_tris)
    if params is not None:
        m.set_params(energy, params)
    xr = np.asarray(x, dtype=NP[prec]).astype(np.float64)
    v = np.random.default_rng(seed).normal(size=xr.shape).astype(NP[prec]).astype(np.float64)
    out = gpu_hvp(m, energy, prec, xr, v)
    P = oracle.Problem(rest, faces, ORC[energy], vd, params=params)
    ref = P.hvp(xr, v)
    assert ref["n_domain_err"] == 0
    tol = TOL[prec]
    assert abs(out["energy"] - ref["energy"]) <= tol * abs(ref["energy"])
    assert rel(out["grad"], ref["grad"]) <= tol
    assert rel(out["hv"], ref["hv"]) <= tol, rel(out["hv"], ref["hv"])
    m.close()


def test_hvp_symdir_grid_fp64():
    g = synth.grid_uv()
    check(adm.SYMDIR2D, adm.FP64, g.rest, g.faces, g.x, 2)


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
@pytest.mark.parametrize("energy", [adm.STVK_MEMBRANE, adm.HINGE_BENDING, adm.NH_MEMBRANE, adm.SHELL])
def test_hvp_shell_terms(energy, prec):
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=21)
    check(energy, prec, V, F, x, 3, params=[0.5, 1.0] if energy == adm.HINGE_BENDING else SHELL_P)


@pytest.mark.parametrize("tile", [32, 100, 777])
def test_hvp_ragged_tiles_and_batch(tile):
    b = synth.shell_batch([2, 3, 1, 2], sigma=1e-2, seed=22)
    check(adm.SHELL, adm.FP32, b.rest, b.faces, b.x, 3, params=SHELL_P, tile_tris=tile)


def test_hvp_under_atomic_assembler_option():
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=1e-2, seed=23)
    check(adm.SHELL, adm.FP64, V, F, x, 3, params=SHELL_P, assembler=1)


def test_hvp_matches_own_bsr_times_v():
    """Same precision, same x: the matrix-free product equals the library's
    own assembled Hessian applied to v (both FP64)."""
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=24)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, SHELL_P)
    _, nV, nnzb, rp, col = m.pattern(adm.SHELL)
    xd = torch.from_numpy(x.reshape(-1).astype(np.float64)).cuda()
    H = torch.zeros(nnzb * 9, dtype=torch.float64, device="cuda")
    m.eval(adm.SHELL, adm.FP64, xd, None, None, H)
    v = np.random.default_rng(5).normal(size=(nV, 3))
    out = gpu_hvp(m, adm.SHELL, adm.FP64, x, v, grad=False)
    vals = H.cpu().numpy().reshape(nnzb, 3, 3)
    rows = np.repeat(np.arange(nV), np.diff(rp.cpu().numpy()))
    ref = np.zeros((nV, 3))
    np.add.at(ref, rows, np.einsum("bij,bj->bi", vals, v[col.cpu().numpy()]))
    assert rel(out["hv"], ref) <= 1e-12
    m.close()


def test_hvp_graph_replay_follows_buffer_contents():
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=25)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_option(adm.OPT_GRAPH, 1)
    P = oracle.Problem(V, F, oracle.SHELL, 3, params=SHELL_P)
    xd = torch.from_numpy(x.reshape(-1).astype(np.float64)).cuda()
    vd = torch.zeros_like(xd)
    hv = torch.zeros_like(xd)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(3):  # capture on the first call, replay on the others with new v
        v = np.random.default_rng(30 + k).normal(size=x.shape)
        vd.copy_(torch.from_numpy(v.reshape(-1)))
        m.eval_hvp(adm.SHELL, adm.FP64, xd, vd, hv, e)
        torch.cuda.synchronize()
        assert rel(hv.cpu().numpy().reshape(-1, 3), P.hvp(x, v)["hv"]) <= 1e-12
    m.close()


def test_hvp_argument_errors():
    V, F = synth.icosphere(1)
    m = adm.Mesh(V, F, 3)
    xd = torch.from_numpy(V.reshape(-1).astype(np.float64)).cuda()
    with pytest.raises(adm.AdmError):
        m.eval_hvp(adm.SHELL, adm.FP64, xd, None, torch.zeros_like(xd))
    with pytest.raises(adm.AdmError):
        m.eval_hvp(adm.ARAP2D_RESIDUAL, adm.FP64, xd, xd, torch.zeros_like(xd))
    m.close()
