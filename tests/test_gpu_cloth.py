"""GPU parity of the mass-spring cloth energy (Sec. 7.1; ADM_MASS_SPRING:
per-edge springs, per-vertex lumped-mass inertia and gravity) against the
FP64 oracle's closed forms, through the C ABI: energy, gradient and 3x3 BSR
Hessian, the matrix-free product, per-term filtering, ragged tiles and a
batch of two cloths.  Bars: FP64 1e-12, FP32 2e-5 relative."""
import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

NP = {adm.FP64: np.float64, adm.FP32: np.float32}
TT = {adm.FP64: torch.float64, adm.FP32: torch.float32}
TOL = {adm.FP64: 1e-12, adm.FP32: 2e-5}
PARAMS = [2.0e3, 0.02, 1.5, 0.1, -0.2, -9.81]


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def evaluate(m, prec, x, batch=False):
    _, nV, nnzb, rp, col = m.pattern(adm.MASS_SPRING)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=NP[prec]).reshape(-1)).cuda()
    g = torch.full((nV * 3,), float("nan"), dtype=TT[prec], device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), dtype=TT[prec], device="cuda")
    if batch:
        e = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda")
        m.eval_batch(adm.MASS_SPRING, prec, xd, e, None, g, H)
    else:
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        m.eval(adm.MASS_SPRING, prec, xd, e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    return (e.cpu().numpy(), g.cpu().numpy().reshape(nV, 3), H.cpu().numpy().reshape(nnzb, 3, 3),
            rp.cpu().numpy(), col.cpu().numpy())


def make(c, tile=None, target=True):
    m = adm.Mesh(c.rest, c.faces, 3)
    m.set_params(adm.MASS_SPRING, PARAMS)
    if tile is not None:
        m.set_option(adm.OPT_TILE_TRIS, tile)
    if target:
        m.set_inertia_target(c.xhat)
    return m


@pytest.mark.parametrize("prec,n", [(adm.FP64, 12), (adm.FP32, 40)])
def test_cloth_matches_oracle(prec, n):
    c = synth.cloth_grid(n, sigma=0.3, seed=41)
    m = make(c)
    x = c.x.astype(NP[prec]).astype(np.float64)
    e, g, H, rp, col = evaluate(m, prec, x)
    P = oracle.pattern(c.nV, c.faces)
    assert np.array_equal(rp, P[0]) and np.array_equal(col, P[1])
    ref = oracle.cloth_assemble(c.rest, c.faces, x, c.xhat, PARAMS, rp, col)
    tol = TOL[prec]
    assert abs(e[0] - ref["energy"]) <= tol * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= tol
    assert rel(H, ref["vals"]) <= tol, rel(H, ref["vals"])
    m.close()


@pytest.mark.parametrize("tile", [32, 100])
def test_cloth_ragged_tiles_fp32(tile):
    c = synth.cloth_grid(30, sigma=0.3, seed=42)
    m = make(c, tile=tile)
    x = c.x.astype(np.float32).astype(np.float64)
    e, g, H, rp, col = evaluate(m, adm.FP32, x)
    ref = oracle.cloth_assemble(c.rest, c.faces, x, c.xhat, PARAMS, rp, col)
    assert rel(H, ref["vals"]) <= 2e-5 and rel(g, ref["grad"]) <= 2e-5
    m.close()


def test_cloth_default_target_is_rest():
    c = synth.cloth_grid(10, sigma=0.3, seed=43)
    m = make(c, target=False)
    e, g, H, rp, col = evaluate(m, adm.FP64, c.x)
    ref = oracle.cloth_assemble(c.rest, c.faces, c.x, c.rest, PARAMS, rp, col)
    assert rel(g, ref["grad"]) <= 1e-12 and abs(e[0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    m.close()


def test_cloth_hvp_and_projection_fp64():
    c = synth.cloth_grid(12, sigma=0.3, seed=44)
    c.x = 0.8 * c.rest + (c.x - c.rest)   # compressed springs: indefinite spring terms
    m = make(c)
    P = oracle.pattern(c.nV, c.faces)
    v = np.random.default_rng(4).normal(size=c.x.shape)
    xd = torch.from_numpy(c.x.reshape(-1)).cuda()
    vd = torch.from_numpy(v.reshape(-1)).cuda()
    hv = torch.zeros_like(xd)
    m.eval_hvp(adm.MASS_SPRING, adm.FP64, xd, vd, hv)
    torch.cuda.synchronize()
    ref = oracle.cloth_assemble(c.rest, c.faces, c.x, c.xhat, PARAMS, P[0], P[1])
    rows = np.repeat(np.arange(c.nV), np.diff(P[0]))
    want = np.zeros((c.nV, 3))
    np.add.at(want, rows, np.einsum("bij,bj->bi", ref["vals"], v[P[1]]))
    assert rel(hv.cpu().numpy().reshape(-1, 3), want) <= 1e-12
    for eps in (0.0, 1e-3):
        m.set_projection(True, eps)
        _, _, H, rp, col = evaluate(m, adm.FP64, c.x)
        refp = oracle.cloth_assemble(c.rest, c.faces, c.x, c.xhat, PARAMS, rp, col, project=True, eps=eps)
        assert rel(refp["vals"], ref["vals"]) > 1e-4       # the filter did something
        assert rel(H, refp["vals"]) <= 1e-12, rel(H, refp["vals"])
    m.close()


def test_cloth_batch_per_mesh_energy():
    a = synth.cloth_grid(8, sigma=0.3, seed=45)
    b = synth.cloth_grid(11, sigma=0.3, seed=46)
    rest = np.concatenate([a.rest, b.rest + [2.0, 0.0, 0.0]])
    faces = np.concatenate([a.faces, b.faces + a.nV]).astype(np.int32)
    x = np.concatenate([a.x, b.x + [2.0, 0.0, 0.0]])
    xhat = np.concatenate([a.xhat, b.xhat + [2.0, 0.0, 0.0]])
    m = adm.Mesh(rest, faces, 3, v_off=np.array([0, a.nV, a.nV + b.nV]), f_off=np.array([0, a.nT, a.nT + b.nT]))
    m.set_params(adm.MASS_SPRING, PARAMS)
    m.set_inertia_target(xhat)
    e, g, H, rp, col = evaluate(m, adm.FP64, x, batch=True)
    ea = oracle.cloth_assemble(a.rest, a.faces, a.x, a.xhat, PARAMS)["energy"]
    eb = oracle.cloth_assemble(b.rest + [2.0, 0.0, 0.0], b.faces, x[a.nV:], xhat[a.nV:], PARAMS)["energy"]
    assert abs(e[0] - ea) <= 1e-12 * abs(ea) and abs(e[1] - eb) <= 1e-12 * abs(eb)
    ref = oracle.cloth_assemble(rest, faces, x, xhat, PARAMS, rp, col)
    assert rel(H, ref["vals"]) <= 1e-12
    m.close()


def test_cloth_argument_errors():
    g = synth.grid_uv(5)
    m2 = adm.Mesh(g.rest, g.faces, 2)
    with pytest.raises(adm.AdmError):
        m2.set_inertia_target(g.rest)
    m2.close()
    c = synth.cloth_grid(5)
    m = adm.Mesh(c.rest, c.faces, 3)
    with pytest.raises(adm.AdmError):
        m.set_params(adm.MASS_SPRING, [1.0] * 7)
    m.close()
