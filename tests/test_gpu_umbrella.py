"""GPU parity of the per-vertex one-ring term (ADM_UMBRELLA: w/2 |x_v -
mean of its neighbours|^2) and its two-ring block pattern, through the C
ABI, against the FP64 oracle: pattern bit-exact, FP64 1e-12 and FP32 2e-5
on energy, gradient, Hessian and H v; 3D and 2D coordinates; a batch."""
import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

W = 1.7
NP = {adm.FP64: np.float64, adm.FP32: np.float32}
TT = {adm.FP64: torch.float64, adm.FP32: torch.float32}
TOL = {adm.FP64: 1e-12, adm.FP32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def run(m, F, x, prec, batch=False):
    vd = x.shape[1]
    _, nV, nnzb, rp, col = m.pattern(adm.UMBRELLA)
    rp, col = rp.cpu().numpy(), col.cpu().numpy()
    orp, ocol = oracle.ring_pattern(nV, F)
    assert np.array_equal(rp, orp) and np.array_equal(col, ocol)
    xr = x.astype(NP[prec]).astype(np.float64)
    xd = torch.from_numpy(np.ascontiguousarray(xr, dtype=NP[prec]).reshape(-1)).cuda()
    g = torch.full((nV * vd,), float("nan"), dtype=TT[prec], device="cuda")
    H = torch.full((nnzb * vd * vd,), float("nan"), dtype=TT[prec], device="cuda")
    v = np.random.default_rng(3).normal(size=xr.shape)
    vv = torch.from_numpy(np.ascontiguousarray(v, dtype=NP[prec]).reshape(-1)).cuda()
    hv = torch.full_like(g, float("nan"))
    if batch:
        e = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda")
        m.eval_batch(adm.UMBRELLA, prec, xd, e, None, g, H)
    else:
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        m.eval(adm.UMBRELLA, prec, xd, e, g, H)
    m.eval_hvp(adm.UMBRELLA, prec, xd, vv, hv)
    torch.cuda.synchronize()
    assert m.status() == 0
    ref = oracle.umbrella_assemble(F, xr, W, orp, ocol)
    tol = TOL[prec]
    assert rel(g.cpu().numpy().reshape(-1, vd), ref["grad"]) <= tol
    assert rel(H.cpu().numpy().reshape(-1, vd, vd), ref["vals"]) <= tol
    vr = v.astype(NP[prec]).astype(np.float64)
    Hd = oracle.bsr_to_dense(nV, vd, orp, ocol, ref["vals"])
    assert rel(hv.cpu().numpy(), Hd @ vr.reshape(-1)) <= tol
    return e.cpu().numpy(), ref


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_umbrella_sphere(prec):
    V, F = synth.icosphere(3)
    x = synth.perturb(V, 2e-2, 61)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.UMBRELLA, [W])
    e, ref = run(m, F, x, prec)
    assert abs(e[0] - ref["energy"]) <= TOL[prec] * ref["energy"]
    m.close()


def test_umbrella_grid_2d_fp64():
    g = synth.grid_uv(n=17, sigma=0.3, seed=62)
    m = adm.Mesh(g.rest, g.faces, 2)
    m.set_params(adm.UMBRELLA, [W])
    e, ref = run(m, g.faces, g.x, adm.FP64)
    assert abs(e[0] - ref["energy"]) <= 1e-12 * ref["energy"]
    m.close()


def test_umbrella_batch_per_mesh():
    b = synth.shell_batch([1, 3, 2], sigma=2e-2, seed=63)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.UMBRELLA, [W])
    e, _ = run(m, b.faces, b.x, adm.FP64, batch=True)
    for k in range(3):
        f = b.faces[b.f_off[k]:b.f_off[k + 1]] - b.v_off[k]
        want = oracle.umbrella_assemble(f, b.x[b.v_off[k]:b.v_off[k + 1]], W)["energy"]
        assert abs(e[k] - want) <= 1e-12 * want
    m.close()
