"""GPU parity of interaction terms over vertex pairs (Sec. 4.3) with the
dynamic block pattern (Sec. 6.3, Alg. 1) and the contact barrier of
Sec. 7.7, through the C ABI, against the oracle: the extended pattern is
compared bit-exactly (mesh columns first, new columns ascending), values
block by block at FP64 1e-12 and FP32 2e-5."""
import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

SHELL_P = [1.0e5, 0.3, 1.0e-3]
KAPPA, DHAT, AREA, HSTEP = 1.0e3, 0.35, 0.05, 0.1
NP = {adm.FP64: np.float64, adm.FP32: np.float32}
TT = {adm.FP64: torch.float64, adm.FP32: torch.float32}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def pick_pairs(V, F, x, n, seed, adjacent=3, far=3):
    """n unique non-adjacent vertex pairs within DHAT of each other, plus a
    few mesh-adjacent pairs and a few beyond DHAT."""
    rng = np.random.default_rng(seed)
    rp, col = oracle.pattern(len(V), F)
    adj = {(i, int(c)) for i in range(len(V)) for c in col[rp[i]:rp[i + 1]]}
    out, seen = [], set()
    for _ in range(200 * n):
        if len(out) == n:
            break
        i = int(rng.integers(len(V)))
        d = np.linalg.norm(x - x[i], axis=1)
        cand = [j for j in np.argsort(d)[1:40] if d[j] < 0.9 * DHAT and (i, int(j)) not in adj]
        if not cand:
            continue
        j = int(rng.choice(cand))
        key = (min(i, j), max(i, j))
        if key not in seen:
            seen.add(key)
            out.append((i, j))
    for i in rng.integers(len(V), size=adjacent):  # already in the mesh pattern
        j = int(col[rp[i] + 1] if col[rp[i]] == i else col[rp[i]])
        key = (min(int(i), j), max(int(i), j))
        if key not in seen:
            seen.add(key)
            out.append((int(i), j))
    assert len(out) >= n // 2, "too few vertex pairs within the activation distance"
    k = 0
    for _ in range(1000):  # beyond the activation distance
        if k == far:
            break
        i, j = (int(v) for v in rng.integers(len(V), size=2))
        key = (min(i, j), max(i, j))
        if i != j and np.linalg.norm(x[i] - x[j]) > DHAT and key not in seen:
            seen.add(key)
            out.append((i, j))
            k += 1
    return np.asarray(out, dtype=np.int32)


def gpu_eval(m, energy, prec, x):
    _, nV, nnzb, rp, col = m.pattern(energy)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=NP[prec]).reshape(-1)).cuda()
    g = torch.full((nV * 3,), float("nan"), dtype=TT[prec], device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), dtype=TT[prec], device="cuda")
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    m.eval(energy, prec, xd, e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    return e.item(), g.cpu().numpy().reshape(-1, 3), H.cpu().numpy().reshape(-1, 3, 3), rp.cpu().numpy(), \
        col.cpu().numpy()


def compare(V, F, x, pairs, base, e, g, H, rp, col, tol):
    brp, bcol = oracle.pattern(len(V), F, oracle.hinges(len(V), F)) if base["shell"] else oracle.pattern(len(V), F)
    erp, ecol = oracle.extended_pattern(brp, bcol, pairs)
    assert np.array_equal(rp, erp) and np.array_equal(col, ecol)       # bit-exact pattern and layout
    ref = oracle.add_interactions(base, x, pairs, KAPPA, DHAT, AREA, HSTEP, brp, bcol)
    assert abs(e - ref["energy"]) <= tol * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= tol
    want = np.stack([ref["blocks"].get((r, int(c)), np.zeros((3, 3))) for r in range(len(V))
                     for c in col[rp[r]:rp[r + 1]]])
    assert len(ref["blocks"]) == len(col)
    assert rel(H, want) <= tol, rel(H, want)


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_shell_with_contacts(prec):
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=51).astype(NP[prec]).astype(np.float64)
    pairs = pick_pairs(V, F, x, 60, seed=52)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_interactions(adm.SHELL, torch.from_numpy(pairs).cuda(), KAPPA, DHAT, AREA, HSTEP)
    e, g, H, rp, col = gpu_eval(m, adm.SHELL, prec, x)
    P = oracle.Problem(V, F, oracle.SHELL, 3, params=SHELL_P)
    base = dict(P.assemble(x), shell=True)
    compare(V, F, x, pairs, base, e, g, H, rp, col, 1e-12 if prec == adm.FP64 else 2e-5)
    m.close()


def test_cloth_contacts_reset_retile_and_graph():
    c = synth.cloth_grid(14, sigma=0.3, seed=53)
    c.x[:, 2] += 0.3 * np.sin(6 * c.rest[:, 0])  # folds bring distant vertices near each other
    m = adm.Mesh(c.rest, c.faces, 3)
    m.set_inertia_target(c.xhat)
    cp = [2.0e3, 0.02, 1.5, 0.0, 0.0, -9.81]
    m.set_params(adm.MASS_SPRING, cp)
    rp0, col0 = oracle.pattern(c.nV, c.faces)
    base = dict(oracle.cloth_assemble(c.rest, c.faces, c.x, c.xhat, cp, rp0, col0), shell=False)
    for k, seed in enumerate((54, 55)):  # two sets in a row (the pattern buffers alternate)
        pairs = pick_pairs(c.rest, c.faces, c.x, 40, seed=seed)
        m.set_interactions(adm.MASS_SPRING, pairs, KAPPA, DHAT, AREA, HSTEP)   # host pairs
        if k == 1:
            m.set_option(adm.OPT_TILE_TRIS, 64)   # tiles rebuilt while pairs are set
            m.set_option(adm.OPT_GRAPH, 1)
        for _ in range(2):
            e, g, H, rp, col = gpu_eval(m, adm.MASS_SPRING, adm.FP64, c.x)
            compare(c.rest, c.faces, c.x, pairs, base, e, g, H, rp, col, 1e-12)
    m.set_interactions(adm.MASS_SPRING, None, KAPPA, DHAT, AREA, HSTEP)      # cleared: the mesh pattern again
    e, g, H, rp, col = gpu_eval(m, adm.MASS_SPRING, adm.FP64, c.x)
    assert np.array_equal(rp, rp0) and np.array_equal(col, col0)
    assert rel(H, base["vals"]) <= 1e-12
    m.close()


def test_hvp_and_batch_energy_with_contacts():
    b = synth.shell_batch([3, 3], sigma=1e-2, seed=56, spacing=2.3)   # two spheres close to each other
    x = b.x
    pairs = pick_pairs(b.rest, b.faces, x, 50, seed=57)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_interactions(adm.SHELL, pairs, KAPPA, DHAT, AREA, HSTEP)
    P = oracle.Problem(b.rest, b.faces, oracle.SHELL, 3, params=SHELL_P)
    base = P.assemble(x, per_element=True)
    ref = oracle.add_interactions(base, x, pairs, KAPPA, DHAT, AREA, HSTEP, P.row_ptr, P.col)
    v = np.random.default_rng(5).normal(size=x.shape)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    vd = torch.from_numpy(v.reshape(-1)).cuda()
    hv = torch.zeros_like(xd)
    m.eval_hvp(adm.SHELL, adm.FP64, xd, vd, hv)
    torch.cuda.synchronize()
    want = np.zeros_like(x)
    for (r, cc), blk in ref["blocks"].items():
        want[r] += blk @ v[cc]
    assert rel(hv.cpu().numpy().reshape(-1, 3), want) <= 1e-12
    em = torch.zeros(2, dtype=torch.float64, device="cuda")
    m.eval_batch(adm.SHELL, adm.FP64, xd, em, None, None, None)
    torch.cuda.synchronize()
    per_mesh = np.zeros(2)
    nT, nH = P.nT, P.nH
    ee = base["elem_energy"]
    for k in range(2):  # mesh energies: triangles, hinges of the mesh, and pairs whose first vertex is in it
        f0, f1 = b.f_off[k], b.f_off[k + 1]
        per_mesh[k] = ee[f0:f1].sum()
    hv_mesh = np.searchsorted(b.v_off, P.H[:, 0], side="right") - 1
    for k in range(2):
        per_mesh[k] += ee[nT:][hv_mesh == k].sum()
    for i, j in pairs:
        f, _, _ = oracle.contact_vv(x[i], x[j], KAPPA, DHAT, AREA, HSTEP)
        per_mesh[np.searchsorted(b.v_off, i, side="right") - 1] += f
    assert rel(em.cpu().numpy(), per_mesh) <= 1e-12
    m.close()


def test_contact_argument_errors():
    V, F = synth.icosphere(1)
    m = adm.Mesh(V, F, 3)
    rp0 = m.pattern(adm.STVK_MEMBRANE)[2]
    brp, bcol = oracle.pattern(len(V), F)
    far = next(j for j in range(len(V)) if j not in bcol[brp[0]:brp[1]])   # not adjacent to vertex 0
    for bad in (np.array([[0, 0]]), np.array([[0, 99999]]), np.array([[far, -1]])):
        with pytest.raises(adm.AdmError):
            m.set_interactions(adm.STVK_MEMBRANE, bad.astype(np.int32), KAPPA, DHAT, AREA, HSTEP)
        assert m.pattern(adm.STVK_MEMBRANE)[2] == rp0            # cleared back to the mesh pattern
    with pytest.raises(adm.AdmError):
        m.set_interactions(adm.STVK_MEMBRANE, np.array([[0, far]], dtype=np.int32), KAPPA, 0.0, AREA, HSTEP)
    m.close()
