"""GPU parity of vertex-face contact terms (Sec. 7.7) together with
vertex-vertex pairs, and the block pattern they induce (Alg. 1 with the
repeated blocks of several terms merged), through the C ABI, against the
oracle: the extended pattern bit-exactly, values at FP64 1e-12 and FP32
2e-5; the matrix-free product, per-mesh energies and per-term filtering.

Points are kept where the nearest part of the triangle (corner, edge,
interior) is the same for small moves of p, so that both sides pick the same
formula for the squared distance."""
import numpy as np
import pytest

import oracle
import synth
from util import rel
from test_gpu_contact import pick_pairs, gpu_eval

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

SHELL_P = [1.0e5, 0.3, 1.0e-3]
KAPPA, DHAT, AREA, HSTEP = 1.0e3, 0.35, 0.05, 0.1
NP = {adm.FP64: np.float64, adm.FP32: np.float32}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def stable_region(p, a, b, c, delta=1e-3):
    reg = oracle.closest_region(p, a, b, c)
    for d in np.vstack([np.eye(3), -np.eye(3)]) * delta:
        if oracle.closest_region(p + d, a, b, c) != reg:
            return None
    return reg


def pick_vf(F, x, n, seed, owner=None, far=3):
    """n vertex-face terms (p, a, b, c), p not a corner of the face, within
    DHAT and with a stable nearest region; plus a few beyond DHAT.  With
    owner (mesh of every vertex), p is mostly drawn from the vertices near
    another mesh, whose nearest parts there are often face interiors."""
    rng = np.random.default_rng(seed)
    cen = x[F].mean(axis=1)
    hot = np.arange(len(x))
    if owner is not None:
        d = np.array([np.linalg.norm(x[owner != owner[i]] - x[i], axis=1).min() for i in range(len(x))])
        hot = np.flatnonzero(d < 0.9 * DHAT)
    out, seen, kinds = [], set(), set()
    for _ in range(100 * n):
        if len(out) == n:
            break
        across = rng.random() < 0.7
        p = int(rng.choice(hot) if across else rng.integers(len(x)))
        dist = np.linalg.norm(cen - x[p], axis=1)
        if owner is not None and across:
            dist[owner[F[:, 0]] == owner[p]] = np.inf                  # faces of the other meshes
        near = np.argsort(dist)[:12]
        f = int(rng.choice(near))
        if p in F[f] or (p, f) in seen:
            continue
        a, b, c = (x[v] for v in F[f])
        if oracle.vf_distance(x[p], a, b, c) >= 0.9 * DHAT:
            continue
        reg = stable_region(x[p], a, b, c)
        if reg is None:
            continue
        seen.add((p, f))
        kinds.add(reg[0])
        out.append((p, *F[f]))
    k = 0
    for _ in range(1000):
        if k == far:
            break
        p, f = int(rng.integers(len(x))), int(rng.integers(len(F)))
        if p not in F[f] and oracle.vf_distance(x[p], *(x[v] for v in F[f])) > DHAT:
            out.append((p, *F[f]))
            k += 1
    assert len(out) >= n // 2, "too few vertex-face terms within the activation distance"
    return np.asarray(out, dtype=np.int32), kinds


def owner(b):
    return np.searchsorted(b.v_off, np.arange(b.v_off[-1]), side="right") - 1


def reference(V, F, x, pairs, vf, shell, project=False, eps=0.0):
    if shell:
        P = oracle.Problem(V, F, oracle.SHELL, 3, params=SHELL_P)
        base = P.assemble_projected(x, eps) if project else P.assemble(x)
        brp, bcol = P.row_ptr, P.col
    else:
        brp, bcol = oracle.pattern(len(V), F)
        P = oracle.Problem(V, F, oracle.STVK, 3, params=SHELL_P)
        base = P.assemble_projected(x, eps) if project else P.assemble(x)
    erp, ecol = oracle.extended_pattern(brp, bcol, pairs, vf)
    ref = oracle.add_interactions(base, x, pairs, KAPPA, DHAT, AREA, HSTEP, brp, bcol, vf, project, eps)
    return erp, ecol, ref


def check(V, F, x, pairs, vf, got, shell, tol, project=False, eps=0.0):
    e, g, H, rp, col = got
    erp, ecol, ref = reference(V, F, x, pairs, vf, shell, project, eps)
    assert np.array_equal(rp, erp) and np.array_equal(col, ecol)       # bit-exact pattern and layout
    assert abs(e - ref["energy"]) <= tol * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= tol
    want = np.stack([ref["blocks"].get((r, int(c)), np.zeros((3, 3))) for r in range(len(V))
                     for c in col[rp[r]:rp[r + 1]]])
    assert rel(H, want) <= tol, rel(H, want)
    return ref


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_two_spheres_vertex_face(prec):
    b = synth.shell_batch([3, 3], sigma=1e-2, seed=61, spacing=2.2)
    x = b.x.astype(NP[prec]).astype(np.float64)
    vf, kinds = pick_vf(b.faces, x, 80, seed=62, owner=owner(b))
    assert kinds == {"v", "e", "f"}                                     # every formula of the distance
    pairs = pick_pairs(b.rest, b.faces, x, 20, seed=63)
    m = adm.Mesh(b.rest, b.faces, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_contacts(adm.SHELL, torch.from_numpy(pairs).cuda(), torch.from_numpy(vf).cuda(), KAPPA, DHAT, AREA, HSTEP)
    got = gpu_eval(m, adm.SHELL, prec, x)
    check(b.rest, b.faces, x, pairs, vf, got, True, 1e-12 if prec == adm.FP64 else 2e-5)
    m.close()


def test_membrane_vertex_face_only_repeated_and_cleared():
    """Vertex-face terms alone, one of them listed twice (it counts twice),
    then a second set (the pattern buffers alternate), then none."""
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=64)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.STVK_MEMBRANE, SHELL_P)
    rp0 = m.pattern(adm.STVK_MEMBRANE)[3].cpu().numpy()
    for seed in (65, 66):
        vf, _ = pick_vf(F, x, 50, seed=seed)
        vf = np.concatenate([vf, vf[:1]])
        m.set_contacts(adm.STVK_MEMBRANE, None, vf, KAPPA, DHAT, AREA, HSTEP)
        for _ in range(2):                                                 # new blocks re-zeroed every pass
            got = gpu_eval(m, adm.STVK_MEMBRANE, adm.FP64, x)
            check(V, F, x, np.zeros((0, 2), np.int32), vf, got, False, 1e-12)
    m.set_contacts(adm.STVK_MEMBRANE, None, None, KAPPA, DHAT, AREA, HSTEP)
    assert np.array_equal(m.pattern(adm.STVK_MEMBRANE)[3].cpu().numpy(), rp0)
    m.close()


def test_vertex_face_hvp_and_mesh_energies():
    b = synth.shell_batch([3, 3], sigma=1e-2, seed=67, spacing=2.2)
    x = b.x
    vf, _ = pick_vf(b.faces, x, 60, seed=68, owner=owner(b))
    pairs = pick_pairs(b.rest, b.faces, x, 20, seed=69)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_contacts(adm.SHELL, pairs, vf, KAPPA, DHAT, AREA, HSTEP)
    P = oracle.Problem(b.rest, b.faces, oracle.SHELL, 3, params=SHELL_P)
    base = P.assemble(x, per_element=True)
    ref = oracle.add_interactions(base, x, pairs, KAPPA, DHAT, AREA, HSTEP, P.row_ptr, P.col, vf)
    v = np.random.default_rng(7).normal(size=x.shape)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    hv = torch.zeros_like(xd)
    m.eval_hvp(adm.SHELL, adm.FP64, xd, torch.from_numpy(v.reshape(-1)).cuda(), hv)
    torch.cuda.synchronize()
    want = np.zeros_like(x)
    for (r, cc), blk in ref["blocks"].items():
        want[r] += blk @ v[cc]
    assert rel(hv.cpu().numpy().reshape(-1, 3), want) <= 1e-12
    em = torch.zeros(2, dtype=torch.float64, device="cuda")
    m.eval_batch(adm.SHELL, adm.FP64, xd, em, None, None, None)
    torch.cuda.synchronize()
    ee = base["elem_energy"]
    per_mesh = np.array([ee[b.f_off[k]:b.f_off[k + 1]].sum() for k in range(2)])
    hv_mesh = np.searchsorted(b.v_off, P.H[:, 0], side="right") - 1
    for k in range(2):
        per_mesh[k] += ee[P.nT:][hv_mesh == k].sum()
    mesh_of = owner(b)
    for i, j in pairs:
        per_mesh[mesh_of[i]] += oracle.contact_vv(x[i], x[j], KAPPA, DHAT, AREA, HSTEP)[0]
    for p, a, bb, c in vf:
        per_mesh[mesh_of[p]] += oracle.contact_vf(x[p], x[a], x[bb], x[c], KAPPA, DHAT, AREA, HSTEP)[0]
    assert rel(em.cpu().numpy(), per_mesh) <= 1e-12
    m.close()


@pytest.mark.parametrize("eps", [0.0, 1e-3])
def test_vertex_face_filtered(eps):
    b = synth.shell_batch([3, 3], sigma=1e-2, seed=70, spacing=2.2)
    x = b.x
    vf, _ = pick_vf(b.faces, x, 60, seed=71, owner=owner(b))
    pairs = pick_pairs(b.rest, b.faces, x, 20, seed=72)
    m = adm.Mesh(b.rest, b.faces, 3)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_projection(True, eps)
    m.set_contacts(adm.SHELL, pairs, vf, KAPPA, DHAT, AREA, HSTEP)
    got = gpu_eval(m, adm.SHELL, adm.FP64, x)
    check(b.rest, b.faces, x, pairs, vf, got, True, 1e-12, project=True, eps=eps)
    m.close()


def test_vertex_face_argument_errors():
    V, F = synth.icosphere(1)
    m = adm.Mesh(V, F, 3)
    rp0 = m.pattern(adm.STVK_MEMBRANE)[2]
    f = F[5]
    for bad in ([f[0], *f], [0, 1, 1, 2], [99999, *f], [-1, *f]):
        with pytest.raises(adm.AdmError):
            m.set_contacts(adm.STVK_MEMBRANE, None, np.array([bad], dtype=np.int32), KAPPA, DHAT, AREA, HSTEP)
        assert m.pattern(adm.STVK_MEMBRANE)[2] == rp0                      # cleared back to the mesh pattern
    m.close()


def test_cloth_vertex_face_hvp_fp64():
    """Vertex-face terms on the mass-spring cloth (the triangle pattern) in a
    folded state, through the Hessian pass and the matrix-free product."""
    c = synth.cloth_grid(14, sigma=0.3, seed=73)
    c.x[:, 2] += 0.3 * np.sin(6 * c.rest[:, 0])  # folds bring distant parts near each other
    m = adm.Mesh(c.rest, c.faces, 3)
    m.set_inertia_target(c.xhat)
    cp = [2.0e3, 0.02, 1.5, 0.0, 0.0, -9.81]
    m.set_params(adm.MASS_SPRING, cp)
    vf, _ = pick_vf(c.faces, c.x, 40, seed=74)
    m.set_contacts(adm.MASS_SPRING, None, vf, KAPPA, DHAT, AREA, HSTEP)
    rp0, col0 = oracle.pattern(c.nV, c.faces)
    base = oracle.cloth_assemble(c.rest, c.faces, c.x, c.xhat, cp, rp0, col0)
    none = np.zeros((0, 2), np.int32)
    erp, ecol = oracle.extended_pattern(rp0, col0, none, vf)
    ref = oracle.add_interactions(base, c.x, none, KAPPA, DHAT, AREA, HSTEP, rp0, col0, vf)
    e, g, H, rp, col = gpu_eval(m, adm.MASS_SPRING, adm.FP64, c.x)
    assert np.array_equal(rp, erp) and np.array_equal(col, ecol)
    assert abs(e - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= 1e-12
    want = np.stack([ref["blocks"].get((r, int(cc)), np.zeros((3, 3))) for r in range(c.nV)
                     for cc in col[rp[r]:rp[r + 1]]])
    assert rel(H, want) <= 1e-12
    v = np.random.default_rng(9).normal(size=c.x.shape)
    xd = torch.from_numpy(np.ascontiguousarray(c.x).reshape(-1)).cuda()
    hv = torch.zeros_like(xd)
    m.eval_hvp(adm.MASS_SPRING, adm.FP64, xd, torch.from_numpy(v.reshape(-1)).cuda(), hv)
    torch.cuda.synchronize()
    hv_ref = np.zeros_like(c.x)
    for (r, cc), blk in ref["blocks"].items():
        hv_ref[r] += blk @ v[cc]
    assert rel(hv.cpu().numpy().reshape(-1, 3), hv_ref) <= 1e-12
    m.close()


def test_autotune_with_contacts_then_parity():
    """The tile-size autotuner runs the pass on the pattern the contact terms
    extend (its scratch Hessian sized for it) and rebuilds the tiles, which
    are then remapped to that pattern: the pass after it still matches."""
    V, F = synth.icosphere(3)
    x = synth.perturb(V, sigma=1e-2, seed=75)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.STVK_MEMBRANE, SHELL_P)
    vf, _ = pick_vf(F, x, 40, seed=76)
    m.set_contacts(adm.STVK_MEMBRANE, None, vf, KAPPA, DHAT, AREA, HSTEP)
    best, thr, ms = m.autotune(adm.STVK_MEMBRANE, adm.FP64, torch.from_numpy(x.reshape(-1)).cuda())
    assert best > 0 and thr == 256 and ms > 0
    got = gpu_eval(m, adm.STVK_MEMBRANE, adm.FP64, x)
    check(V, F, x, np.zeros((0, 2), np.int32), vf, got, False, 1e-12)
    m.close()
