"""Parity at the full sizes of the timed workloads, in the launch
configuration the bench times, on outputs the oracle can recompute piece by
piece:

* the 700-icosphere shell batch (2.16M vertices, FP32, default tiles), the
  shell and its bending term alone: sampled meshes, each recomputed alone by
  the oracle (per-mesh energy and gradient norm, its gradient rows and
  Hessian block rows; its rows of the batch pattern bit-exact against the
  oracle's pattern shifted by the mesh's first vertex);
* the 1M-triangle ARAP residual disk (FP32): sampled triangles, their four
  residual rows and 24 Jacobian entries (values and columns) recomputed by
  the oracle on those triangles alone;
* the matrix-free product on the whole shell batch: sampled meshes' H v
  rows against the oracle's mesh Hessian times v;
* the batch with 100k vertex-vertex and 100k vertex-face contact terms:
  sampled meshes' rows of the extended pattern and their values;
* the filtered pass on the whole batch: sampled meshes against the oracle's
  per-element projection;
* the 1000 x 1000 mass-spring cloth, whole;
* the shell batch in FP64: sampled meshes at 1e-12;
* the learned membrane with weights trained by the bench's recipe, on the
  bench's batch and on the batch stretched inside the training range:
  sampled meshes (and sampled rows of a 160-tile mesh) against the oracle's
  network on the same BF16 weights."""
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
TOL = 2e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def batch_eval(m, energy, x32):
    _, nV, nnzb, rp, col = m.pattern(energy)
    xd = torch.from_numpy(x32).cuda()
    e = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda")
    gn = torch.zeros_like(e)
    g = torch.full((nV * 3,), float("nan"), device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), device="cuda")
    m.eval_batch(energy, adm.FP32, xd, e, gn, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    assert not torch.isnan(H).any() and not torch.isnan(g).any()     # every output written
    return (rp.cpu().numpy(), col.cpu().numpy(), e.cpu().numpy(), gn.cpu().numpy(),
            g.cpu().numpy().reshape(-1, 3), H.cpu().numpy().reshape(-1, 3, 3))


# the shell, and its bending term alone: the hinge Hessian is about 1e-8 of
# the membrane's, so only a separate check sees its errors
@pytest.mark.parametrize("energy,params", [(adm.SHELL, SHELL_P), (adm.HINGE_BENDING, [0.5, 1.0])])
def test_shell_batch_700_sampled_meshes_fp32(energy, params):
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x32 = b.x.astype(np.float32)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(energy, params)
    rp, col, e, gn, g, H = batch_eval(m, energy, x32)
    nv_mesh = np.diff(b.v_off)
    rng = np.random.default_rng(7)
    big = np.flatnonzero(nv_mesh == nv_mesh.max())
    small = np.flatnonzero(nv_mesh == nv_mesh.min())
    picks = [int(rng.choice(big)), int(rng.choice(small)), int(rng.choice(small)), b.n_mesh - 1]
    orc = oracle.SHELL if energy == adm.SHELL else oracle.HINGE
    for k in picks:
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, orc, 3, params=params)
        ref = P.assemble(x32[v0:v1].astype(np.float64))          # hyper-dual route: every Hessian
        blk = slice(rp[v0], rp[v1])
        assert np.array_equal(rp[v0:v1 + 1] - rp[v0], P.row_ptr) and np.array_equal(col[blk] - v0, P.col)
        assert abs(e[k] - ref["energy"]) <= TOL * abs(ref["energy"])
        assert rel(g[v0:v1], ref["grad"]) <= TOL
        assert abs(gn[k] - np.linalg.norm(ref["grad"])) <= TOL * np.linalg.norm(ref["grad"])
        assert rel(H[blk], ref["vals"]) <= TOL
    m.close()


def test_arap_disk_1m_sampled_triangles_fp32():
    d = synth.noisy_disk()
    m = adm.Mesh(d.rest, d.faces, 2)
    nr, nc, nnz, jrp, jcol = m.jac_pattern()
    _, nV, nnzb, _, _ = m.pattern(adm.ARAP2D_RESIDUAL)
    x32 = d.x.astype(np.float32)
    r = torch.zeros(nr, device="cuda")
    jv = torch.zeros(nnz, device="cuda")
    jtj = torch.zeros(nnzb * 4, device="cuda")
    m.eval_jacobian(adm.ARAP2D_RESIDUAL, adm.FP32, torch.from_numpy(x32).cuda(), r, jv, jtj)
    torch.cuda.synchronize()
    assert m.status() == 0
    r, jv, jcol = r.cpu().numpy(), jv.cpu().numpy(), jcol.cpu().numpy()
    ts = np.sort(np.random.default_rng(8).choice(d.faces.shape[0], 500, replace=False))
    P = oracle.Problem(d.rest, d.faces[ts], oracle.ARAP, 2)
    ref = P.arap_jacobian(x32.astype(np.float64))
    rows = (4 * ts[:, None] + np.arange(4)).ravel()
    ents = (24 * ts[:, None] + np.arange(24)).ravel()
    assert rel(r[rows], ref["r"]) <= TOL
    assert rel(jv[ents], ref["val"]) <= TOL
    assert np.array_equal(jcol[ents], ref["col"])
    m.close()


def test_shell_batch_700_hvp_sampled_meshes_fp32():
    """The matrix-free product on the whole batch (the bench's H v line):
    sampled meshes' H v rows against the oracle's assembled Hessian of that
    mesh times v."""
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x32 = b.x.astype(np.float32)
    v32 = np.random.default_rng(7).normal(size=x32.shape).astype(np.float32)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    xd = torch.from_numpy(x32.reshape(-1)).cuda()
    vd = torch.from_numpy(v32.reshape(-1)).cuda()
    hv = torch.full_like(xd, float("nan"))
    m.eval_hvp(adm.SHELL, adm.FP32, xd, vd, hv)
    torch.cuda.synchronize()
    assert m.status() == 0 and not torch.isnan(hv).any()
    hv = hv.cpu().numpy().reshape(-1, 3)
    nv_mesh = np.diff(b.v_off)
    rng = np.random.default_rng(9)
    picks = [int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.max()))),
             int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.min())))]
    for k in picks:
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.SHELL, 3, params=SHELL_P)
        ref = P.assemble(x32[v0:v1].astype(np.float64))
        vm = v32[v0:v1].astype(np.float64)
        want = np.zeros_like(vm)
        for r in range(P.nV):
            for q in range(P.row_ptr[r], P.row_ptr[r + 1]):
                want[r] += ref["vals"][q] @ vm[P.col[q]]
        assert rel(hv[v0:v1], want) <= TOL
    m.close()


def contact_terms(b, seed):
    """Vertex-vertex pairs and vertex-face elements drawn within meshes of the
    batch (as the bench's contact workload draws them)."""
    rng = np.random.default_rng(seed)
    nv_mesh, nf_mesh = np.diff(b.v_off), np.diff(b.f_off)
    mi = rng.integers(b.n_mesh, size=150_000)
    pi = b.v_off[mi] + rng.integers(nv_mesh[mi])
    pj = b.v_off[mi] + rng.integers(nv_mesh[mi])
    keep = pi != pj
    pr = np.unique(np.sort(np.stack([pi[keep], pj[keep]], axis=1), axis=1), axis=0)
    pr = rng.permutation(pr)[:100_000].astype(np.int32)
    mi = rng.integers(b.n_mesh, size=110_000)
    vp = b.v_off[mi] + rng.integers(nv_mesh[mi])
    fq = b.faces[b.f_off[mi] + rng.integers(nf_mesh[mi])]
    keep = (fq != vp[:, None]).all(axis=1)
    vf = np.concatenate([vp[keep, None], fq[keep]], axis=1)[:100_000].astype(np.int32)
    return pr, vf


def test_shell_batch_700_with_contacts_sampled_meshes_fp32():
    """100k vertex-vertex and 100k vertex-face terms on the whole batch (the
    bench's contact line): sampled meshes' rows of the extended pattern
    bit-exact, and their energies, gradient rows and Hessian rows against the
    oracle's mesh terms plus the contact terms inside that mesh."""
    kappa, dhat, area, hstep = 1.0e3, 0.2, 1e-3, 1.0
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x32 = b.x.astype(np.float32)
    pr, vf = contact_terms(b, 9)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_contacts(adm.SHELL, pr, vf, kappa, dhat, area, hstep)
    rp, col, e, gn, g, H = batch_eval(m, adm.SHELL, x32)
    nv_mesh = np.diff(b.v_off)
    rng = np.random.default_rng(10)
    picks = [int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.max()))),
             int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.min())))]
    for k in picks:
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        pk = pr[(pr[:, 0] >= v0) & (pr[:, 0] < v1)] - v0
        qk = vf[(vf[:, 0] >= v0) & (vf[:, 0] < v1)] - v0
        xk = x32[v0:v1].astype(np.float64)
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.SHELL, 3, params=SHELL_P)
        base = P.assemble(xk)
        erp, ecol = oracle.extended_pattern(P.row_ptr, P.col, pk, qk)
        ref = oracle.add_interactions(base, xk, pk, kappa, dhat, area, hstep, P.row_ptr, P.col, qk)
        blk = slice(rp[v0], rp[v1])
        assert np.array_equal(rp[v0:v1 + 1] - rp[v0], erp) and np.array_equal(col[blk] - v0, ecol)
        assert abs(e[k] - ref["energy"]) <= TOL * abs(ref["energy"])
        assert rel(g[v0:v1], ref["grad"]) <= TOL
        want = np.stack([ref["blocks"].get((r, int(c)), np.zeros((3, 3)))
                         for r in range(P.nV) for c in ecol[erp[r]:erp[r + 1]]])
        assert rel(H[blk], want) <= TOL
    m.close()


def test_shell_batch_700_filtered_sampled_meshes_fp32():
    """Per-term Hessian filtering on the whole batch (the bench's filtered
    line): two sampled meshes against the oracle's per-element eigh
    projection."""
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x32 = b.x.astype(np.float32)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    m.set_projection(True, 0.0)
    rp, col, e, gn, g, H = batch_eval(m, adm.SHELL, x32)
    nv_mesh = np.diff(b.v_off)
    small = np.flatnonzero(nv_mesh == nv_mesh.min())
    for k in np.random.default_rng(11).choice(small, 2, replace=False):
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.SHELL, 3, params=SHELL_P)
        ref = P.assemble_projected(x32[v0:v1].astype(np.float64), 0.0)
        blk = slice(rp[v0], rp[v1])
        assert rel(H[blk], ref["vals"]) <= TOL
        assert rel(g[v0:v1], ref["grad"]) <= TOL
    m.close()


def test_cloth_1000_full_fp32():
    """The largest cloth of the bench (1000 x 1000 vertices, 3M springs,
    FP32), whole: energy, gradient and every Hessian block against the
    oracle."""
    c = synth.cloth_grid(1000, sigma=0.05, seed=6)
    cp = [1.0e4, 1.0 / 60.0, 1.0, 0.0, 0.0, -9.81]
    m = adm.Mesh(c.rest, c.faces, 3)
    m.set_inertia_target(c.xhat)
    m.set_params(adm.MASS_SPRING, cp)
    x32 = c.x.astype(np.float32)
    _, nV, nnzb, rp, col = m.pattern(adm.MASS_SPRING)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.full((nV * 3,), float("nan"), device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), device="cuda")
    m.eval(adm.MASS_SPRING, adm.FP32, torch.from_numpy(x32.reshape(-1)).cuda(), e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    orp, ocol = oracle.pattern(c.nV, c.faces)
    assert np.array_equal(rp.cpu().numpy(), orp) and np.array_equal(col.cpu().numpy(), ocol)
    ref = oracle.cloth_assemble(c.rest, c.faces, x32.astype(np.float64), c.xhat, cp, orp, ocol)
    assert abs(e.item() - ref["energy"]) <= TOL * abs(ref["energy"])
    assert rel(g.cpu().numpy().reshape(-1, 3), ref["grad"]) <= TOL
    assert rel(H.cpu().numpy().reshape(-1, 3, 3), ref["vals"]) <= TOL
    m.close()


def test_shell_batch_700_sampled_meshes_fp64():
    """The FP64 form of the shell batch (the bench's FP64 line): sampled
    meshes against the oracle at the FP64 bar."""
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x64 = b.x.astype(np.float32).astype(np.float64)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    _, nV, nnzb, rp, col = m.pattern(adm.SHELL)
    e = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda")
    gn = torch.zeros_like(e)
    g = torch.full((nV * 3,), float("nan"), dtype=torch.float64, device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), dtype=torch.float64, device="cuda")
    m.eval_batch(adm.SHELL, adm.FP64, torch.from_numpy(x64).cuda(), e, gn, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0 and not torch.isnan(H).any() and not torch.isnan(g).any()
    rp, e, gn = rp.cpu().numpy(), e.cpu().numpy(), gn.cpu().numpy()
    g, H = g.cpu().numpy().reshape(-1, 3), H.cpu().numpy().reshape(-1, 3, 3)
    nv_mesh = np.diff(b.v_off)
    rng = np.random.default_rng(12)
    picks = [int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.max()))),
             int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.min()))), b.n_mesh - 1]
    for k in picks:
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.SHELL, 3, params=SHELL_P)
        ref = P.assemble(x64[v0:v1])
        blk = slice(rp[v0], rp[v1])
        assert abs(e[k] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
        assert rel(g[v0:v1], ref["grad"]) <= 1e-12
        assert abs(gn[k] - np.linalg.norm(ref["grad"])) <= 1e-12 * np.linalg.norm(ref["grad"])
        assert rel(H[blk], ref["vals"]) <= 1e-12
    m.close()


def _bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def _train_bench_recipe():
    """The bench's learned-membrane training: 2^20 samples (stretches in
    [0.7, 1.4], seed 5) with the library's analytic Neo-Hookean targets,
    20,000 Adam steps of 8,192 (reshuffled every epoch), gradient weight 4,
    lr 3e-3 decaying geometrically to 3e-5, seeded start (the bench's recipe)."""
    ns = 1 << 20
    Fs = torch.from_numpy(synth.membrane_samples(ns, seed=5).reshape(ns, 6).astype(np.float32)).cuda()
    Ig = torch.zeros((ns, 3), device="cuda")
    pg = torch.zeros(ns, device="cuda")
    gg = torch.zeros((ns, 3), device="cuda")
    adm.MLP.nh_targets(Fs, SHELL_P[0], SHELL_P[1], Ig, pg, gg)
    norm = torch.cat([Ig.mean(0), Ig.std(0), pg.mean()[None], pg.std()[None]]).contiguous()
    rng = np.random.default_rng(0)
    th0 = np.zeros(adm.MLP_NPARAM, dtype=np.float32)
    th0[:192] = rng.normal(scale=0.6, size=192)
    th0[256:4352] = rng.normal(scale=1 / 8, size=4096)
    th0[4416:4480] = rng.normal(scale=1 / 8, size=64)
    th = torch.from_numpy(th0).cuda()
    adm.MLP.train(th, norm, Ig, pg, gg, steps=20000, batch=8192, beta=4.0, lr0=3e-3, lr_end=3e-5)
    torch.cuda.synchronize()
    return th, norm


@pytest.mark.parametrize("deform", ["bench", "in_range"])
def test_learned_membrane_batch_700_trained_sampled_meshes(deform):
    """The timed learned-membrane path -- per-triangle network table, then the
    tiled composition -- with trained weights on the whole 700-mesh batch,
    against the oracle's network on the same BF16 weights (FP64, no
    activation rounding; reading: BF16-level agreement, 3e-2).  Sampled
    meshes: two of the smallest and the last one whole (energy, gradient rows,
    Hessian rows), and 200 sampled vertices of a level-6 mesh (160 tiles):
    their gradient and Hessian rows.

    On the bench's batch (within 1e-3 of rest) the gradient is left out: the
    terms psi_a dI_a/dx of a stress-free state cancel to about 1e-3 of their
    size, so the BF16 rounding of the network's activations (about 1e-3 of
    psi_a) is of the order of the gradient itself.  The batch stretched inside
    the training range checks the gradient on the level-4 meshes; on the
    level-6 mesh a homogeneous stretch leaves each vertex only the net force
    of its ring, about h/R = 1/64 of the element forces, which amplifies the
    same rounding, so there its Hessian rows alone are checked."""
    b = synth.shell_batch(synth.shell_batch_levels("paper"), sigma=1e-3, seed=4)
    x = b.x if deform == "bench" else synth.stretched_batch(b)
    x32 = x.astype(np.float32)
    th, norm = _train_bench_recipe()
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.MLP_MEMBRANE, SHELL_P)
    m.mlp_attach(th, norm)
    rp, col, e, gn, g, H = batch_eval(m, adm.MLP_MEMBRANE, x32)
    oracle.mlp_set(_bf16(th.cpu().numpy()), norm.cpu().numpy().astype(np.float64))
    nv_mesh = np.diff(b.v_off)
    rng = np.random.default_rng(13)
    small = np.flatnonzero(nv_mesh == nv_mesh.min())
    whole = [int(k) for k in rng.choice(small[small != b.n_mesh - 1], 2, replace=False)] + [b.n_mesh - 1]
    for k in whole:
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.MLP, 3, params=SHELL_P)
        ref = P.assemble(x32[v0:v1].astype(np.float64))
        blk = slice(rp[v0], rp[v1])
        assert abs(e[k] - ref["energy"]) <= 3e-2 * abs(ref["energy"]), (k, e[k], ref["energy"])
        if deform == "in_range":
            assert rel(g[v0:v1], ref["grad"]) <= 3e-2
        assert rel(H[blk], ref["vals"]) <= 3e-2
    k = int(rng.choice(np.flatnonzero(nv_mesh == nv_mesh.max())))
    v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
    P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.MLP, 3, params=SHELL_P)
    rows = np.sort(rng.choice(P.nV, 200, replace=False))
    ref = P.assemble(x32[v0:v1].astype(np.float64), rows=rows)
    bl = np.concatenate([np.arange(P.row_ptr[r], P.row_ptr[r + 1]) for r in rows])
    Hm = H[rp[v0]:rp[v1]]
    assert rel(Hm[bl], ref["vals"][bl]) <= 3e-2
    # the other network kernel on the whole batch: the same BF16 network,
    # FP32 contractions summed in another order (mma.sync against tcgen05)
    m.set_option(adm.OPT_MLP_NET, 1)
    _, _, e2, _, g2, H2 = batch_eval(m, adm.MLP_MEMBRANE, x32)
    m.set_option(adm.OPT_MLP_NET, 0)
    _, _, e0, _, g0, H0 = batch_eval(m, adm.MLP_MEMBRANE, x32)
    assert rel(e2, e0) <= 2e-3 and rel(H2, H0) <= 2e-3
    if deform == "in_range":
        assert rel(g2, g0) <= 2e-3
    m.close()
