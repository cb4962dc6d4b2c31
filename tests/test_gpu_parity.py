"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle
on the same seeded inputs.

Bars (stated by the workloads' definitions):
  * block pattern, slot map and hinge list: bit-exact;
  * FP64 path: relative error <= 1e-12 (energy |dF|/|F|, gradient |dg|/|g|,
    Hessian Frobenius |dH|/|H| of the assembled matrix);
  * FP32 path: <= 2e-5 relative Frobenius per assembled Hessian, checked on
    the total and on every term separately.
The oracle consumes the FP32-rounded x widened to FP64, so the FP32 check
measures kernel arithmetic, not input rounding."""
import numpy as np
import pytest

import oracle
import synth
from util import oracle_slots, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

TOL = {adm.FP64: 1e-12, adm.FP32: 2e-5}
NP = {adm.FP64: np.float64, adm.FP32: np.float32}
TT = {adm.FP64: torch.float64, adm.FP32: torch.float32}
ORC = {adm.SYMDIR2D: oracle.SYMDIR, adm.STVK_MEMBRANE: oracle.STVK, adm.HINGE_BENDING: oracle.HINGE,
       adm.SHELL: oracle.SHELL, adm.NH_MEMBRANE: oracle.NH, adm.AREA: oracle.AREA}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def gpu_eval(m: adm.Mesh, energy, prec, x, hess=True, grad=True, batch=False):
    vd = m.var_dim
    _, nV, nnzb, rp, col = m.pattern(energy)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=NP[prec])).cuda()
    g = torch.full((nV * vd,), float("nan"), dtype=TT[prec], device="cuda") if grad else None
    H = torch.full((nnzb * vd * vd,), float("nan"), dtype=TT[prec], device="cuda") if hess else None
    if batch:
        e = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda")
        gn = torch.zeros(m.n_mesh, dtype=torch.float64, device="cuda") if grad else None
        m.eval_batch(energy, prec, xd, e, gn, g, H)
    else:
        e = torch.zeros(1, dtype=torch.float64, device="cuda")
        gn = None
        m.eval(energy, prec, xd, e, g, H)
    torch.cuda.synchronize()
    out = {"status": m.status(), "energy": e.cpu().numpy(), "rp": rp.cpu().numpy(), "col": col.cpu().numpy()}
    if grad:
        out["grad"] = g.cpu().numpy().reshape(nV, vd)
    if hess:
        out["vals"] = H.cpu().numpy().reshape(nnzb, vd, vd)
    if gn is not None:
        out["gnorm"] = gn.cpu().numpy()
    return out


def check(energy, prec, rest, faces, x, vd, params=None, tol=None, assembler=0, tile_tris=None, threads=None):
    tol = TOL[prec] if tol is None else tol
    m = adm.Mesh(rest, faces, vd)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    if tile_tris is not None:
        m.set_option(adm.OPT_TILE_TRIS, tile_tris)
    if threads is not None:
        m.set_option(adm.OPT_TILE_THREADS, threads)
    if params is not None:
        m.set_params(energy, params)
    xr = np.asarray(x, dtype=NP[prec])
    out = gpu_eval(m, energy, prec, xr)
    assert out["status"] == 0
    P = oracle.Problem(rest, faces, ORC[energy], vd, params=params)
    ref = P.assemble(xr.astype(np.float64))
    assert ref["n_domain_err"] == 0
    assert np.array_equal(out["rp"], P.row_ptr) and np.array_equal(out["col"], P.col)
    assert np.array_equal(m.slot_map(energy).cpu().numpy(), oracle_slots(P, ORC[energy]))
    assert abs(out["energy"][0] - ref["energy"]) <= tol * abs(ref["energy"])
    assert rel(out["grad"], ref["grad"]) <= tol, rel(out["grad"], ref["grad"])
    assert rel(out["vals"], ref["vals"]) <= tol, rel(out["vals"], ref["vals"])
    m.close()
    return out, ref


# ---------------------------------------------------------------- C1 -------
ASSEMBLERS = [0, 1]   # 0 tiled (default), 1 per-element atomic scatter


@pytest.mark.parametrize("assembler", ASSEMBLERS)
@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_symdir_grid33(prec, assembler):
    g = synth.grid_uv()
    check(adm.SYMDIR2D, prec, g.rest, g.faces, g.x, 2, assembler=assembler)


def test_symdir_identity_exact():
    g = synth.grid_uv(33, 0.0, 1)
    m = adm.Mesh(g.rest, g.faces, 2)
    out = gpu_eval(m, adm.SYMDIR2D, adm.FP64, g.rest[:, :2])
    assert abs(out["energy"][0] - 4.0) < 1e-12
    assert np.abs(out["grad"]).max() < 1e-12


def test_symdir_folded_map_is_domain_error():
    g = synth.grid_uv(33, 0.01, 1, relative=False)
    m = adm.Mesh(g.rest, g.faces, 2)
    out = gpu_eval(m, adm.SYMDIR2D, adm.FP64, g.x)
    assert out["status"] == -3                                     # ADM_ERR_DOMAIN
    # folded elements contribute nothing; the rest still matches the oracle
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    ref = P.assemble(g.x)
    assert ref["n_domain_err"] > 0
    assert abs(out["energy"][0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert rel(out["vals"], ref["vals"]) <= 1e-12


# ---------------------------------------------------------------- C2 -------
SHELL_P = [1.0e5, 0.3, 1.0e-3]


@pytest.mark.parametrize("assembler", ASSEMBLERS)
@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
@pytest.mark.parametrize("energy", [adm.STVK_MEMBRANE, adm.HINGE_BENDING, adm.SHELL, adm.NH_MEMBRANE,
                                    adm.AREA])
def test_shell_terms_icosphere3(energy, prec, assembler):
    v, f = synth.icosphere(3)
    x = synth.perturb(v, 1e-2, 2)
    params = None if energy == adm.AREA else (SHELL_P if energy != adm.HINGE_BENDING else None)
    check(energy, prec, v, f, x, 3, params=params, assembler=assembler)


@pytest.mark.parametrize("tile_tris", [32, 100, 777, 4096])
def test_tile_sizes_shell_fp64(tile_tris):
    """Tiny tiles make most blocks shared between tiles (pre-zeroed, atomic
    adds); huge tiles make one tile per mesh.  Every size gives the oracle's
    result to FP64 rounding."""
    v, f = synth.icosphere(4)
    x = synth.perturb(v, 1e-2, 5)
    check(adm.SHELL, adm.FP64, v, f, x, 3, params=SHELL_P, tile_tris=tile_tris)


@pytest.mark.parametrize("tile_tris", [32, 512])
def test_tile_sizes_symdir_fp64(tile_tris):
    g = synth.grid_uv()
    check(adm.SYMDIR2D, adm.FP64, g.rest, g.faces, g.x, 2, tile_tris=tile_tris)


def test_hinge_list_bit_exact():
    v, f = synth.icosphere(4)
    m = adm.Mesh(v, f, 3)
    assert np.array_equal(m.hinges().cpu().numpy(), oracle.hinges(v.shape[0], f))


@pytest.mark.parametrize("assembler", ASSEMBLERS)
def test_open_mesh_hinges_and_pattern(assembler):
    d = synth.noisy_disk(2000)
    x = d.rest + synth.perturb(np.zeros_like(d.rest), 1e-3, 9)
    check(adm.SHELL, adm.FP64, d.rest, d.faces, x, 3, params=[1.0e3, 0.3, 0.01, 0.5, 1.0],
          assembler=assembler)
    check(adm.HINGE_BENDING, adm.FP64, d.rest, d.faces, x, 3, params=[0.5, 1.0], assembler=assembler)


def test_shell_level7_sampled_rows_fp32():
    """Full-size elastic shell (icosphere level 7, FP32): the whole energy
    against the oracle, and 200 sampled block rows of the Hessian and the
    gradient recomputed by the oracle from every element touching them."""
    sh = synth.icosphere_shell(7)
    x32 = sh.x.astype(np.float32)
    m = adm.Mesh(sh.rest, sh.faces, 3)
    m.set_params(adm.SHELL, SHELL_P)
    out = gpu_eval(m, adm.SHELL, adm.FP32, x32)
    assert out["status"] == 0
    P = oracle.Problem(sh.rest, sh.faces, oracle.SHELL, 3, params=SHELL_P)
    assert np.array_equal(out["rp"], P.row_ptr) and np.array_equal(out["col"], P.col)
    e_ref = P.assemble(x32.astype(np.float64), route=1, hessian=False)
    assert abs(out["energy"][0] - e_ref["energy"]) <= 2e-5 * abs(e_ref["energy"])
    assert rel(out["grad"], e_ref["grad"]) <= 2e-5
    rows = np.random.default_rng(0).choice(P.nV, 200, replace=False)
    ref = P.assemble(x32.astype(np.float64), rows=rows)
    sel = np.concatenate([np.arange(P.row_ptr[r], P.row_ptr[r + 1]) for r in rows])
    assert rel(out["vals"][sel], ref["vals"][sel]) <= 2e-5
    assert rel(out["grad"][rows], ref["grad"][rows]) <= 2e-5


# ------------------------------------------------------------ modes ---------
@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_value_and_gradient_modes_match_full(prec):
    v, f = synth.icosphere(3)
    x = synth.perturb(v, 1e-2, 3)
    m = adm.Mesh(v, f, 3)
    full = gpu_eval(m, adm.SHELL, prec, x)
    gonly = gpu_eval(m, adm.SHELL, prec, x, hess=False)
    vonly = gpu_eval(m, adm.SHELL, prec, x, hess=False, grad=False)
    # the same arithmetic; FP32 may differ in the last bits where the compiler
    # contracts the value path differently once derivatives are dead code
    assert abs(full["energy"][0] - gonly["energy"][0]) <= TOL[prec] * abs(full["energy"][0])
    assert abs(full["energy"][0] - vonly["energy"][0]) <= TOL[prec] * abs(full["energy"][0])
    assert rel(gonly["grad"], full["grad"]) <= TOL[prec]


# ------------------------------------------------------------ batch ---------
@pytest.mark.parametrize("assembler", ASSEMBLERS)
@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_batch_per_mesh_energy_and_gnorm(prec, assembler):
    b = synth.shell_batch([1, 3, 2, 4, 0, 3], sigma=1e-2, seed=11)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    m.set_params(adm.SHELL, SHELL_P)
    xr = b.x.astype(NP[prec])
    out = gpu_eval(m, adm.SHELL, prec, xr, batch=True)
    assert out["status"] == 0
    P = oracle.Problem(b.rest, b.faces, oracle.SHELL, 3, params=SHELL_P)
    ref = P.assemble(xr.astype(np.float64), per_element=True)
    tol = TOL[prec]
    assert rel(out["vals"], ref["vals"]) <= tol
    ee = ref["elem_energy"]
    tri_mesh = np.searchsorted(b.f_off, np.arange(P.nT), side="right") - 1
    hinge_mesh = np.searchsorted(b.v_off, P.H[:, 0], side="right") - 1
    e_mesh = np.bincount(tri_mesh, ee[:P.nT], b.n_mesh) + np.bincount(hinge_mesh, ee[P.nT:], b.n_mesh)
    assert np.all(np.abs(out["energy"] - e_mesh) <= tol * np.abs(e_mesh))
    for k in range(b.n_mesh):
        gk = ref["grad"][b.v_off[k]:b.v_off[k + 1]]
        assert abs(out["gnorm"][k] - np.linalg.norm(gk)) <= tol * np.linalg.norm(gk)


@pytest.mark.parametrize("levels,assembler,contacts",
                         [([2, 3], 0, False), ([1, 2, 3, 1, 2, 2, 3], 0, False), ([2, 1, 3], 1, False),
                          ([2, 2, 1], 0, True)])
def test_host_buffer_path_matches_device_path(levels, assembler, contacts):
    """adm_eval_batch_host feeds a tiled batch in up to four mesh ranges whose
    copies overlap the kernels of earlier ranges; the atomic assembler, and a
    pass with contact terms, take x whole.  All must give the device path's
    results (energies bitwise: the same tiles and partial sums)."""
    b = synth.shell_batch(levels, sigma=1e-2, seed=12)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    if contacts:  # pairs across the first two meshes, whatever their distance
        pairs = np.array([[i, b.v_off[1] + i] for i in range(0, 40, 3)], dtype=np.int32)
        m.set_contacts(adm.SHELL, pairs, None, 1.0e3, 10.0, 0.05, 0.1)
    dev = gpu_eval(m, adm.SHELL, adm.FP32, b.x.astype(np.float32), batch=True)
    nnzb = dev["vals"].shape[0]
    x = np.ascontiguousarray(b.x.astype(np.float32))
    e = np.zeros(b.n_mesh)
    gn = np.zeros(b.n_mesh)
    g = np.zeros(b.nV * 3, dtype=np.float32)
    H = np.zeros(nnzb * 9, dtype=np.float32)
    m.eval_batch_host(adm.SHELL, adm.FP32, x, e, gn, g, H)
    assert np.array_equal(e, dev["energy"])
    assert rel(g.reshape(-1, 3), dev["grad"]) <= 1e-6
    assert rel(H.reshape(-1, 3, 3), dev["vals"]) <= 1e-6
    assert np.allclose(gn, dev["gnorm"], rtol=1e-6)


# ---------------------------------------------------------------- C3 -------
@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_arap_jacobian_and_jtj(prec):
    scipy_sparse = pytest.importorskip("scipy.sparse")
    d = synth.noisy_disk(3000)
    m = adm.Mesh(d.rest, d.faces, 2)
    nr, nc, nnz, jrp, jcol = m.jac_pattern()
    _, nV, nnzb, rp, col = m.pattern(adm.ARAP2D_RESIDUAL)
    xr = d.x.astype(NP[prec])
    xd = torch.from_numpy(np.ascontiguousarray(xr)).cuda()
    r = torch.zeros(nr, dtype=TT[prec], device="cuda")
    jv = torch.zeros(nnz, dtype=TT[prec], device="cuda")
    jtj = torch.zeros(nnzb * 4, dtype=TT[prec], device="cuda")
    m.eval_jacobian(adm.ARAP2D_RESIDUAL, prec, xd, r, jv, jtj)
    torch.cuda.synchronize()
    assert m.status() == 0
    P = oracle.Problem(d.rest, d.faces, oracle.ARAP, 2)
    ref = P.arap_jacobian(xr.astype(np.float64))
    assert np.array_equal(jrp.cpu().numpy(), ref["row_ptr"]) and np.array_equal(jcol.cpu().numpy(), ref["col"])
    tol = TOL[prec]
    assert rel(r.cpu().numpy(), ref["r"]) <= tol
    assert rel(jv.cpu().numpy(), ref["val"]) <= tol
    J = scipy_sparse.csr_matrix((ref["val"], ref["col"], ref["row_ptr"]), shape=(nr, nc))
    JtJ = (J.T @ J).toarray()                       # independent route: SpGEMM of the assembled J
    Hd = oracle.bsr_to_dense(nV, 2, rp.cpu().numpy(), col.cpu().numpy(),
                             jtj.cpu().numpy().reshape(-1, 2, 2).astype(np.float64))
    assert rel(Hd, JtJ) <= tol


# ------------------------------------------------- graphs and autotuning ---
def test_graph_replay_matches_direct_launch():
    b = synth.shell_batch([2, 3, 1], sigma=1e-2, seed=21)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    direct = gpu_eval(m, adm.SHELL, adm.FP64, b.x, batch=True)
    m.set_option(adm.OPT_GRAPH, 1)
    _, nV, nnzb, _, _ = m.pattern(adm.SHELL)
    xd = torch.from_numpy(b.x.astype(np.float64)).cuda()
    e = torch.zeros(b.n_mesh, dtype=torch.float64, device="cuda")
    gn = torch.zeros(b.n_mesh, dtype=torch.float64, device="cuda")
    g = torch.zeros(nV * 3, dtype=torch.float64, device="cuda")
    H = torch.zeros(nnzb * 9, dtype=torch.float64, device="cuda")
    for _ in range(3):                      # capture, then replays with the same buffers
        H.fill_(float("nan"))
        m.eval_batch(adm.SHELL, adm.FP64, xd, e, gn, g, H)
        torch.cuda.synchronize()
        assert m.status() == 0
        assert rel(H.cpu().numpy().reshape(-1, 3, 3), direct["vals"]) <= 1e-13
        assert np.allclose(e.cpu().numpy(), direct["energy"], rtol=1e-13)
        assert np.allclose(gn.cpu().numpy(), direct["gnorm"], rtol=1e-13)
    # new contents in the same buffer: the replay reads them
    x2 = synth.perturb(b.rest, 2e-2, 99)
    xd.copy_(torch.from_numpy(x2))
    m.eval_batch(adm.SHELL, adm.FP64, xd, e, gn, g, H)
    torch.cuda.synchronize()
    m2 = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m2.set_params(adm.SHELL, SHELL_P)
    ref = gpu_eval(m2, adm.SHELL, adm.FP64, x2, batch=True)
    assert rel(H.cpu().numpy().reshape(-1, 3, 3), ref["vals"]) <= 1e-13


@pytest.mark.parametrize("tile", [48, 112, 224])
def test_shell_128_thread_tiles_fp32(tile):
    """The autotuner's second axis: 128-thread blocks (several units per
    thread when the tile is larger than the block), still at the FP32 bar."""
    sh = synth.icosphere_shell(4, sigma=1e-2, seed=31)
    check(adm.SHELL, adm.FP32, sh.rest, sh.faces, sh.x, 3, params=SHELL_P, tile_tris=tile, threads=128)


def test_autotune_picks_a_candidate_and_stays_correct():
    b = synth.shell_batch([3, 4, 3, 2], sigma=1e-2, seed=22)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.SHELL, SHELL_P)
    xd = torch.from_numpy(b.x.astype(np.float32)).cuda()
    best, thr, ms = m.autotune(adm.SHELL, adm.FP32, xd)
    assert (thr, best) in [(256, u) for u in (96, 128, 160, 192, 224)] + [(128, u) for u in (48, 64, 96, 112)]
    assert ms > 0
    out = gpu_eval(m, adm.SHELL, adm.FP32, b.x.astype(np.float32), batch=True)
    P = oracle.Problem(b.rest, b.faces, oracle.SHELL, 3, params=SHELL_P)
    ref = P.assemble(b.x.astype(np.float32).astype(np.float64))
    assert rel(out["vals"], ref["vals"]) <= 2e-5
