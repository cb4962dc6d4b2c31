"""Edge cases through the C ABI against the oracle: a vertex no triangle
references (zero gradient row, zero diagonal block), a batch with a mesh
that has vertices but no triangles (zero energy), and the smallest mesh (one
triangle), on the tiled and the atomic assembler.  FP64, 1e-12."""
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


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def evaluate(m, energy, x, batch=False):
    _, nV, nnzb, rp, col = m.pattern(energy)
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64).reshape(-1)).cuda()
    g = torch.full((nV * 3,), float("nan"), dtype=torch.float64, device="cuda")
    H = torch.full((nnzb * 9,), float("nan"), dtype=torch.float64, device="cuda")
    e = torch.zeros(m.n_mesh if batch else 1, dtype=torch.float64, device="cuda")
    if batch:
        m.eval_batch(energy, adm.FP64, xd, e, None, g, H)
    else:
        m.eval(energy, adm.FP64, xd, e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    return e.cpu().numpy(), g.cpu().numpy().reshape(-1, 3), H.cpu().numpy().reshape(-1, 3, 3), rp.cpu().numpy(), \
        col.cpu().numpy()


@pytest.mark.parametrize("assembler", [0, 1])
def test_unused_vertex(assembler):
    V, F = synth.icosphere(2)
    rest = np.concatenate([V, [[3.0, 0.0, 0.0]]])
    x = np.concatenate([synth.perturb(V, 1e-2, 71), [[3.1, 0.2, 0.0]]])
    m = adm.Mesh(rest, F, 3)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    m.set_params(adm.SHELL, SHELL_P)
    for _ in range(2):   # the second pass reuses buffers that held the first pass's values
        e, g, H, rp, col = evaluate(m, adm.SHELL, x)
    P = oracle.Problem(rest, F, oracle.SHELL, 3, params=SHELL_P)
    assert np.array_equal(rp, P.row_ptr) and np.array_equal(col, P.col)
    ref = P.assemble(x)
    v = len(rest) - 1
    assert np.all(g[v] == 0) and np.all(H[rp[v]:rp[v + 1]] == 0) and rp[v + 1] - rp[v] == 1
    assert rel(g, ref["grad"]) <= 1e-12 and rel(H, ref["vals"]) <= 1e-12
    m.close()


def test_batch_with_empty_mesh():
    a = synth.shell_batch([1, 2], sigma=1e-2, seed=72)
    extra = np.array([[9.0, 0.0, 0.0], [9.5, 0.0, 0.0], [9.0, 0.5, 0.0]])
    rest = np.concatenate([a.rest[:a.v_off[1]], extra, a.rest[a.v_off[1]:]])
    x = np.concatenate([a.x[:a.v_off[1]], extra, a.x[a.v_off[1]:]])
    faces = np.concatenate([a.faces[:a.f_off[1]], a.faces[a.f_off[1]:] + 3]).astype(np.int32)
    v_off = np.array([0, a.v_off[1], a.v_off[1] + 3, len(rest)])
    f_off = np.array([0, a.f_off[1], a.f_off[1], len(faces)])
    m = adm.Mesh(rest, faces, 3, v_off=v_off, f_off=f_off)
    m.set_params(adm.SHELL, SHELL_P)
    e, g, H, rp, col = evaluate(m, adm.SHELL, x, batch=True)
    P = oracle.Problem(rest, faces, oracle.SHELL, 3, params=SHELL_P)
    ref = P.assemble(x)
    assert e[1] == 0.0 and abs(e.sum() - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= 1e-12 and rel(H, ref["vals"]) <= 1e-12
    m.close()


@pytest.mark.parametrize("assembler", [0, 1])
def test_single_triangle(assembler):
    rest = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.2, 0.9, 0.0]])
    x = rest + np.array([[0.01, -0.02, 0.03], [0.1, 0.0, -0.05], [0.0, 0.04, 0.02]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    m = adm.Mesh(rest, F, 3)
    m.set_option(adm.OPT_ASSEMBLER, assembler)
    m.set_params(adm.STVK_MEMBRANE, SHELL_P)
    e, g, H, rp, col = evaluate(m, adm.STVK_MEMBRANE, x)
    P = oracle.Problem(rest, F, oracle.STVK, 3, params=SHELL_P)
    ref = P.assemble(x)
    assert abs(e[0] - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert rel(g, ref["grad"]) <= 1e-12 and rel(H, ref["vals"]) <= 1e-12
    m.close()
