"""Failure detection without a GPU fault: every device wait of the library is
bounded.  adm_check_bounded_wait runs the tiled kernel's bounded wait on a
barrier that nothing completes; it must give up (ADM_ERR_TIMEOUT) within a
few seconds, and the context must stay usable: a pass right after it still
matches the oracle."""
import time

import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def test_bounded_wait_gives_up_and_context_stays_usable():
    t0 = time.perf_counter()
    st = adm.check_bounded_wait()
    dt = time.perf_counter() - t0
    assert adm.STATUS[st] == "ADM_ERR_TIMEOUT"
    assert dt < 10.0
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=1e-2, seed=81)
    m = adm.Mesh(V, F, 3)
    m.set_params(adm.SHELL, [1e5, 0.3, 1e-3])
    _, nV, nnzb, _, _ = m.pattern(adm.SHELL)
    xd = torch.from_numpy(x.reshape(-1)).cuda()
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(nV * 3, dtype=torch.float64, device="cuda")
    H = torch.zeros(nnzb * 9, dtype=torch.float64, device="cuda")
    m.eval(adm.SHELL, adm.FP64, xd, e, g, H)
    torch.cuda.synchronize()
    assert m.status() == 0
    ref = oracle.Problem(V, F, oracle.SHELL, 3, params=[1e5, 0.3, 1e-3]).assemble(x)
    assert abs(e.item() - ref["energy"]) <= 1e-12 * abs(ref["energy"])
    assert rel(H.cpu().numpy().reshape(-1, 3, 3), ref["vals"]) <= 1e-12
    m.close()
