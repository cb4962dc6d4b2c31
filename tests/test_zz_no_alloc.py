"""adm_grad_norm_noalloc: the FP64 gradient-norm reduction for callers that
cannot allocate device memory where they need it (in a loop with a fixed
memory budget, inside a host framework that owns the device's memory, under
a host-owned allocator).  Its
scratch is a static device array of the library, so it needs no handle and
calls no cudaMalloc.  It must give the same norm as the handle-based batched
evaluation (adm_eval_batch) within the tolerances of the other GPU tests, on
two calls in a row through the C ABI.

The file name sorts last so that a run stopping at its first failure has run
every other test before this one."""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

TOL = {adm.FP64: 1e-12, adm.FP32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("prec", [adm.FP64, adm.FP32])
def test_noalloc_norm_matches_batched_gradient_norm(prec):
    sh = synth.icosphere_shell(6)
    dt = torch.float64 if prec == adm.FP64 else torch.float32
    m = adm.Mesh(sh.rest, sh.faces, 3)
    _, nV, nnzb, _, _ = m.pattern(adm.SHELL)
    x = torch.from_numpy(sh.x).to(dt).cuda()
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    gn = torch.zeros(1, dtype=torch.float64, device="cuda")
    g = torch.zeros(nV * 3, dtype=dt, device="cuda")
    H = torch.zeros(nnzb * 9, dtype=dt, device="cuda")
    m.eval_batch(adm.SHELL, prec, x, e, gn, g, H)
    torch.cuda.synchronize()
    ref = gn.item()
    assert ref > 0
    L = adm.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = [torch.full((1,), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free = []
    for out in outs:   # two calls in a row share the static scratch
        s = L.adm_grad_norm_noalloc(C.c_void_p(g.data_ptr()), g.numel(), prec, C.c_void_p(out.data_ptr()),
                                    stream)
        assert s == 0, adm.strerror(s)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        assert abs(out.item() - ref) <= TOL[prec] * ref
    # the second call finds its scratch set up by the first and takes no
    # device memory (the first may load the library's module on this device)
    assert free[1] == free[0]
    # the norm itself, checked on the host
    assert abs(ref - np.linalg.norm(g.cpu().double().numpy())) <= TOL[prec] * ref
    m.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = adm.lib()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    too_many = 4096 * 8192 + 1
    s = L.adm_grad_norm_noalloc(C.c_void_p(v.data_ptr()), too_many, adm.FP32, C.c_void_p(out.data_ptr()), None)
    assert s == -1                                                  # ADM_ERR_ARG, nothing launched
    assert L.adm_grad_norm_noalloc(None, 16, adm.FP32, C.c_void_p(out.data_ptr()), None) == -1
    s = L.adm_grad_norm_noalloc(C.c_void_p(v.data_ptr()), 0, adm.FP32, C.c_void_p(out.data_ptr()), None)
    assert s == 0
    torch.cuda.synchronize()
    assert out.item() == 0.0
