"""Learned membrane energy on the GPU: the BF16 tensor-core network against
the FP64 oracle (forward mode through the network, the Sobolev-loss
gradient, the analytic Neo-Hookean targets), training on oracle-generated
samples, what the trained network gains over the method without it, and the
ADM_MLP_MEMBRANE mesh energy against the oracle's hyper-dual evaluation of
the same network.

The network contracts BF16-rounded activations on the tensor cores (FP32
accumulation), so agreement with the FP64 oracle is at the BF16 level:
relative errors of a few 1e-3, bounded here by 3e-2."""
import numpy as np
import pytest

import oracle
import synth
from util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import __graft_entry__  # noqa: E402
import paper_2509_00406_gb300 as adm  # noqa: E402

E, NU = 1.0e5, 0.3
MU = E / (2 * (1 + NU))
LAM = E * NU / (1 - NU * NU)


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def bf16(a):
    return torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()


def init_theta(rng):
    th = np.zeros(adm.MLP_NPARAM)
    th[:192] = rng.normal(scale=0.6, size=192)
    th[256:4352] = rng.normal(scale=1 / 8, size=4096)
    th[4416:4480] = rng.normal(scale=1 / 8, size=64)
    return th


def samples(n, seed):
    F = synth.membrane_samples(n, seed=seed)
    I = oracle.invariants_from_F(F)
    psi, g = oracle.nh_targets(I)
    return F, I, psi, g


def norm_of(I, psi):
    return np.concatenate([I.mean(0), I.std(0), [psi.mean(), psi.std()]])


def cuda32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_mlp_eval_matches_oracle():
    rng = np.random.default_rng(0)
    _, I, psi, _ = samples(1003, 11)  # ragged: not a multiple of the 8 samples of a warp
    th = init_theta(rng)
    norm = norm_of(I, psi)
    out = torch.zeros((I.shape[0], 10), dtype=torch.float32, device="cuda")
    adm.MLP.eval(cuda32(th), cuda32(norm), cuda32(I), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    ref = oracle.mlp_eval(bf16(th), norm, I.astype(np.float32).astype(np.float64))
    assert rel(got[:, 0], ref[:, 0]) < 3e-2
    assert rel(got[:, 1:4], ref[:, 1:4]) < 3e-2
    assert rel(got[:, 4:], ref[:, 4:]) < 3e-2


def test_mlp_nh_targets_match_oracle():
    F, I, psi, g = samples(500, 12)
    Fd = cuda32(F.reshape(-1, 6))
    Ig = torch.zeros((500, 3), device="cuda")
    pg = torch.zeros(500, device="cuda")
    gg = torch.zeros((500, 3), device="cuda")
    adm.MLP.nh_targets(Fd, E, NU, Ig, pg, gg)
    torch.cuda.synchronize()
    I32 = oracle.invariants_from_F(F.astype(np.float32).astype(np.float64))
    p32, g32 = oracle.nh_targets(I32)
    assert rel(Ig.cpu().numpy(), I32) < 1e-6
    assert rel(pg.cpu().numpy(), p32) < 1e-5
    assert rel(gg.cpu().numpy(), g32) < 1e-5


def test_mlp_loss_gradient_matches_oracle():
    rng = np.random.default_rng(3)
    _, I, psi, g = samples(2000, 13)
    th = init_theta(rng)
    norm = norm_of(I, psi)
    ws = torch.zeros(adm.MLP.workspace_size() // 4 + 1, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros(adm.MLP_NPARAM, dtype=torch.float32, device="cuda")
    adm.MLP.loss_grad(cuda32(th), cuda32(norm), cuda32(I), cuda32(psi), cuda32(g), 0.5, loss, grad, ws)
    torch.cuda.synchronize()
    Lref, gref = oracle.mlp_loss(bf16(th), norm, I.astype(np.float32).astype(np.float64),
                                 psi.astype(np.float32).astype(np.float64),
                                 g.astype(np.float32).astype(np.float64), beta=0.5)
    assert abs(loss.item() - Lref) <= 3e-2 * Lref
    gg = grad.cpu().numpy()
    for lo, hi in ((0, 192), (192, 256), (256, 4352), (4352, 4416), (4416, 4480), (4480, 4481)):
        assert rel(gg[lo:hi], gref[lo:hi]) < 3e-2, (lo, hi, rel(gg[lo:hi], gref[lo:hi]))


def train(I, psi, g, norm, steps=600, batch=8192, lr=3e-3, seed=0):
    rng = np.random.default_rng(seed)
    th = cuda32(init_theta(rng))
    m = torch.zeros_like(th)
    v = torch.zeros_like(th)
    nd = cuda32(norm)
    Id, pd, gd = cuda32(I), cuda32(psi), cuda32(g)
    ws = torch.zeros(adm.MLP.workspace_size() // 4 + 1, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    grad = torch.zeros_like(th)
    hist = []
    perm = torch.from_numpy(rng.permutation(I.shape[0])).cuda()
    for step in range(1, steps + 1):
        k = (step - 1) * batch % I.shape[0]
        idx = perm[k:k + batch]
        adm.MLP.loss_grad(th, nd, Id[idx].contiguous(), pd[idx].contiguous(), gd[idx].contiguous(), 1.0, loss,
                          grad, ws)
        adm.MLP.adam(th, m, v, grad, step, lr * (0.1 ** (step / steps)))
        if step % 50 == 1:
            hist.append(loss.item())
    return th, hist


def test_mlp_training_gains_over_stvk():
    """Trained on oracle Neo-Hookean samples, the network's density, gradient
    and Hessian in the invariants are far closer to Neo-Hookean than the
    membrane without it (StVK with the same Lame parameters) on held-out
    stretches in [0.7, 1.4]."""
    _, I, psi, g = samples(65536, 5)
    norm = norm_of(I, psi)
    th, hist = train(I, psi, g, norm)
    assert hist[-1] < 0.05 * hist[0]
    _, It, pt, gt = samples(4000, 77)
    out = torch.zeros((It.shape[0], 10), dtype=torch.float32, device="cuda")
    adm.MLP.eval(th, cuda32(norm), cuda32(It), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    # StVK in the invariants: tr C = I1 - 1, det C = I3
    trC, detC = It[:, 0] - 1, It[:, 2]
    nE2 = 0.25 * (trC ** 2 - 2 * detC - 2 * trC + 2)
    psi_stvk = MU * nE2 + 0.5 * LAM * (0.5 * (trC - 2)) ** 2
    err_mlp = rel(got[:, 0], pt)
    err_stvk = rel(psi_stvk, pt)
    assert err_mlp < 0.05 and err_stvk / err_mlp > 5.0, (err_mlp, err_stvk)
    # gradient in the invariants against Neo-Hookean
    assert rel(got[:, 1:4], gt) < 0.1


def test_mlp_membrane_mesh_matches_oracle():
    rng = np.random.default_rng(4)
    v, f = synth.icosphere(1)
    x = synth.perturb(v, 2e-2, 8)
    _, I, psi, _ = samples(2000, 14)
    th = init_theta(rng)
    norm = norm_of(I, psi)
    m = adm.Mesh(v, f, 3)
    m.set_params(adm.MLP_MEMBRANE, [E, NU, 1e-3])
    m.mlp_attach(cuda32(th), cuda32(norm))
    _, nV, nnzb, rp, col = m.pattern(adm.MLP_MEMBRANE)
    xd = cuda32(x)
    e = torch.zeros(1, dtype=torch.float64, device="cuda")
    gd = torch.zeros(nV * 3, dtype=torch.float32, device="cuda")
    Hd = torch.zeros(nnzb * 9, dtype=torch.float32, device="cuda")
    m.eval(adm.MLP_MEMBRANE, adm.FP32, xd, e, gd, Hd)
    torch.cuda.synchronize()
    assert m.status() == 0
    oracle.mlp_set(bf16(th), norm)
    P = oracle.Problem(v, f, oracle.MLP, 3, params=[E, NU, 1e-3])
    ref = P.assemble(x.astype(np.float32).astype(np.float64))
    assert abs(e.item() - ref["energy"]) <= 3e-2 * abs(ref["energy"])
    assert rel(gd.cpu().numpy().reshape(-1, 3), ref["grad"]) < 3e-2
    assert rel(Hd.cpu().numpy().reshape(-1, 3, 3), ref["vals"]) < 3e-2


@pytest.mark.parametrize("net", [0, 1])
def test_mlp_membrane_batch_both_networks_match_oracle(net):
    """Both network kernels (0: warp-level mma.sync, 1: tcgen05 with TMEM
    accumulators, 128 triangles per MMA tile) on a batch whose 1,680
    triangles span 13 MMA tiles with a ragged last one: each against the
    oracle's network on the same BF16 weights (3e-2), and the tcgen05 one
    against the mma.sync one.  The two round the same FP32 activations to
    BF16 and differ only in the FP32 summation order of the contractions,
    which can move a BF16 rounding of rho by one unit, so they agree to
    about 1e-4; the bound is 2e-3."""
    rng = np.random.default_rng(6)
    b = synth.shell_batch([1, 2, 3], sigma=2e-2, seed=9)
    x = b.x.astype(np.float32)
    _, I, psi, _ = samples(2000, 15)
    th = init_theta(rng)
    norm = norm_of(I, psi)
    m = adm.Mesh(b.rest, b.faces, 3, v_off=b.v_off, f_off=b.f_off)
    m.set_params(adm.MLP_MEMBRANE, [E, NU, 1e-3])
    m.mlp_attach(cuda32(th), cuda32(norm))
    _, nV, nnzb, rp, col = m.pattern(adm.MLP_MEMBRANE)
    rp = rp.cpu().numpy()

    def run(option):
        m.set_option(adm.OPT_MLP_NET, option)
        e = torch.zeros(b.n_mesh, dtype=torch.float64, device="cuda")
        gd = torch.full((nV * 3,), float("nan"), device="cuda")
        Hd = torch.full((nnzb * 9,), float("nan"), device="cuda")
        m.eval_batch(adm.MLP_MEMBRANE, adm.FP32, cuda32(x), e, None, gd, Hd)
        torch.cuda.synchronize()
        assert m.status() == 0
        return e.cpu().numpy(), gd.cpu().numpy().reshape(-1, 3), Hd.cpu().numpy().reshape(-1, 3, 3)

    e, g, H = run(net)
    assert np.isfinite(H).all() and np.isfinite(g).all()
    oracle.mlp_set(bf16(th), norm)
    for k in range(b.n_mesh):
        v0, v1, f0, f1 = b.v_off[k], b.v_off[k + 1], b.f_off[k], b.f_off[k + 1]
        P = oracle.Problem(b.rest[v0:v1], b.faces[f0:f1] - v0, oracle.MLP, 3, params=[E, NU, 1e-3])
        ref = P.assemble(x[v0:v1].astype(np.float64))
        assert abs(e[k] - ref["energy"]) <= 3e-2 * abs(ref["energy"]), (k, e[k], ref["energy"])
        assert rel(g[v0:v1], ref["grad"]) < 3e-2
        assert rel(H[rp[v0]:rp[v1]], ref["vals"]) < 3e-2
    if net == 1:
        e0, g0, H0 = run(0)
        assert rel(e, e0) < 2e-3 and rel(g, g0) < 2e-3 and rel(H, H0) < 2e-3
        # the same network kernel twice: bit-identical
        e1, g1, H1 = run(1)
        assert np.array_equal(e1, e) and np.array_equal(g1, g) and np.array_equal(H1, H)
    m.close()
