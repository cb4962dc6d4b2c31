"""Pins of the oracle's learned-membrane functions: the network on
hyper-duals against finite differences and a plain numpy forward pass, the
Neo-Hookean targets against their closed form, and the hand-written Sobolev
loss backpropagation against Richardson finite differences."""
import numpy as np

import oracle
import synth

E, NU = 1.0e5, 0.3
MU = E / (2 * (1 + NU))
LAM = E * NU / (1 - NU * NU)


def rand_theta(rng, scale=0.5):
    th = rng.normal(scale=scale, size=oracle.MLP_NPARAM)
    return th


def norm_of(I, psi):
    return np.concatenate([I.mean(0), I.std(0), [psi.mean(), psi.std()]])


def numpy_forward(th, norm, I):
    W1 = th[:192].reshape(64, 3)
    b1 = th[192:256]
    W2 = th[256:4352].reshape(64, 64)
    b2 = th[4352:4416]
    w3 = th[4416:4480]
    b3 = th[4480]
    silu = lambda z: z / (1 + np.exp(-z))  # noqa: E731
    u = (I - norm[:3]) / norm[3:6]
    a1 = silu(u @ W1.T + b1)
    a2 = silu(a1 @ W2.T + b2)
    return (a2 @ w3 + b3) * norm[7] + norm[6]


def test_invariants_closed_form():
    F = synth.membrane_samples(50, seed=9)
    I = oracle.invariants_from_F(F)
    C = np.einsum("nia,nib->nab", F, F)
    assert np.allclose(I[:, 0], np.trace(C, axis1=1, axis2=2) + 1)
    assert np.allclose(I[:, 2], np.linalg.det(C))
    assert np.allclose(I[:, 1], np.linalg.det(C) + np.trace(C, axis1=1, axis2=2))
    s = np.linalg.svd(F, compute_uv=False)                   # principal stretches
    assert np.allclose(I[:, 2], (s[:, 0] * s[:, 1]) ** 2)


def test_nh_targets_closed_form():
    I = oracle.invariants_from_F(synth.membrane_samples(20, seed=3))
    psi, g = oracle.nh_targets(I)
    lnJ = 0.5 * np.log(I[:, 2])
    assert np.allclose(psi, 0.5 * MU * (I[:, 0] - 3) - MU * lnJ + 0.5 * LAM * lnJ ** 2)
    assert np.allclose(g[:, 0], 0.5 * MU) and np.allclose(g[:, 1], 0.0)
    assert np.allclose(g[:, 2], (-MU + LAM * lnJ) / (2 * I[:, 2]))


def test_mlp_eval_value_and_derivatives():
    rng = np.random.default_rng(0)
    I = oracle.invariants_from_F(synth.membrane_samples(8, seed=4))
    th = rand_theta(rng)
    norm = np.array([3.0, 3.0, 1.0, 0.4, 0.5, 0.3, 0.2, 1.5])
    out = oracle.mlp_eval(th, norm, I)
    assert np.allclose(out[:, 0], numpy_forward(th, norm, I), rtol=1e-13)
    h = 1e-5
    for k in range(3):
        d = np.zeros(3)
        d[k] = h
        fd = (numpy_forward(th, norm, I + d) - numpy_forward(th, norm, I - d)) / (2 * h)
        assert np.allclose(out[:, 1 + k], fd, rtol=1e-6, atol=1e-9)
        gp = oracle.mlp_eval(th, norm, I + d)[:, 1:4]
        gm = oracle.mlp_eval(th, norm, I - d)[:, 1:4]
        col = (gp - gm) / (2 * h)
        hidx = {0: (4, 5, 7), 1: (5, 6, 8), 2: (7, 8, 9)}[k]   # packed upper Hessian
        for kk in range(3):
            assert np.allclose(out[:, hidx[kk]], col[:, kk], rtol=1e-5, atol=1e-8)


def test_mlp_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    F = synth.membrane_samples(40, seed=6)
    I = oracle.invariants_from_F(F)
    psi, g = oracle.nh_targets(I)
    norm = norm_of(I, psi)
    th = rand_theta(rng, 0.3)
    L, grad = oracle.mlp_loss(th, norm, I, psi, g, beta=0.7)
    assert L > 0
    idx = np.concatenate([rng.choice(192, 4, replace=False), 192 + rng.choice(64, 3, replace=False),
                          256 + rng.choice(4096, 8, replace=False), 4352 + rng.choice(64, 3, replace=False),
                          4416 + rng.choice(64, 3, replace=False), [4480]])
    for i in idx:
        def f(step):
            t = th.copy()
            t[i] += step
            return oracle.mlp_loss(t, norm, I, psi, g, beta=0.7, grad=False)
        h = 1e-4
        d = lambda s: (f(s) - f(-s)) / (2 * s)  # noqa: E731
        fd = (4 * d(h / 2) - d(h)) / 3
        assert abs(grad[i] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, grad[i], fd)


def test_mlp_mesh_energy_matches_network_on_invariants():
    """The MLP membrane mesh energy (hyper-duals over the 9 DOFs) equals
    t A psi(I) with psi from the invariant-space network, and its gradient
    and Hessian match finite differences."""
    rng = np.random.default_rng(2)
    V = np.array([[0.1, -0.2, 0.3], [1.2, 0.1, 0.2], [0.3, 0.9, -0.1]])
    Dinv, area = oracle.tri_rest(V, np.array([[0, 1, 2]], dtype=np.int32))
    th = rand_theta(rng, 0.3)
    norm = np.array([3.0, 3.0, 1.0, 0.4, 0.5, 0.3, 1.0, 2.0])
    oracle.mlp_set(th, norm)
    x = V.ravel() + rng.normal(scale=0.05, size=9)
    out = oracle.local(oracle.MLP, x, Dinv=Dinv[0], area=area[0], params=[1e5, 0.3, 2e-3])
    xe = x.reshape(3, 3)
    Ds = np.stack([xe[1] - xe[0], xe[2] - xe[0]], 1)
    Fd = Ds @ Dinv[0].reshape(2, 2)
    I = oracle.invariants_from_F(Fd[None])
    assert np.isclose(out["f"], 2e-3 * area[0] * oracle.mlp_eval(th, norm, I)[0, 0], rtol=1e-13)
    f = lambda y: oracle.local(oracle.MLP, y, Dinv=Dinv[0], area=area[0], params=[1e5, 0.3, 2e-3])["f"]  # noqa: E731
    g = np.array([(f(x + h) - f(x - h)) / 2e-6 for h in np.eye(9) * 1e-6])
    assert np.allclose(out["g"], g, rtol=1e-6, atol=1e-12)
    assert np.allclose(out["H"], out["H"].T, atol=1e-12 * np.abs(out["H"]).max())
