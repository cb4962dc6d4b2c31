"""Pins of the oracle's vertex-vertex barrier (the contact term of
Sec. 7.7) and of the pattern extension of Alg. 1:

* gradient and Hessian are the derivatives of the energy (Richardson
  central differences), inside the activation distance;
* the energy is zero at and beyond the activation distance and its
  value and first derivative vanish as d -> dhat from below (the barrier
  switches on continuously);
* at s = d / dhat = 1/2 the energy is kappa/2 dhat A_c (-1/2) ln(1/2) h^2,
  the printed formula evaluated by hand;
* the extended pattern is the union of the mesh pattern and the pairs'
  blocks, original columns first, each block once."""
import numpy as np

import oracle

K, DH, AC, HH = 1.0e4, 0.1, 0.02, 0.05


def test_barrier_derivatives():
    rng = np.random.default_rng(1)
    for _ in range(5):
        xi = rng.normal(size=3)
        xj = xi + 0.03 * rng.normal(size=3) + 0.02
        x = np.concatenate([xi, xj])
        f, g, H = oracle.contact_vv(xi, xj, K, DH, AC, HH)
        assert f > 0

        def fun(y):
            return oracle.contact_vv(y[:3], y[3:], K, DH, AC, HH)[0]

        def grad(y):
            return oracle.contact_vv(y[:3], y[3:], K, DH, AC, HH)[1]

        h = 1e-6
        for k in range(6):
            e = np.zeros(6)
            e[k] = 1.0
            d = lambda t: (fun(x + t * e) - fun(x - t * e)) / (2 * t)  # noqa: E731
            assert abs((4 * d(h / 2) - d(h)) / 3 - g[k]) <= 1e-6 * np.abs(g).max()
            dg = lambda t: (grad(x + t * e) - grad(x - t * e)) / (2 * t)  # noqa: E731
            assert np.abs((4 * dg(h / 2) - dg(h)) / 3 - H[:, k]).max() <= 1e-5 * np.abs(H).max()
        assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_barrier_switches_on_continuously():
    xi = np.zeros(3)
    for d in (DH, 1.5 * DH):
        f, g, H = oracle.contact_vv(xi, np.array([d, 0, 0]), K, DH, AC, HH)
        assert f == 0 and not g.any() and not H.any()
    f, g, _ = oracle.contact_vv(xi, np.array([DH * (1 - 1e-6), 0, 0]), K, DH, AC, HH)
    assert 0 < f < 1e-9 and np.abs(g).max() < 1e-4


def test_barrier_value_at_half():
    f, _, _ = oracle.contact_vv(np.zeros(3), np.array([0, 0.5 * DH, 0]), K, DH, AC, HH)
    want = 0.5 * K * DH * AC * (-0.5) * np.log(0.5) * HH * HH
    assert abs(f - want) <= 1e-14 * want


def test_extended_pattern_union():
    rp = np.array([0, 2, 4, 6, 7])
    col = np.array([0, 1, 0, 1, 2, 3, 3])      # rows: {0,1}, {0,1}, {2,3}, {3}
    pairs = np.array([[0, 3], [1, 2], [0, 1], [3, 0]])
    erp, ecol = oracle.extended_pattern(rp, col, pairs)
    rows = [list(ecol[erp[r]:erp[r + 1]]) for r in range(4)]
    assert rows == [[0, 1, 3], [0, 1, 2], [2, 3, 1], [3, 0]]
