"""Pins of the oracle's vertex-face contact (Sec. 7.7):

* the region-wise distance equals the brute-force minimum of |p - x| over
  a fine sampling of the triangle (so the region test and every region's
  formula are right);
* gradient and Hessian of the barrier are the derivatives of its energy
  (Richardson central differences), in each kind of region;
* the energy is invariant under translation, and zero beyond dhat."""
import numpy as np
import pytest

import oracle

K, DH, AC, HH = 2.0e3, 0.15, 0.3, 0.1
A = np.array([0.0, 0.0, 0.0])
B = np.array([1.0, 0.1, 0.0])
C = np.array([0.2, 0.9, 0.05])
POINTS = {  # one point per kind of closest region
    "face": np.array([0.4, 0.35, 0.08]),
    "vertex_a": np.array([-0.06, -0.05, 0.03]),
    "vertex_b": np.array([1.05, 0.05, -0.04]),
    "edge_ab": np.array([0.5, -0.03, 0.04]),
    "edge_bc": np.array([0.68, 0.6, 0.02]),
    "edge_ca": np.array([0.02, 0.5, 0.05]),
}


def brute_distance(p, a, b, c, n=400):
    u = np.linspace(0.0, 1.0, n + 1)
    U, W = np.meshgrid(u, u)
    keep = U + W <= 1.0
    X = a + U[keep, None] * (b - a) + W[keep, None] * (c - a)
    return np.linalg.norm(X - p, axis=1).min()


@pytest.mark.parametrize("name", list(POINTS))
def test_distance_is_minimum(name):
    p = POINTS[name]
    d = oracle.vf_distance(p, A, B, C)
    assert abs(d - brute_distance(p, A, B, C)) <= 5e-3 * max(d, 1e-3)  # sampling step 1/400


@pytest.mark.parametrize("name", list(POINTS))
def test_barrier_derivatives(name):
    X = np.concatenate([POINTS[name], A, B, C])
    f, g, H = oracle.contact_vf(X[:3], X[3:6], X[6:9], X[9:], K, DH, AC, HH)
    assert f > 0

    def fun(Y):
        return oracle.contact_vf(Y[:3], Y[3:6], Y[6:9], Y[9:], K, DH, AC, HH)

    rng = np.random.default_rng(1)
    v = rng.normal(size=12)
    h = 1e-6
    d = lambda k, t: (fun(X + t * v)[k] - fun(X - t * v)[k]) / (2 * t)  # noqa: E731
    assert abs((4 * d(0, h / 2) - d(0, h)) / 3 - g @ v) <= 1e-6 * np.abs(g).max() * np.abs(v).sum()
    fd = (4 * d(1, h / 2) - d(1, h)) / 3
    assert np.abs(fd - H @ v).max() <= 1e-5 * np.abs(H).max() * np.abs(v).sum()
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


def test_translation_and_cutoff():
    X = np.concatenate([POINTS["face"], A, B, C])
    f, g, _ = oracle.contact_vf(X[:3], X[3:6], X[6:9], X[9:], K, DH, AC, HH)
    t = np.array([0.3, -1.2, 2.0])
    f2, _, _ = oracle.contact_vf(X[:3] + t, X[3:6] + t, X[6:9] + t, X[9:] + t, K, DH, AC, HH)
    assert abs(f2 - f) <= 1e-12 * f
    assert np.abs(g.reshape(4, 3).sum(0)).max() <= 1e-10 * np.abs(g).max()   # forces balance
    far = np.array([0.3, 0.3, 0.5])
    assert oracle.contact_vf(far, A, B, C, K, DH, AC, HH)[0] == 0.0


def test_vertex_region_matches_vertex_vertex():
    """In a vertex region the vertex-face barrier is the vertex-vertex barrier
    of (p, that vertex), whose derivatives are written in closed form."""
    p = POINTS["vertex_b"]
    assert oracle.closest_region(p, A, B, C) == ("v", 1)
    f, g, H = oracle.contact_vf(p, A, B, C, K, DH, AC, HH)
    f2, g2, H2 = oracle.contact_vv(p, B, K, DH, AC, HH)
    assert abs(f - f2) <= 1e-14 * f2
    idx = [0, 1, 2, 6, 7, 8]                               # p and b in (p, a, b, c)
    assert np.abs(g[idx] - g2).max() <= 1e-12 * np.abs(g2).max()
    assert np.abs(H[np.ix_(idx, idx)] - H2).max() <= 1e-12 * np.abs(H2).max()
    rest = [3, 4, 5, 9, 10, 11]
    assert np.abs(g[rest]).max() == 0.0 and np.abs(H[rest]).max() == 0.0


def test_extended_pattern_with_quads():
    """Blocks of vertex-face elements: every pair of the element's four
    vertices, once, on top of the mesh pattern; the assembled blocks stay
    inside that pattern."""
    V, F = oracle_icosphere()
    nV = len(V)
    rp, col = oracle.pattern(nV, F)
    quads = np.array([[0, *F[20]], [0, *F[21]], [5, *F[20]]])
    quads = quads[[0 not in F[20], 0 not in F[21], 5 not in F[20]]]
    pairs = np.array([[0, int(F[20][0])]])
    erp, ecol = oracle.extended_pattern(rp, col, pairs, quads)
    dense = np.zeros((nV, nV), dtype=bool)
    for r in range(nV):
        dense[r, col[rp[r]:rp[r + 1]]] = True
    for t in np.concatenate([quads, np.tile(pairs, (1, 2))]):
        for i in t:
            for j in t:
                dense[i, j] = True
    for r in range(nV):
        got = ecol[erp[r]:erp[r + 1]]
        assert len(set(got.tolist())) == len(got)
        assert set(got.tolist()) == set(np.flatnonzero(dense[r]).tolist())
        assert list(got[:rp[r + 1] - rp[r]]) == list(col[rp[r]:rp[r + 1]])
    x = V + 0.0
    base = {"energy": 0.0, "grad": np.zeros((nV, 3)), "vals": np.zeros((len(col), 3, 3))}
    ref = oracle.add_interactions(base, x, pairs, K, 10.0, AC, HH, rp, col, quads)
    keys = {(r, int(c)) for r in range(nV) for c in ecol[erp[r]:erp[r + 1]]}
    assert set(ref["blocks"]) <= keys


def oracle_icosphere():
    import synth
    return synth.icosphere(1)
