"""Seeded synthetic inputs shared by the oracle, the tests and the bench.

This module only *constructs inputs*: meshes (vertex positions and triangle
index lists), deformed positions and deformation samples.  It holds none of
the differentiated method's arithmetic (no energies, no rest-frame data, no
connectivity beyond the triangle lists themselves), so the CPU oracle and the
CUDA path can both consume it without sharing any of the computation they are
compared on.

Every generator takes an explicit integer seed and draws from
``numpy.random.default_rng(seed)`` (PCG64); the same seed gives bit-identical
arrays on x86_64 and aarch64.

Workloads (sizes follow the paper's application scales, Sec. 7; they stand
in for the paper's meshes, which are not available):

* ``grid_uv``        -- 33x33 regular grid of the unit square, 2,048 triangles,
                        UV = rest + N(0, 0.01^2)  (symmetric Dirichlet, Sec. 7.2)
* ``icosphere``      -- subdivided icosahedron on the unit sphere
                        (level 7: 163,842 vertices, 327,680 triangles)
* ``noisy_disk``     -- jittered grid disk of ~1M triangles with a paraboloid
                        rest cap (least-squares Jacobian workload)
* ``shell_batch``    -- hundreds of rigidly placed, perturbed icospheres
                        (the paper's ~700-body, 2.1M-vertex shell scene, Sec. 7.7)
* ``membrane_samples`` -- deformation gradients with principal stretches in
                        [0.7, 1.4] for the learned membrane energy
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh",
    "grid_uv",
    "icosphere",
    "perturb",
    "noisy_disk",
    "cloth_grid",
    "shell_batch",
    "shell_batch_levels",
    "membrane_samples",
    "stretched_batch",
    "tiny_meshes",
]


@dataclass
class Mesh:
    """A (possibly batched) triangle mesh.

    rest   : (nV, 3) float64 rest positions
    faces  : (nT, 3) int32 vertex indices, counter-clockwise seen from outside
    x      : (nV, d) float64 current positions (d = 3) or UV coordinates (d = 2)
    v_off  : (n_mesh + 1,) int64 vertex offsets of the meshes in a batch
    f_off  : (n_mesh + 1,) int64 face offsets of the meshes in a batch
    """

    rest: np.ndarray
    faces: np.ndarray
    x: np.ndarray
    v_off: np.ndarray = field(default=None)
    f_off: np.ndarray = field(default=None)
    name: str = ""
    xhat: np.ndarray = field(default=None)  # (nV, 3) inertial target of a time step (cloth), or None

    def __post_init__(self):
        if self.v_off is None:
            self.v_off = np.array([0, self.rest.shape[0]], dtype=np.int64)
        if self.f_off is None:
            self.f_off = np.array([0, self.faces.shape[0]], dtype=np.int64)

    @property
    def nV(self) -> int:
        return int(self.rest.shape[0])

    @property
    def nT(self) -> int:
        return int(self.faces.shape[0])

    @property
    def n_mesh(self) -> int:
        return int(self.v_off.shape[0] - 1)


# --------------------------------------------------------------------------
# 2D grid (symmetric Dirichlet parameterisation workload)
# --------------------------------------------------------------------------
def grid_uv(n: int = 33, sigma: float = 0.01, seed: int = 1, relative: bool = True) -> Mesh:
    """n x n vertex grid on [0,1]^2; every quad split along its
    (i,j)->(i+1,j+1) diagonal, both triangles counter-clockwise.
    Rest shape is the grid at z = 0; x is the UV map rest_xy + N(0, s^2) on
    every coordinate (boundary included), with s = sigma * h (h = 1/(n-1),
    the grid spacing) when ``relative`` and s = sigma otherwise.  The relative
    reading keeps the map fold-free; sigma = 0.01 in absolute units folds
    about 5% of the triangles of the 33 x 33 grid."""
    s = np.linspace(0.0, 1.0, n)
    gx, gy = np.meshgrid(s, s, indexing="xy")          # gy varies with row j
    rest = np.zeros((n * n, 3))
    rest[:, 0] = gx.ravel()
    rest[:, 1] = gy.ravel()
    faces = []
    for j in range(n - 1):
        for i in range(n - 1):
            v00 = j * n + i
            v10 = v00 + 1
            v01 = v00 + n
            v11 = v01 + 1
            faces.append((v00, v10, v11))
            faces.append((v00, v11, v01))
    faces = np.asarray(faces, dtype=np.int32)
    rng = np.random.default_rng(seed)
    s_abs = sigma / (n - 1) if relative else sigma
    x = rest[:, :2] + rng.normal(0.0, s_abs, size=(n * n, 2))
    return Mesh(rest=rest, faces=faces, x=x, name=f"grid{n}")


# --------------------------------------------------------------------------
# Cloth grid (mass-spring workload)
# --------------------------------------------------------------------------
def cloth_grid(n: int = 100, sigma: float = 0.05, seed: int = 6) -> Mesh:
    """n x n vertex cloth on [0,1]^2 at z = 0, triangulated as grid_uv.
    x = rest + N(0, s^2) on all three coordinates and the inertial target
    xhat (standing for x^n + h v^n of an implicit Euler step) = rest +
    N(0, s^2) independently, with s = sigma / (n - 1), a fraction of the
    grid spacing."""
    s = np.linspace(0.0, 1.0, n)
    gx, gy = np.meshgrid(s, s, indexing="xy")
    rest = np.zeros((n * n, 3))
    rest[:, 0] = gx.ravel()
    rest[:, 1] = gy.ravel()
    j, i = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    v00 = (j * n + i).ravel()
    v10, v01 = v00 + 1, v00 + n
    v11 = v01 + 1
    faces = np.empty((2 * v00.size, 3), dtype=np.int32)
    faces[0::2] = np.stack([v00, v10, v11], axis=1)
    faces[1::2] = np.stack([v00, v11, v01], axis=1)
    rng = np.random.default_rng(seed)
    sd = sigma / (n - 1)
    x = rest + rng.normal(0.0, sd, size=rest.shape)
    xhat = rest + rng.normal(0.0, sd, size=rest.shape)
    return Mesh(rest=rest, faces=faces, x=x, name=f"cloth{n}", xhat=xhat)


# --------------------------------------------------------------------------
# Icosphere
# --------------------------------------------------------------------------
def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    return v, f


@functools.lru_cache(maxsize=16)
def _icosphere_cached(level: int):
    v, f = _icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        # midpoints of the three edges of every face, deduplicated by the
        # unordered endpoint pair
        ends = np.stack([np.stack([a, b], 1), np.stack([b, c], 1), np.stack([c, a], 1)], 1)
        lo = ends.min(axis=2)
        hi = ends.max(axis=2)
        key = (lo * nv + hi).ravel()
        uniq, inv = np.unique(key, return_inverse=True)
        ulo = uniq // nv
        uhi = uniq % nv
        mid = v[ulo] + v[uhi]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid], 0)
        m = (inv.reshape(-1, 3) + nv).astype(np.int64)
        mab, mbc, mca = m[:, 0], m[:, 1], m[:, 2]
        f = np.concatenate(
            [
                np.stack([a, mab, mca], 1),
                np.stack([b, mbc, mab], 1),
                np.stack([c, mca, mbc], 1),
                np.stack([mab, mbc, mca], 1),
            ],
            0,
        )
    v.setflags(write=False)
    f32 = f.astype(np.int32)
    f32.setflags(write=False)
    return v, f32


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit-sphere icosphere: icosahedron, ``level`` midpoint subdivisions,
    every new vertex projected to the sphere; faces outward, counter-clockwise.
    Returns copies of (vertices (nV,3) float64, faces (nT,3) int32)."""
    v, f = _icosphere_cached(int(level))
    return v.copy(), f.copy()


def perturb(rest: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """rest + N(0, sigma^2) on every coordinate."""
    rng = np.random.default_rng(seed)
    return rest + rng.normal(0.0, sigma, size=rest.shape)


def icosphere_shell(level: int = 7, sigma: float = 1e-3, seed: int = 2) -> Mesh:
    """Single elastic-shell workload: rest = icosphere, x = rest + N(0, sigma^2)."""
    v, f = icosphere(level)
    return Mesh(rest=v, faces=f, x=perturb(v, sigma, seed), name=f"icosphere{level}")


# --------------------------------------------------------------------------
# Noisy-grid disk (least-squares UV workload)
# --------------------------------------------------------------------------
def noisy_disk(n_tri_target: float = 1.0e6, jitter: float = 0.2, cap: float = 0.3,
               seed: int = 3) -> Mesh:
    """Square grid of spacing h = sqrt(2*pi/n_tri_target) over [-1,1]^2; keep
    every quad whose four corners lie strictly inside the unit disk and split
    it as in ``grid_uv``.  Vertices all of whose four surrounding quads are
    kept (interior vertices) are jittered by U[-jitter*h, jitter*h]^2.
    Rest shape: (x, y, cap*(x^2+y^2)) of the jittered points; x (the initial
    UV map) is the jittered (x, y)."""
    h = float(np.sqrt(2.0 * np.pi / n_tri_target))
    m = int(np.floor(1.0 / h))
    coords = np.arange(-m, m + 1) * h                    # 2m+1 samples per axis
    n = coords.shape[0]
    gx, gy = np.meshgrid(coords, coords, indexing="xy")
    inside = (gx * gx + gy * gy) < 1.0
    q = inside[:-1, :-1] & inside[:-1, 1:] & inside[1:, :-1] & inside[1:, 1:]  # quad (j,i)
    jj, ii = np.nonzero(q)
    v00 = jj * n + ii
    v10 = v00 + 1
    v01 = v00 + n
    v11 = v01 + 1
    faces = np.empty((2 * jj.shape[0], 3), dtype=np.int64)
    faces[0::2] = np.stack([v00, v10, v11], 1)
    faces[1::2] = np.stack([v00, v11, v01], 1)
    used = np.zeros(n * n, dtype=bool)
    used[faces.ravel()] = True
    remap = -np.ones(n * n, dtype=np.int64)
    remap[used] = np.arange(int(used.sum()))
    faces = remap[faces].astype(np.int32)
    # interior = all four quads around the grid vertex are kept
    qp = np.zeros((n + 1, n + 1), dtype=bool)
    qp[1:n, 1:n] = q
    interior_grid = qp[:-1, :-1] & qp[:-1, 1:] & qp[1:, :-1] & qp[1:, 1:]
    interior = interior_grid.ravel()[used]
    xy = np.stack([gx.ravel()[used], gy.ravel()[used]], 1)
    rng = np.random.default_rng(seed)
    jit = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    xy = xy + jit * interior[:, None]
    rest = np.concatenate([xy, cap * (xy * xy).sum(1, keepdims=True)], 1)
    return Mesh(rest=rest, faces=faces, x=xy.copy(), name="noisy_disk")


# --------------------------------------------------------------------------
# Batched shells
# --------------------------------------------------------------------------
def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def shell_batch_levels(kind: str = "paper", n_mesh: int = 700, seed: int = 4) -> np.ndarray:
    """Subdivision level of every mesh of the batched-shell workload.

    kind="paper":   700 meshes whose levels are a seeded shuffle of the fixed
                    multiset {4: 668, 5: 28, 6: 4} -> 2,162,040 vertices,
                    4,321,280 triangles (the paper's ~700 bodies / 2.1M
                    vertices scene, Sec. 7.7).
    kind="uniform": every level drawn uniformly from {4, 5, 6} (about 12.5M
                    vertices for 700 meshes).
    kind="level4":  all level 4 (2,562 vertices each)."""
    rng = np.random.default_rng(seed)
    if kind == "paper":
        if n_mesh != 700:
            raise ValueError("the paper-scale mix is defined for 700 meshes")
        lv = np.array([4] * 668 + [5] * 28 + [6] * 4, dtype=np.int64)
        rng.shuffle(lv)
        return lv
    if kind == "uniform":
        return rng.integers(4, 7, size=n_mesh).astype(np.int64)
    if kind == "level4":
        return np.full(n_mesh, 4, dtype=np.int64)
    raise ValueError(kind)


def shell_batch(levels, sigma: float = 1e-3, spacing: float = 3.0, seed: int = 4) -> Mesh:
    """Batch of icospheres: mesh m gets level levels[m], a seeded uniform random
    rotation, a translation to lattice cell (m%10, (m//10)%10, m//100)*spacing,
    and x = rest + N(0, sigma^2) per coordinate."""
    levels = np.asarray(levels, dtype=np.int64)
    rng = np.random.default_rng(seed)
    rests, faces, v_off, f_off = [], [], [0], [0]
    for m, lv in enumerate(levels):
        v, f = _icosphere_cached(int(lv))
        R = _random_rotation(rng)
        cell = np.array([m % 10, (m // 10) % 10, m // 100], dtype=np.float64) * spacing
        rests.append(v @ R.T + cell)
        faces.append(f.astype(np.int64) + v_off[-1])
        v_off.append(v_off[-1] + v.shape[0])
        f_off.append(f_off[-1] + f.shape[0])
    rest = np.concatenate(rests, 0)
    x = rest + rng.normal(0.0, sigma, size=rest.shape)
    return Mesh(
        rest=rest,
        faces=np.concatenate(faces, 0).astype(np.int32),
        x=x,
        v_off=np.asarray(v_off, dtype=np.int64),
        f_off=np.asarray(f_off, dtype=np.int64),
        name=f"shell_batch{len(levels)}",
    )


def stretched_batch(mesh: Mesh, lo: float = 0.7, hi: float = 1.4, seed: int = 9) -> np.ndarray:
    """Deformed positions of a shell batch inside the learned membrane's
    training range: mesh m is mapped about its rest centroid c_m by
    x = c_m + R_m diag(s_1, s_2, s_3) R_m^T (X - c_m), s_k ~ U[lo, hi] and
    R_m a uniform random rotation, so every triangle's in-plane principal
    stretches lie in [lo, hi]."""
    rng = np.random.default_rng(seed)
    x = np.empty_like(mesh.rest)
    for m in range(len(mesh.v_off) - 1):
        a, b = mesh.v_off[m], mesh.v_off[m + 1]
        R = _random_rotation(rng)
        A = R @ np.diag(rng.uniform(lo, hi, size=3)) @ R.T
        c = mesh.rest[a:b].mean(0)
        x[a:b] = c + (mesh.rest[a:b] - c) @ A.T
    return x


# --------------------------------------------------------------------------
# Learned membrane: deformation samples
# --------------------------------------------------------------------------
def membrane_samples(n: int, lo: float = 0.7, hi: float = 1.4, seed: int = 5) -> np.ndarray:
    """n membrane deformation gradients F (n, 3, 2) = U diag(l1, l2) V^T with
    principal stretches l1, l2 ~ U[lo, hi], V a uniform in-plane rotation and
    U = the first two columns of a uniform random 3D rotation."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(lo, hi, size=(n, 2))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    c, s = np.cos(phi), np.sin(phi)
    V = np.stack([np.stack([c, -s], -1), np.stack([s, c], -1)], -2)       # (n,2,2)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    U = np.stack(
        [
            np.stack([1 - 2 * (y * y + z * z), 2 * (x * y + z * w), 2 * (x * z - y * w)], -1),
            np.stack([2 * (x * y - z * w), 1 - 2 * (x * x + z * z), 2 * (y * z + x * w)], -1),
        ],
        -1,
    )                                                                      # (n,3,2)
    return np.einsum("nij,nj,nkj->nik", U, lam, V)


# --------------------------------------------------------------------------
# Tiny meshes for brute-force checks
# --------------------------------------------------------------------------
def tiny_meshes() -> dict[str, tuple[np.ndarray, np.ndarray]]:
    """Small closed and open meshes (rest positions, faces)."""
    out = {}
    out["two_triangles"] = (
        np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], dtype=np.float64),
        np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32),
    )
    tv = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64)
    out["tetrahedron"] = (tv, np.array([[0, 1, 2], [0, 3, 1], [0, 2, 3], [1, 3, 2]], dtype=np.int32))
    for lv in (0, 1, 2):
        out[f"icosphere{lv}"] = icosphere(lv)
    g = grid_uv(3, 0.0, 0)
    out["grid3"] = (g.rest, g.faces)
    return out
