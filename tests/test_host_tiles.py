"""Creation-time builders of the staged-gather assembler, run on the host
without a GPU (libadm_host.so is the same mesh.cpp/tiles.cpp code compiled
with the C++ compiler alone).  For every mesh and tile size: every chunk of a
tile is written by exactly one unit role and summed by the segments of its
outputs; every block of the pattern is produced by one tile (a plain store)
or is "shared": the lowest of its tiles stores it, every other one writes a
partial slot of its own (the slots of one output contiguous, in tile order,
listed by the output's fix-up entry, every slot used exactly once); and every
triangle and hinge belongs to exactly one tile."""
import ctypes as C

import numpy as np
import pytest

import synth
from paper_2509_00406_gb300 import _build


@pytest.fixture(scope="module")
def H():
    return C.CDLL(_build.build_host())


def run(L, mesh, with_hinges, tile):
    V = np.ascontiguousarray(mesh.rest, dtype=np.float64)
    F = np.ascontiguousarray(mesh.faces, dtype=np.int32)
    vo = np.ascontiguousarray(mesh.v_off, dtype=np.int64)
    fo = np.ascontiguousarray(mesh.f_off, dtype=np.int64)
    cap = 64 * mesh.nV + 100
    bw = np.zeros(cap, dtype=np.int32)
    ba = np.zeros(cap, dtype=np.int32)
    st = np.zeros(9)
    p = lambda a: a.ctypes.data_as(C.c_void_p)  # noqa: E731
    rc = L.adm_host_tile_check(p(V), C.c_int64(mesh.nV), p(F), C.c_int64(mesh.nT), p(vo), p(fo),
                               C.c_int32(mesh.n_mesh), C.c_int32(with_hinges), C.c_int32(tile), p(bw), p(ba),
                               C.c_int64(cap), p(st))
    nnzb = int(st[4])
    return rc, bw[:nnzb], ba[:nnzb], st


CASES = {
    "icosphere3": lambda: synth.icosphere_shell(3),
    "batch": lambda: synth.shell_batch([0, 2, 3, 1, 4], seed=3),
    "disk": lambda: synth.noisy_disk(3000),
    "grid": lambda: synth.grid_uv(),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("tile", [1, 7, 64, 512, 4096])
@pytest.mark.parametrize("hinges", [0, 1])
def test_every_block_written_once_or_shared(H, name, tile, hinges):
    mesh = CASES[name]()
    if hinges and name == "grid":
        pytest.skip("flat grid: same structure as the disk")
    if tile < 32 and name == "batch":
        pytest.skip("tiny tiles covered on the single meshes")
    rc, bw, ba, st = run(H, mesh, hinges, tile)
    assert rc == 0, rc
    assert (bw != -1).all()                       # every block is produced
    shared = bw == -2
    assert (ba[shared] >= 2).all()                # a shared block has two or more adders
    assert (ba[~shared] == 0).all()               # a plain block has exactly one writer
    assert (int(st[1]) > 0) == bool(shared.any()) # partial slots exist exactly when outputs are shared
    assert st[3] <= 227 * 1024                    # every tile fits FP64 shared memory


def test_one_tile_per_mesh_has_nothing_shared(H):
    mesh = synth.shell_batch([1, 0, 1], seed=2)
    rc, bw, ba, st = run(H, mesh, 1, 100000)
    assert rc == 0
    assert int(st[0]) == 3 and int(st[1]) == 0 and int(st[2]) == 0 and int(st[7]) == 0


def test_unused_vertex_is_zeroed(H):
    """A vertex no triangle references: nothing writes its gradient row or
    diagonal block, so the builder lists both for the per-pass zero fill."""
    V, F = synth.icosphere(2)
    rest = np.concatenate([V, [[3.0, 0.0, 0.0]]])
    mesh = synth.Mesh(rest=rest, faces=F, x=rest)
    rc, bw, ba, st = run(H, mesh, 1, 64)
    assert rc == 0, rc
    assert (bw != -1).all()
    assert int(st[2]) >= 1                          # the unused vertex is in the zero list


@pytest.mark.parametrize("tile", [96, 192, 224])
def test_tiles_keep_two_fp32_blocks_per_sm(H, tile):
    """Every tile's shared memory, with its x region sized for the set's
    largest footprint (the next tile's x is staged there while the current
    tile's chunks are summed), stays within what two FP32 blocks per SM
    allow (228 KB per SM, 1 KB reserved per block), and FP64 within one
    block's 227 KB, on the shell batch's mesh levels."""
    mesh = synth.shell_batch([4, 5, 6, 4], seed=3)
    rc, bw, ba, st = run(H, mesh, 1, tile)
    assert rc == 0, rc
    assert st[8] <= (228 * 1024) // 2 - 1024, st[8]
    assert st[3] <= 227 * 1024, st[3]


@pytest.mark.parametrize("rows,k", [(128, 64), (64, 64), (8, 8)])
def test_tcgen05_operand_layout_and_descriptor(H, rows, k):
    """The learned membrane's tcgen05 operands: the canonical K-major layout
    without swizzle places each BF16 element of a rows x k operand in its
    own slot of the buffer, with 16-byte aligned row pieces (one store of 8
    elements each), and the instruction descriptor encodes BF16 inputs, FP32
    accumulation, K-major operands, N = 64 and M = 128."""
    assert H.adm_host_umma_check(rows, k) == 0
