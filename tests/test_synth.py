"""Seeded synthetic inputs: sizes of the paper-scale workloads, determinism,
orientation."""
import numpy as np

import synth


def test_grid_sizes_and_determinism():
    a, b = synth.grid_uv(), synth.grid_uv()
    assert a.nV == 1089 and a.nT == 2048
    assert np.array_equal(a.x, b.x)
    assert not np.array_equal(a.x, synth.grid_uv(seed=2).x)


def test_icosphere_level7_sizes_and_orientation():
    v, f = synth.icosphere(7)
    assert v.shape[0] == 163842 and f.shape[0] == 327680
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    assert (np.einsum("ij,ij->i", a, np.cross(b - a, c - a)) > 0).all()   # outward


def test_noisy_disk_size():
    d = synth.noisy_disk()
    assert 0.95e6 < d.nT < 1.05e6
    assert d.faces.max() < d.nV
    u, w = d.x[d.faces[:, 1]] - d.x[d.faces[:, 0]], d.x[d.faces[:, 2]] - d.x[d.faces[:, 0]]
    assert (u[:, 0] * w[:, 1] - u[:, 1] * w[:, 0] > 0).all()          # no folded UV triangle


def test_shell_batch_paper_scale():
    lv = synth.shell_batch_levels("paper")
    assert lv.shape[0] == 700 and set(np.unique(lv)) == {4, 5, 6}
    b = synth.shell_batch(lv)
    assert b.nV == 2162040 and b.nT == 4321280 and b.n_mesh == 700
    assert b.v_off[-1] == b.nV and b.f_off[-1] == b.nT
    # faces of mesh m index only its own vertices
    m = 123
    fm = b.faces[b.f_off[m]:b.f_off[m + 1]]
    assert fm.min() >= b.v_off[m] and fm.max() < b.v_off[m + 1]


def test_membrane_samples_stretch_range():
    F = synth.membrane_samples(1000)
    s = np.linalg.svd(F, compute_uv=False)
    assert s.min() >= 0.7 - 1e-12 and s.max() <= 1.4 + 1e-12
