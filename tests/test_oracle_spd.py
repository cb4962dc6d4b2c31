"""Pins of the oracle's per-term Hessian filtering (Sec. 7.1: negative
eigenvalues of each element term's local Hessian clamped before assembly)
to facts outside it:

* on a matrix built from a chosen orthonormal basis and spectrum, the
  projection is that basis with the clamped spectrum;
* it leaves a positive semidefinite matrix unchanged and is idempotent;
* the assembled projected Hessian is positive semidefinite, and it exceeds
  the plain Hessian by a positive semidefinite matrix (only eigenvalues
  below zero were raised);
* at the rest state, where StVK's local Hessians are already semidefinite,
  projection changes nothing;
* a term's translations, exact zeros of its Hessian, stay zero when eps > 0
  (the reading of the filter), while its negative eigenvalues become eps."""
import numpy as np
import pytest

import oracle
import synth

SHELL_P = [1.0e5, 0.3, 1.0e-3]


def test_spd_project_known_eigensystem():
    rng = np.random.default_rng(1)
    Q, _ = np.linalg.qr(rng.normal(size=(12, 12)))
    lam = np.array([-3.0, -1e-3, 0.0, 0.5, 2.0, 5.0, -7.0, 1.0, 3.0, 4.0, -0.25, 9.0])
    H = (Q * lam) @ Q.T
    for eps in (0.0, 1e-2):
        want = (Q * np.where(lam < 0, eps, lam)) @ Q.T
        assert np.abs(oracle.spd_project(H, eps) - want).max() <= 1e-13 * np.abs(lam).max()


def test_spd_project_idempotent_and_identity_on_psd():
    rng = np.random.default_rng(2)
    A = rng.normal(size=(9, 9))
    H = A + A.T
    P = oracle.spd_project(H)
    assert np.abs(oracle.spd_project(P) - P).max() <= 1e-13 * np.abs(P).max()
    S = A @ A.T
    assert np.abs(oracle.spd_project(S) - S).max() <= 1e-13 * np.abs(S).max()


def dense(P, vals):
    return oracle.bsr_to_dense(P.nV, P.vdim, P.row_ptr, P.col, vals)


@pytest.mark.parametrize("energy,params", [(oracle.SHELL, SHELL_P), (oracle.HINGE, [0.5, 1.0]),
                                           (oracle.STVK, SHELL_P), (oracle.NH, SHELL_P)])
def test_projected_assembly_psd_and_dominates(energy, params):
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=5e-2, seed=3)
    P = oracle.Problem(V, F, energy, 3, params)
    H = dense(P, P.assemble(x)["vals"])
    Hp = dense(P, P.assemble_projected(x)["vals"])
    scale = np.abs(H).max()
    assert np.linalg.eigvalsh(H).min() < -1e-3 * scale       # the plain Hessian is indefinite here
    assert np.linalg.eigvalsh(Hp).min() >= -1e-12 * scale
    assert np.linalg.eigvalsh(Hp - H).min() >= -1e-12 * scale


def test_symdir_projection_psd():
    g = synth.grid_uv(n=9, sigma=0.2, seed=5)
    P = oracle.Problem(g.rest, g.faces, oracle.SYMDIR, 2)
    Hp = dense(P, P.assemble_projected(g.x)["vals"])
    assert np.linalg.eigvalsh(Hp).min() >= -1e-12 * np.abs(Hp).max()


def test_rest_state_unchanged():
    V, F = synth.icosphere(2)
    P = oracle.Problem(V, F, oracle.STVK, 3, SHELL_P)
    a = P.assemble(V)["vals"]
    b = P.assemble_projected(V)["vals"]
    assert np.abs(a - b).max() <= 1e-10 * np.abs(a).max()


def test_eps_sets_clamped_eigenvalues():
    V, F = synth.icosphere(1)
    x = synth.perturb(V, sigma=5e-2, seed=6)
    P = oracle.Problem(V, F, oracle.NH, 3, SHELL_P)
    for t in range(P.nT):  # the first triangle whose Hessian is indefinite
        loc = oracle.local(oracle.NH, x[P.F[t]], 3, P.Dinv[t], P.area[t], params=SHELL_P)
        lam = np.linalg.eigvalsh(loc["H"])
        if lam.min() < -1e-3 * np.abs(lam).max():
            break
    eps = 1e-3 * np.abs(lam).max()
    lp = np.sort(np.linalg.eigvalsh(oracle.spd_project(loc["H"], eps)))
    # negative: below -tau max|lambda|; the translations' round-off zeros stay zero
    want = np.sort(np.where(lam < -oracle.SPD_TAU * np.abs(lam).max(), eps, lam))
    assert np.sum(lam < -oracle.SPD_TAU * np.abs(lam).max()) >= 1
    assert np.abs(lp - want).max() <= 1e-10 * np.abs(lam).max()


def test_translations_stay_null_with_positive_eps():
    V, F = synth.icosphere(1)
    x = synth.perturb(V, sigma=5e-2, seed=7)
    P = oracle.Problem(V, F, oracle.HINGE, 3, [0.5, 1.0])
    loc = oracle.local(oracle.HINGE, x[P.H[0]], 3, thetabar=P.thetabar[0], abar=P.abar[0], params=[0.5, 1.0])
    T = oracle.translations(4, 3)
    eps = 1e-2 * np.abs(loc["H"]).max()
    Hp = oracle.spd_project(loc["H"], eps, T)
    assert np.abs(Hp @ T).max() <= 1e-12 * np.abs(Hp).max()       # translations stay in the null space
    B = np.linalg.svd(T, full_matrices=True)[0][:, 3:]
    lam = np.linalg.eigvalsh(B.T @ loc["H"] @ B)
    want = np.sort(np.where(lam < 0, eps, lam))
    got = np.sort(np.linalg.eigvalsh(B.T @ Hp @ B))
    assert np.abs(got - want).max() <= 1e-10 * np.abs(lam).max()


def test_hinge_structural_zero_not_clamped():
    """Every hinge Hessian has one structural zero besides its translations
    (theta depends on 5 of the 6 Gram invariants of its edge vectors); with
    eps > 0 it must stay zero whatever sign round-off gives it."""
    V, F = synth.icosphere(2)
    x = synth.perturb(V, sigma=5e-2, seed=33)
    P = oracle.Problem(V, F, oracle.HINGE, 3, [0.5, 1.0])
    T = oracle.translations(4, 3)
    B = np.linalg.svd(T, full_matrices=True)[0][:, 3:]
    for h in range(0, P.nH, 37):
        loc = oracle.local(oracle.HINGE, x[P.H[h]], 3, thetabar=P.thetabar[h], abar=P.abar[h], params=[0.5, 1.0])
        lam = np.linalg.eigvalsh(B.T @ loc["H"] @ B)
        assert np.sort(np.abs(lam))[0] <= 1e-14 * np.abs(lam).max()      # the structural zero
        eps = 1e-2 * np.abs(lam).max()
        lp = np.linalg.eigvalsh(B.T @ oracle.spd_project(loc["H"], eps, T) @ B)
        assert np.sort(np.abs(lp))[0] <= 1e-12 * np.abs(lam).max()       # still zero, not eps
