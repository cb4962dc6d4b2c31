"""The oracle's count of dense forward-mode operations (route 0, the paper's
ActiveT form): the per-element cost that structured forward mode is
measured against.  The counter is bookkeeping only: it must not change the
route-0 results, and it must scale like the dense rules (a k x k Hessian
per operation)."""
import numpy as np

import oracle

REST = np.array([[0.0, 0, 0], [1, 0, 0], [0.2, 0.9, 0], [0.6, -0.8, 0.1]])
X = REST + 0.01 * np.random.default_rng(0).normal(size=REST.shape)
F = np.array([[0, 1, 2], [1, 0, 3]], dtype=np.int32)
P = oracle.Problem(REST, F, oracle.SHELL, 3, params=[1e5, 0.3, 1e-3])


def test_counts_are_deterministic_and_leave_results_alone():
    xl = X[F[0]].ravel()
    a = oracle.local(oracle.STVK, xl, 3, P.Dinv[0], P.area[0], params=[1e5, 0.3, 1e-3])
    n1 = oracle.dense_flops(oracle.STVK, xl, 3, P.Dinv[0], P.area[0], params=[1e5, 0.3, 1e-3])
    n2 = oracle.dense_flops(oracle.STVK, xl, 3, P.Dinv[0], P.area[0], params=[1e5, 0.3, 1e-3])
    b = oracle.local(oracle.STVK, xl, 3, P.Dinv[0], P.area[0], params=[1e5, 0.3, 1e-3])
    assert n1 == n2 > 0
    assert a["f"] == b["f"] and np.array_equal(a["g"], b["g"]) and np.array_equal(a["H"], b["H"])


def test_hinge_costs_more_than_a_triangle():
    """k = 12 against k = 9: every rule carries a k x k Hessian, and the
    hinge's angle takes more operations than the triangle's strain."""
    t = oracle.dense_flops(oracle.STVK, X[F[0]].ravel(), 3, P.Dinv[0], P.area[0], params=[1e5, 0.3, 1e-3])
    h = oracle.dense_flops(oracle.HINGE, X[P.H[0]].ravel(), 3, thetabar=P.thetabar[0], abar=P.abar[0],
                           params=[0.5, 1.0])
    assert h > t
