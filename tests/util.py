"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle


def rel(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_slots(P: "oracle.Problem", energy: int) -> np.ndarray:
    """Slot map derived from the oracle's pattern: for every element in
    canonical order and every ordered local pair, the block index."""
    out = []
    if energy != oracle.HINGE:
        for vid in P.F:
            for a in vid:
                for b in vid:
                    lo, hi = P.row_ptr[a], P.row_ptr[a + 1]
                    out.append(lo + int(np.searchsorted(P.col[lo:hi], b)))
    if energy in (oracle.HINGE, oracle.SHELL):
        for vid in P.H:
            for a in vid:
                for b in vid:
                    lo, hi = P.row_ptr[a], P.row_ptr[a + 1]
                    out.append(lo + int(np.searchsorted(P.col[lo:hi], b)))
    return np.asarray(out, dtype=np.int64)


def shell_params_split(p):
    """Split shell parameters into the membrane and hinge parameter lists."""
    return list(p[:3]), list(p[3:5])
