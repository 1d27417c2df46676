"""Error measure of Eq. 5.1 (oracle).

Test infrastructure only; see the package docstring.

error = max over f in {E, B} of ( sum_i |f_i^t - f_i^b|^2 / sum_i |f_i^b|^2 )^(1/2),
f^t from the FMM and f^b from the brute-force sum (the paper's second sum
index reads "i = i"; i = 1..N is meant).
"""
from __future__ import annotations

import numpy as np


def rel_l2(f_test, f_ref) -> float:
    a = np.asarray(f_test, dtype=np.float64)
    b = np.asarray(f_ref, dtype=np.float64)
    den = float(np.sum(b * b))
    num = float(np.sum((a - b) ** 2))
    if den == 0.0:
        return 0.0 if num == 0.0 else float("inf")
    return (num / den) ** 0.5


def field_error(E_t, B_t, E_b, B_b) -> float:
    """Eq. 5.1."""
    return max(rel_l2(E_t, E_b), rel_l2(B_t, B_b))
