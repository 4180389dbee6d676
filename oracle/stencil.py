"""Oracle for the paper's two other parametric kernels (Section 5) -- TEST
INFRASTRUCTURE ONLY.

* Matrix transposition (Fig. "transpose"): c[j][i] = a[i][j].  The figure prints
  c[i*N+j] = a[i][j], which is a copy; the text (and the table's name) describe a
  transposition, which is what this oracle defines.
* 1D Jacobi (Fig. "1dj"): int a[2N]; at time step t, for every interior point p
  (0 <= p < N-2): if t is odd, a[p+1] = (a[N+p] + a[N+p+1] + a[N+p+2]) / 3,
  else a[N+p+1] = (a[p] + a[p+1] + a[p+2]) / 3, with C's integer division
  (truncation toward zero).  A step reads one half and writes the other, so all
  points of a step may be taken at once.
"""
from __future__ import annotations

import numpy as np


def transpose(a: np.ndarray) -> np.ndarray:
    """c with c[j][i] = a[i][j] (numpy's transpose, made contiguous)."""
    return np.ascontiguousarray(np.asarray(a).T)


def c_div3(x: np.ndarray) -> np.ndarray:
    """C integer division by 3: the quotient truncated toward zero."""
    x = np.asarray(x, dtype=np.int64)
    return np.sign(x) * (np.abs(x) // 3)


def jacobi(a: np.ndarray, n: int, steps: int) -> np.ndarray:
    """The array after `steps` time steps; a has 2n int32 entries."""
    a = np.array(a, dtype=np.int64).copy()
    if a.shape != (2 * n,):
        raise ValueError("a must hold 2n entries")
    p = np.arange(n - 2)
    for t in range(steps):
        if t % 2:
            a[p + 1] = c_div3(a[n + p] + a[n + p + 1] + a[n + p + 2])
        else:
            a[n + p + 1] = c_div3(a[p] + a[p + 1] + a[p + 2])
    return a.astype(np.int32)
