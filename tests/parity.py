"""Parity measure of the GPU tests: the relative l2 error of every grid function on its
own -- every (slice, node) of a PFASST state, every grid of a batch -- and the worst of
them, so that an error confined to one slice or one node cannot hide under the norm of
all the others.  The last axis of the arrays is the grid; every leading index names
one grid function."""
import numpy as np


def per_array_rel(a, b):
    """Relative l2 error of a against b per grid function (last axis); returns an array
    shaped like the leading axes.  A grid function that is exactly zero in b is measured
    against the norm of the whole of b instead."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (a.shape, b.shape)
    if a.ndim == 1:
        a, b = a[None], b[None]
    A, B = a.reshape(-1, a.shape[-1]), b.reshape(-1, b.shape[-1])
    num = np.linalg.norm(A - B, axis=1)
    den = np.linalg.norm(B, axis=1)
    whole = max(np.linalg.norm(B), 1e-300)
    den = np.where(den > 0.0, den, whole)
    return (num / den).reshape(a.shape[:-1])


def worst_rel(a, b, what=""):
    """Worst per-grid-function relative l2 error; prints it with its (slice, node, ...) index."""
    errs = per_array_rel(a, b)
    idx = np.unravel_index(int(np.argmax(errs)), errs.shape)
    worst = float(errs[idx])
    print(f"parity{(' ' + what) if what else ''}: worst per-array rel l2 {worst:.3e} at index "
          f"{tuple(int(i) for i in idx)} of {errs.shape}")
    return worst
