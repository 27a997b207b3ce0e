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


# The FP64 path and the oracle differ only in the order of rounding.  Where the problem
# itself magnifies rounding -- a late slice whose solution has decayed by orders of
# magnitude carries the absolute rounding of the earlier slices, high-order uniform
# nodes have large quadrature weights of both signs -- no implementation can agree
# with the oracle to 1e-12 relative on that array.  The conditioning is measured by the
# oracle alone: the change of each array when the oracle's own input is moved by one
# unit in the last place.  The bound per array is max(tol, K_FLOOR x that change);
# K_FLOOR covers the many roundings along the way against the single one of the input.
K_FLOOR = 10.0


def ulp_perturbed(u, seed=12345):
    """u with every entry moved by one unit in the last place (random sign)."""
    u = np.asarray(u, dtype=np.float64)
    rng = np.random.default_rng(seed)
    return u * (1.0 + rng.choice([-1.0, 1.0], size=u.shape) * 2.0 ** -52)


def worst_rel_floor(a, b, b_pert, tol, what=""):
    """Worst per-array error of a against b in units of the per-array bound
    max(tol, K_FLOOR * per-array change of b under the one-ulp input perturbation that
    gave b_pert); below 1 passes.  Prints the worst array, its error and its bound."""
    err = per_array_rel(a, b)
    bound = np.maximum(tol, K_FLOOR * per_array_rel(b_pert, b))
    ratio = err / bound
    idx = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    print(f"parity{(' ' + what) if what else ''}: worst per-array rel l2 {float(err.max()):.3e}; worst "
          f"error/bound {float(ratio[idx]):.3f} at index {tuple(int(i) for i in idx)} of {ratio.shape} "
          f"(error {float(err[idx]):.3e}, bound {float(bound[idx]):.3e})")
    return float(ratio[idx])
