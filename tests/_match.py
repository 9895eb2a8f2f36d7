"""Test helpers: map the library's master ordering onto the oracle's by coordinates."""
import numpy as np


def coord_permutation(X_lib, X_orc, tol=1e-9):
    """perm such that X_orc[perm[k]] == X_lib[k] (within tol); asserts a bijection."""
    assert X_lib.shape == X_orc.shape, (X_lib.shape, X_orc.shape)
    scale = max(1.0, np.abs(X_orc).max())
    q_lib = np.round(X_lib / (tol * scale)).astype(np.int64)
    q_orc = np.round(X_orc / (tol * scale)).astype(np.int64)
    o_lib = np.lexsort(q_lib.T[::-1])
    o_orc = np.lexsort(q_orc.T[::-1])
    assert np.array_equal(q_lib[o_lib], q_orc[o_orc]), "master coordinate sets differ"
    perm = np.empty(len(X_lib), dtype=np.int64)
    perm[o_lib] = o_orc
    return perm


def rel_errors(got, ref, axis=None):
    """(L2 relative error, largest entry error over the largest reference entry).

    The L2 norm over millions of entries can hide a few wrong entries (hanging
    points, surface masters); the second figure is the per-entry check beside it.
    With axis=0 both are taken per column and the worst column is returned."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    if axis is None:
        den = max(np.linalg.norm(ref), 1e-300)
        amax = max(np.max(np.abs(ref)), 1e-300)
        return np.linalg.norm(got - ref) / den, np.max(np.abs(got - ref)) / amax
    den = np.maximum(np.linalg.norm(ref, axis=axis), 1e-300)
    amax = np.maximum(np.max(np.abs(ref), axis=axis), 1e-300)
    return (np.max(np.linalg.norm(got - ref, axis=axis) / den),
            np.max(np.max(np.abs(got - ref), axis=axis) / amax))


def assert_close(got, ref, bar, axis=None, what=""):
    """Both the L2 relative error and the per-entry error (scaled by max|ref|) below bar."""
    l2, ent = rel_errors(got, ref, axis)
    assert l2 < bar and ent < bar, f"{what}: L2 {l2:.3e}, per entry {ent:.3e}, bar {bar:.1e}"
    return l2, ent
