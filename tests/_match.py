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
