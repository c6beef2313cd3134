"""Helpers shared by the scripts that write stored expected values under
tests/golden/ and the tests that read them (no method arithmetic)."""
import numpy as np


def mesh_checksum(X, T):
    """Order-sensitive checksum of a mesh: sizes and index-weighted sums, so a
    test notices when the seeded mesh generators no longer give the mesh a
    stored solution was computed on."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T)
    w = np.arange(1, len(X) + 1, dtype=np.float64)
    return np.array([len(X), len(T), float(w @ X[:, 0]), float(w @ X[:, 1]), float(w @ X[:, 2]),
                     float(np.arange(1, len(T) + 1, dtype=np.float64) @ T.astype(np.float64).sum(1))])
