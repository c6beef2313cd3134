"""6-vector form of a symmetric 3x3 matrix (paper §3, Eq. 6: "we use a 6-vector s_k").

The paper does not fix the basis.  The Mandel basis is used: the three
diagonal entries, then sqrt(2) times the (1,2), (0,2), (0,1) entries.  With it
the Frobenius inner product of symmetric matrices equals the dot product of
their 6-vectors, so the 9x6 map R_k of Eq. 6 has orthonormal columns and its
pseudo-inverse is its transpose.  The result x* does not depend on the basis.
"""
import numpy as np

SQ2 = np.sqrt(2.0)
# Mandel index -> (row, col) of the symmetric matrix
PAIRS = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
I6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])     # the identity matrix as a 6-vector


def to_mandel(S):
    """(..., 3, 3) symmetric -> (..., 6)."""
    S = np.asarray(S)
    return np.stack([S[..., 0, 0], S[..., 1, 1], S[..., 2, 2],
                     SQ2 * S[..., 1, 2], SQ2 * S[..., 0, 2], SQ2 * S[..., 0, 1]], axis=-1)


def from_mandel(s):
    """(..., 6) -> (..., 3, 3) symmetric."""
    s = np.asarray(s)
    S = np.empty(s.shape[:-1] + (3, 3))
    S[..., 0, 0] = s[..., 0]
    S[..., 1, 1] = s[..., 1]
    S[..., 2, 2] = s[..., 2]
    S[..., 1, 2] = S[..., 2, 1] = s[..., 3] / SQ2
    S[..., 0, 2] = S[..., 2, 0] = s[..., 4] / SQ2
    S[..., 0, 1] = S[..., 1, 0] = s[..., 5] / SQ2
    return S


def basis():
    """The six symmetric basis matrices E_j with from_mandel(e_j) = E_j."""
    return from_mandel(np.eye(6))
