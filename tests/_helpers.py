"""Test-side helpers built from numpy/scipy only (no oracle, no CUDA code)."""
import numpy as np
import scipy.linalg

# the three SU(2) Pauli matrices and the diagonal abelian generator used by flux fixtures
H_ABELIAN = np.diag([1.0, -1.0, 0.0]).astype(np.complex128)


def random_su3(rng, n=None):
    """Haar-random SU(3) from the QR decomposition of a complex Ginibre matrix."""
    shape = (3, 3) if n is None else (n, 3, 3)
    Z = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=-2, axis2=-1)
    Q = Q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[..., None, None]


def random_hermitian_traceless(rng, scale=1.0):
    A = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    H = (A + A.conj().T) / 2
    H -= np.trace(H) / 3 * np.eye(3)
    return scale * H


def gauge_transform(U, dims, g):
    """U'_mu(x) = g(x) U_mu(x) g(x+mu)^+ in the canonical layout."""
    L = [int(v) for v in dims]
    V = int(np.prod(L))
    idx = np.arange(V)
    x = np.stack([(idx // int(np.prod(L[:m]))) % L[m] for m in range(4)], axis=1)
    out = np.empty_like(U)
    for mu in range(4):
        xs = x.copy()
        xs[:, mu] = (xs[:, mu] + 1) % L[mu]
        s2 = xs[:, 0] + L[0] * (xs[:, 1] + L[1] * (xs[:, 2] + L[2] * xs[:, 3]))
        out[:, mu] = g @ U[:, mu] @ np.conj(np.transpose(g[s2], (0, 2, 1)))
    return out


def su3_distance(A, B):
    return float(np.max(np.abs(A - B)))


def unitarity_violation(U):
    U = U.reshape(-1, 3, 3)
    eye = np.eye(3)
    uu = U @ np.conj(np.transpose(U, (0, 2, 1)))
    return float(max(np.max(np.abs(uu - eye)), np.max(np.abs(np.linalg.det(U) - 1))))


def expm(X):
    return scipy.linalg.expm(X)


def gell_mann():
    """The eight Gell-Mann matrices (textbook definition)."""
    l = np.zeros((8, 3, 3), dtype=np.complex128)
    l[0][0, 1] = l[0][1, 0] = 1
    l[1][0, 1] = -1j
    l[1][1, 0] = 1j
    l[2][0, 0], l[2][1, 1] = 1, -1
    l[3][0, 2] = l[3][2, 0] = 1
    l[4][0, 2] = -1j
    l[4][2, 0] = 1j
    l[5][1, 2] = l[5][2, 1] = 1
    l[6][1, 2] = -1j
    l[6][2, 1] = 1j
    l[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return l


def flux_field(dims, n01, n23):
    """Constant abelian field strength in the (0,1) and (2,3) planes.

    Every (0,1) plaquette equals exp(i f H), every (2,3) plaquette exp(i g H),
    H = diag(1,-1,0), f = 2 pi n01/(L0 L1), g = 2 pi n23/(L2 L3); all other
    plaquettes are 1.  Built with the usual twist on the last slice.
    """
    L = [int(v) for v in dims]
    V = int(np.prod(L))
    f = 2 * np.pi * n01 / (L[0] * L[1])
    gg = 2 * np.pi * n23 / (L[2] * L[3])
    U = np.zeros((V, 4, 3, 3), dtype=np.complex128)
    for s in range(V):
        x = [(s // int(np.prod(L[:m]))) % L[m] for m in range(4)]
        ph = [0.0, 0.0, 0.0, 0.0]
        ph[1] = f * x[0]
        if x[0] == L[0] - 1:
            ph[0] = -f * L[0] * x[1]
        ph[3] = gg * x[2]
        if x[2] == L[2] - 1:
            ph[2] = -gg * L[2] * x[3]
        for mu in range(4):
            U[s, mu] = np.diag(np.exp(1j * ph[mu] * np.array([1.0, -1.0, 0.0])))
    return U, f, gg
