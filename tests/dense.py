"""Dense-matrix helpers for pinning the oracle on tiny systems.

Independent of both the oracle and the CUDA path: every operator is built from
the textbook 2x2 matrices of the paper's Sec. "Pauli and Clifford Group" with
numpy Kronecker products.  Qubit j is bit j of the index, so the leftmost
Kronecker factor is qubit n-1.
"""
import numpy as np

I2 = np.eye(2, dtype=complex)
X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.array([[1, 0], [0, -1]], dtype=complex)
H = np.array([[1, 1], [1, -1]], dtype=complex) / np.sqrt(2)
S = np.array([[1, 0], [0, 1j]], dtype=complex)
SDG = S.conj().T


def one_qubit(n, q, m):
    out = np.array([[1.0 + 0j]])
    for j in reversed(range(n)):
        out = np.kron(out, m if j == q else I2)
    return out


def pauli(n, x, z):
    out = np.array([[1.0 + 0j]])
    for j in reversed(range(n)):
        xb, zb = (x >> j) & 1, (z >> j) & 1
        m = Y if (xb and zb) else X if xb else Z if zb else I2
        out = np.kron(out, m)
    return out


def cnot(n, c, t):
    dim = 1 << n
    m = np.zeros((dim, dim), dtype=complex)
    for k in range(dim):
        m[k ^ (1 << t) if (k >> c) & 1 else k, k] = 1.0
    return m


def rz(n, q, theta):
    return one_qubit(n, q, np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)]))


def rotation(n, x, z, theta):
    """exp(-i theta/2 P) = cos(theta/2) I - i sin(theta/2) P, exact since P^2 = I."""
    return np.cos(theta / 2) * np.eye(1 << n) - 1j * np.sin(theta / 2) * pauli(n, x, z)


def all_paulis(n):
    for x in range(1 << n):
        for z in range(1 << n):
            yield x, z
