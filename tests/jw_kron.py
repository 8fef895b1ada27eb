"""Jordan-Wigner operators as dense Kronecker products (test helper).

Independent of the oracle: the annihilator of spin orbital p on the 2^(2L)
Fock space, mode order 1up, 1down, 2up, ... (Eq. fci), basis index
sum_p n_p 2^p, is Z x ... x Z (p factors, on the lower modes) x a x 1 x ... x 1.
"""
import numpy as np


def spin_orbital_ops(L):
    n = 2 * L
    a1 = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1| on one mode
    z = np.diag([1.0, -1.0])
    eye = np.eye(2)
    ops = []
    for p in range(n):
        mats = [z] * p + [a1] + [eye] * (n - p - 1)
        M = np.array([[1.0]])
        for m in reversed(mats):   # mode 0 is the least significant bit
            M = np.kron(M, m)
        ops.append(M)
    return ops


def site_config_index(L):
    """For every Kronecker basis index (a determinant mask), the index of the
    same configuration in the 4^L site basis, sum_i sigma_i 4^(L-1-i) with
    sigma_i = n_{i,up} + 2 n_{i,down}."""
    J = np.arange(4 ** L, dtype=np.int64)
    idx = np.zeros_like(J)
    for i in range(L):
        up = (J >> (2 * i)) & 1
        dn = (J >> (2 * i + 1)) & 1
        idx = idx * 4 + up + 2 * dn
    return idx
