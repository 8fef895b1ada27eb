"""Seeded synthetic integrals standing in for the paper's active spaces.

The paper takes h_ij (its t_ij) and V_ijkl from quantum-chemistry packages for
H10/STO-6G, H2O/6-31G and C2HI (Section 3); those integral files are not
available, so the workloads use random integrals with the same shape:

* h symmetric; diagonal ~ U[-2, -0.5]; off-diagonal ~ N(0, sd=0.1/(1+|i-j|)^2)
  (hopping that decays along the orbital chain like a hydrogen chain).
* Two-electron integrals in chemist order (ij|kl) = sum_g L^g_ij L^g_kl with
  n_chol symmetric factors L^g_ij ~ N(0, sd=0.3/(1+|i-j|)), which makes the
  (ij),(kl) supermatrix positive semidefinite like real repulsion integrals.
* Optional "localised block": orbitals 0..L/4-1 get h_ii = -3 (a deep,
  iodine-like group split from the rest), used for the large active space.

Draw order (numpy PCG64, ``default_rng(seed)``): the L diagonal entries of h,
the strict upper triangle of h row-major, then for each g the upper triangle of
L^g (diagonal included) row-major.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class IntegralSet:
    """h: (L, L) float64; eri: (L, L, L, L) float64 chemist order (ij|kl); e0."""
    h: np.ndarray
    eri: np.ndarray
    e0: float = 0.0

    @property
    def L(self) -> int:
        return self.h.shape[0]


def make_integrals(L: int, seed: int = 0, n_chol: int = 16,
                   localised_block: bool = False) -> IntegralSet:
    rng = np.random.default_rng(seed)
    h = np.zeros((L, L))
    h[np.diag_indices(L)] = rng.uniform(-2.0, -0.5, size=L)
    iu = np.triu_indices(L, k=1)
    sd = 0.1 / (1.0 + np.abs(iu[0] - iu[1])) ** 2
    h[iu] = rng.standard_normal(len(iu[0])) * sd
    h[(iu[1], iu[0])] = h[iu]
    if localised_block:
        for i in range(max(1, L // 4)):
            h[i, i] = -3.0
    iu0 = np.triu_indices(L, k=0)
    sdc = 0.3 / (1.0 + np.abs(iu0[0] - iu0[1]))
    chol = np.zeros((n_chol, L, L))
    for g in range(n_chol):
        vals = rng.standard_normal(len(iu0[0])) * sdc
        chol[g][iu0] = vals
        chol[g][(iu0[1], iu0[0])] = vals
    eri = np.einsum("gij,gkl->ijkl", chol, chol)
    return IntegralSet(h=h, eri=eri, e0=0.0)
