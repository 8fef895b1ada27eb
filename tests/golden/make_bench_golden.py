"""Write the expected values of one Krylov time step at the benchmark size.

Workload (Sec. 2.2.3 with the fit of Sec. 2.2.1): L = 16 orbitals, 15
electrons (2S_z = +1), the seeded synthetic integrals (seed 0), the seeded
random MPS of bond dimension D = 256 (seed 0) as psi_0, one orthogonal Krylov
step with m = 10 basis vectors (the benchmark's step; also m = 4), dt = 0.05
a.u., D = 256, eps = 1e-8, every fit 0 two-site + 2 one-site sweeps.

Only ``oracle`` (the block-sparse MPO/MPS oracle) and ``synth`` run here; no
value comes from the CUDA library.  Run from the repository root:

    python tests/golden/make_bench_golden.py [m]

It takes several minutes on a few CPU cores and writes
tests/golden/krylov_L16_N15_D256.json (m = 10) or
tests/golden/krylov_L16_N15_D256_m<m>.json.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import bsmps as ob  # noqa: E402

L, N_ELEC, TWO_SZ, D, EPS = 16, 15, 1, 256, 1e-8
DT = 0.05
SCHEDULE = (0, 2)
N_SAMPLES = 64


def sample_occupations(n_up, n_dn, count, seed):
    """Distinct determinants of the sector, as local states per orbital."""
    rng = np.random.default_rng(seed)
    out, seen = [], set()
    while len(out) < count:
        ups = rng.choice(L, n_up, replace=False)
        dns = rng.choice(L, n_dn, replace=False)
        occ = [0] * L
        for i in ups:
            occ[i] |= 1
        for i in dns:
            occ[i] |= 2
        key = tuple(occ)
        if key not in seen:
            seen.add(key)
            out.append(occ)
    return out


def cplx(a):
    a = np.asarray(a, dtype=np.complex128)
    return [a.real.tolist(), a.imag.tolist()]


def main(M=10):
    t0 = time.time()
    I = synth.make_integrals(L, seed=0)
    mpo = ob.hamiltonian_mpo(I.h, I.eri, I.e0)
    A, q = synth.random_mps(L, N_ELEC, TWO_SZ, D, seed=0)
    psi0 = ob.from_dense(A, q)
    sch = ob.Schedule(D, EPS, *SCHEDULE)
    fl = ob.Flops()
    psi1, c, Nk, Hk = ob.krylov_step(mpo, psi0, DT, M, sch, True, fl)
    occs = sample_occupations((N_ELEC + TWO_SZ) // 2, (N_ELEC - TWO_SZ) // 2, N_SAMPLES, 7)
    out = {
        "workload": {"L": L, "n_elec": N_ELEC, "two_sz": TWO_SZ, "D": D, "eps": EPS,
                     "dt": DT, "m": M, "schedule": list(SCHEDULE), "integral_seed": 0,
                     "state_seed": 0},
        "norm2": ob.overlap(psi1, psi1).real,
        "overlap_with_psi0": cplx(ob.overlap(psi0, psi1)),
        "energy": ob.sandwich(mpo, psi1, psi1).real,
        "one_rdm": cplx(ob.one_rdm(psi1)),
        "samples": occs,
        "coefficients": cplx(ob.coefficients(psi1, occs)),
        "krylov_c": cplx(c),
        "krylov_N": cplx(Nk),
        "krylov_H": cplx(Hk),
        "bond_dims": psi1.bond_dims(),
        "oracle_flops": fl.total,
        "oracle_seconds": time.time() - t0,
    }
    name = "krylov_L16_N15_D256.json" if M == 10 else "krylov_L16_N15_D256_m%d.json" % M
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), name)
    with open(path, "w") as f:
        json.dump(out, f)
    print("wrote %s (%.0f s)" % (path, time.time() - t0))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 10)
