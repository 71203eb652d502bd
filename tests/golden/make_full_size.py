"""Write tests/golden/full_n24_trotter.json with the oracle alone.

The n = 24 workload (seeded JW-shaped Hamiltonian, 2000 terms, 10 first-order
Trotter steps at dt = 0.05, 20,000 rotations, Hartree-Fock state with 12
electrons) evolved by the FP64 gate-level oracle; stores 64 amplitudes at
seeded indices plus the basis state's own amplitude, the norm and <H>.  Used by
tests/test_gpu_full_size.py to check the GPU path at full size.  Run from the
repository root:  python tests/golden/make_full_size.py [output.json]
(about 15 minutes on 16 cores; the default output is this folder).
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_09020_gb300 import synth  # noqa: E402

N, TERMS, SEED, DT, STEPS = 24, 2000, 1, 0.05, 10


def main():
    ham = synth.jw_hamiltonian(N, TERMS, SEED)
    rx, rz, rt = oracle.trotter_rotations(ham.x, ham.z, ham.c, DT, STEPS, 1)
    basis = synth.hartree_fock_index(N // 2)
    psi = oracle.basis_state(N, basis)
    t0 = time.time()
    for k in range(0, len(rt), 500):
        oracle.apply_rotations(psi, N, rx[k:k + 500], rz[k:k + 500], rt[k:k + 500])
        print(f"{k + 500} rotations, {time.time() - t0:.0f} s", flush=True)
    g = np.random.Generator(np.random.PCG64(2024))
    idx = sorted(set(g.integers(0, 1 << N, size=64).tolist()) | {basis} |
                 set(np.argsort(-np.abs(psi))[:16].tolist()))
    energy = oracle.expval(psi, N, ham.x, ham.z, ham.c)
    out = {
        "what": "oracle (FP64, gate-decomposed) after the n=24 Trotter workload",
        "n": N, "terms": TERMS, "seed": SEED, "dt": DT, "steps": STEPS, "order": 1,
        "basis_state": basis, "rotations": int(len(rt)),
        "norm2": oracle.norm2(psi, N), "energy": energy,
        "indices": [int(i) for i in idx],
        "re": [float(psi[i].real) for i in idx],
        "im": [float(psi[i].imag) for i in idx],
        "seconds": time.time() - t0, "threads": oracle.num_threads(),
    }
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                               "full_n24_trotter.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path, "energy", energy)


if __name__ == "__main__":
    main()
