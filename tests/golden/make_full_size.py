"""Write tests/golden/full_n24_trotter.npz with the oracle alone.

The n = 24 workload (seeded JW-shaped Hamiltonian, 2000 terms, 10 first-order
Trotter steps at dt = 0.05, 20,000 rotations, Hartree-Fock state with 12
electrons) evolved by the FP64 gate-level oracle.  Stored: 8192 amplitudes at
seeded indices drawn uniformly among the basis states where the oracle's state
is non-zero (every string's X/Y part has even weight, so the parity of the
electron number is conserved: these are the 8,388,608 states with an even
number of ones), the 16 largest amplitudes and the initial basis state's own
amplitude, plus the norm, <H> and the Hamiltonian's seed and shape.  Used by
tests/test_gpu_full_size.py (complex128 at 1e-12 on every stored amplitude;
complex64 infidelity and energy error against these values) and by bench.py's
precision report.

Run from the repository root:  python tests/golden/make_full_size.py [out.npz]
(about an hour on 8 cores; the default output is this folder).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2602_09020_gb300 import synth  # noqa: E402

N, TERMS, SEED, DT, STEPS = 24, 2000, 1, 0.05, 10
SAMPLES, SAMPLE_SEED = 8192, 2024


def main():
    ham = synth.jw_hamiltonian(N, TERMS, SEED)
    rx, rz, rt = oracle.trotter_rotations(ham.x, ham.z, ham.c, DT, STEPS, 1)
    basis = synth.hartree_fock_index(N // 2)
    psi = oracle.basis_state(N, basis)
    t0 = time.time()
    for k in range(0, len(rt), 500):
        oracle.apply_rotations(psi, N, rx[k:k + 500], rz[k:k + 500], rt[k:k + 500])
        print(f"{k + 500} rotations, {time.time() - t0:.0f} s", flush=True)
    seconds = time.time() - t0
    nonzero = np.flatnonzero(psi != 0)
    g = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    drawn = g.choice(nonzero, size=SAMPLES, replace=False)
    top = np.argsort(-np.abs(psi))[:16]
    idx = np.unique(np.concatenate([drawn, top, [basis]])).astype(np.int64)
    energy = oracle.expval(psi, N, ham.x, ham.z, ham.c)
    path = sys.argv[1] if len(sys.argv) > 1 else os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                               "full_n24_trotter.npz")
    np.savez_compressed(
        path,
        what=np.array("oracle (FP64, gate-decomposed) after the n=24 Trotter workload"),
        n=N, terms=TERMS, seed=SEED, dt=DT, steps=STEPS, order=1,
        basis_state=basis, rotations=len(rt), nonzero_count=len(nonzero),
        norm2=oracle.norm2(psi, N), energy=energy,
        indices=idx, amps=psi[idx].astype(np.complex128),
        seconds=seconds, threads=oracle.num_threads())
    print("wrote", path, "energy", energy, "nonzero", len(nonzero), "stored", len(idx))


if __name__ == "__main__":
    main()
