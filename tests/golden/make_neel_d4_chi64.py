"""Writes neel_d4_chi64_50it.txt: the oracle's reduced-sequential run of the D=4,
chi=64 Neel-like state (1e-2 noise, seed 0) for 50 iterations of left, up, right,
down moves from the environment grown from the fold (Sec. II; Sec. III-IV for the
move).  Records the corner-spectrum change of every iteration, and after the 50th
the mean Heisenberg bond energy, ln kappa and the largest corner singular value.
Calls the oracle only.  Run from the repository root:
    python tests/golden/make_neel_d4_chi64.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import ctm_oracle as O  # noqa: E402
from paper_2306_08212_gb300 import inputs as I  # noqa: E402


def main():
    A, B = I.neel_sites(4, eps=1e-2, seed=0)
    chi, iters = 64, 50
    env = O.init_env(A, B, chi)
    spec = O.corner_spectra(env)
    deltas = []
    for _ in range(iters):
        for d in O.MOVE_ORDER:
            O.move(env, d, A, B, chi, chi, "reduced_sequential")
        new = O.corner_spectra(env)
        deltas.append(O.spectrum_delta(spec, new))
        spec = new
    H = O.heisenberg_bond()
    energy = float(np.mean([O.expect_bond(env, A, B, b, H) for b in range(4)]))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "neel_d4_chi64_50it.txt")
    with open(out, "w") as f:
        f.write("# Oracle (oracle/ctm_oracle.py), reduced-sequential, D=4 chi=64 Neel-like sites\n")
        f.write("# (inputs.neel_sites(4, eps=1e-2, seed=0)), 50 iterations of left, up, right,\n")
        f.write("# down from init_env; written by tests/golden/make_neel_d4_chi64.py\n")
        f.write(f"energy_mean {energy:.15e}\n")
        f.write(f"log_kappa {O.log_kappa_sites(env, A, B):.15e}\n")
        f.write(f"sigma0 {spec[0][0]:.15e}\n")
        f.write("deltas " + " ".join(f"{d:.3e}" for d in deltas) + "\n")
    print(out)


if __name__ == "__main__":
    main()
