"""Writes the stored expected values under tests/golden from the oracle's closed forms only.

free_field_spectrum_2x2x2x4_k0.12.txt: eigenvalues of the Wilson matrix at U = 1,
kappa = 0.12, lattice 2x2x2x4, antiperiodic in time (Re, Im per line), from
1 - 2 kappa sum cos p +- 2 i kappa sqrt(sum sin^2 p), p_k = 2 pi n/L_k,
p_4 = pi (2 n + 1)/L_4, each with multiplicity 2 (spin) x 3 (colour).
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

if __name__ == "__main__":
    ev = oracle.free_field_eigenvalues((2, 2, 2, 4), 0.12, (1, 1, 1, -1))
    np.savetxt(os.path.join(HERE, "free_field_spectrum_2x2x2x4_k0.12.txt"),
               np.stack([ev.real, ev.imag], axis=1), fmt="%.17e",
               header="Wilson free-field spectrum, 2x2x2x4, kappa=0.12, bc=(1,1,1,-1): Re Im")
