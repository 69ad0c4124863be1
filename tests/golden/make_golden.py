"""Write the stored expected values under tests/golden/. Calls only oracle/ and synth/.

* d3_p010_bruteforce.txt: ln Z_l(s) for all 256 syndromes of the d=3 rotated
  code under depolarizing p=0.10 (Sec. 2.2), summed over all 4^9 Paulis
  (Eq. 3 taken literally), plus the MLD decision (Eq. 4). Covers every
  syndrome of the d=3 workload (1024 errors from seed 0).
* d5_group_enum.txt: ln Z_l(s) for 4 syndromes of the d=5 code under
  depolarizing p=0.12, each summed term by term over the 2^24 stabiliser-group
  elements (first line of Eq. 7).

Run: python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    d, n = 3, 9
    Z = oracle.bruteforce_table(d, synth.depolarizing(n, 0.10))
    with open(os.path.join(HERE, "d3_p010_bruteforce.txt"), "w") as f:
        f.write("# d=3 rotated code, depolarizing p=0.10; brute force over 4^9 Paulis (Eq. 3)\n")
        f.write("# columns: syndrome_index lnZ_I lnZ_X lnZ_Z lnZ_Y argmax (ties -> lowest)\n")
        for s in range(Z.shape[0]):
            lz = np.log(Z[s])
            top = lz.max()
            am = int(np.flatnonzero(lz >= top - 1e-12)[0])
            f.write(f"{s} " + " ".join(f"{v:.15e}" for v in lz) + f" {am}\n")
    d, n = 5, 25
    noise = synth.depolarizing(n, 0.12)
    E = synth.sample_errors(d, noise, 4, seed=synth.config_seed(1, 5, 0.12))
    syn = synth.syndromes_of(d, E)
    reps = oracle.representatives(d, syn)
    with open(os.path.join(HERE, "d5_group_enum.txt"), "w") as f:
        f.write("# d=5 rotated code, depolarizing p=0.12; stabiliser-group enumeration (Eq. 7)\n")
        f.write("# columns: syndrome word0 (decimal) lnZ_I lnZ_X lnZ_Z lnZ_Y\n")
        for b in range(len(E)):
            vals = [oracle.group_logz(d, noise, reps[b, l]) for l in range(4)]
            f.write(f"{int(syn[b, 0])} " + " ".join(f"{v:.15e}" for v in vals) + "\n")


if __name__ == "__main__":
    main()
