"""Write the stored expected values under tests/golden/. Calls only oracle/ and synth/.

* d3_p010_bruteforce.txt: ln Z_l(s) for all 256 syndromes of the d=3 rotated
  code under depolarizing p=0.10 (Sec. 2.2), summed over all 4^9 Paulis
  (Eq. 3 taken literally), plus the MLD decision (Eq. 4). Covers every
  syndrome of the d=3 workload (1024 errors from seed 0).
* d5_group_enum.txt: ln Z_l(s) for 4 syndromes of the d=5 code under
  depolarizing p=0.12, each summed term by term over the 2^24 stabiliser-group
  elements (first line of Eq. 7).
* large_mps.txt: ln Z_l(s) of the FP64 boundary-MPS sweep (Sec. 3.2.1, left
  QR sweep then right-to-left SVD keeping min(chi, #values), no cutoff) for
  d=13, 15, 17 and 25: depolarizing p=0.12 and biased eta=100 at p=0.12,
  syndromes from seed config_seed(5, d, 0.12), the X_L string of the l_X = 1
  classes on column d-1. Noise tables are the FP32-rounded ones the GPU tests
  pass.
* d17_exact_64.txt: exact ln Z_l(s) (dense contraction of Eq. 7) of the first
  64 syndromes of the d=17 depolarizing p=0.12 workload (seed
  config_seed(5, 17, 0.12)).

Run: python tests/golden/make_golden.py [--large-only]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


LARGE_CASES = [(13, 32, "depolarizing", 16), (13, 56, "depolarizing", 2), (15, 72, "depolarizing", 2),
               (17, 32, "depolarizing", 4), (17, 64, "depolarizing", 4), (17, 32, "biased", 4), (17, 64, "biased", 4),
               (25, 32, "depolarizing", 2)]


def large_noise(d, kind):
    n = d * d
    t = synth.depolarizing(n, 0.12) if kind == "depolarizing" else synth.biased(n, 0.12, 100.0)
    return t.astype(np.float32)


def write_large():
    import oracle.mps as omps
    with open(os.path.join(HERE, "large_mps.txt"), "w") as f:
        f.write("# FP64 boundary-MPS sweep (Sec. 3.2.1), no cutoff; X_L of l_X = 1 on column d-1\n")
        f.write("# columns: d chi noise b lnZ_I lnZ_X lnZ_Z lnZ_Y\n")
        for d, chi, kind, B in LARGE_CASES:
            noise = large_noise(d, kind)
            E = synth.sample_errors(d, noise, B, seed=synth.config_seed(5, d, 0.12))
            syn = synth.syndromes_of(d, E)
            ref = omps.decode_mps(d, noise.astype(np.float64), syn, chi, xl_column=d - 1)
            for b in range(B):
                f.write(f"{d} {chi} {kind} {b} " + " ".join(f"{v:.15e}" for v in ref[b]) + "\n")
            f.flush()
    d = 17
    noise = large_noise(d, "depolarizing")
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, 64, seed=synth.config_seed(5, d, 0.12)))
    ref, _ = oracle.decode(d, noise.astype(np.float64), syn)
    with open(os.path.join(HERE, "d17_exact_64.txt"), "w") as f:
        f.write("# d=17, depolarizing p=0.12 (FP32-rounded table), first 64 syndromes of seed config_seed(5, 17, 0.12)\n")
        f.write("# exact dense contraction (Eq. 7); columns: b lnZ_I lnZ_X lnZ_Z lnZ_Y\n")
        for b in range(64):
            f.write(f"{b} " + " ".join(f"{v:.15e}" for v in ref[b]) + "\n")


def main():
    if "--large-only" in sys.argv:
        write_large()
        return
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
    write_large()


if __name__ == "__main__":
    main()
