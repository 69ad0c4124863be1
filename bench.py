"""Benchmark: batched boundary-MPS MLD of the rotated surface code on GB300.

Workload (one "step"): decode 65,536 seeded syndromes of the d=9 rotated code
under depolarizing p=0.10 at bond dimension chi=32 (4 coset log-probabilities
each, plus the argmax) in one mld_decode call on inputs resident in HBM. At
this point chi is at or above the exact bond 2^floor(9/2) = 16, so no
singular value is discarded: the step is the pure error, the column MPO.MPS
products, power-of-two renormalisation, the final contraction and the argmax
(no QR or SVD runs). Synthetic inputs: errors drawn from the counter
generator in synth/, syndromes extracted.

Other workloads (--workload): mixed (the d=3..13 graph batch), large (d=17
and 25 at truncating chi), ler (logical-error rates of the d/p grid against
the oracle), grad, dmle, dem, point (one (d, chi, p) decode point), kw (the
Kac-Ward decode under independent X/Z noise, d=9..25).

Prints one JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle
on the host cores instead (a bounded sample per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

D, CHI, P, B = 9, 32, 0.10, 65536
SEED = synth.config_seed(1, D, P)
L2_FLUSH_BYTES = 256 << 20
METRIC = "syndromes/s at d=9 χ=32 (4 cosets), mixed-precision vs FP32, |ΔlogP|≤1e-3"
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense TF32 / BF16 tensor rates of GB300

# DRAM bytes per syndrome of the decode kernel (dram__bytes_read.sum + write.sum of one ncu
# capture of 8,192 syndromes of the headline kernel), valid only for the kernel sources they
# were taken on: any change to them makes the traffic unknown (null).
TRAFFIC_SOURCES_SHA = "a2b856029856e7f9"
TRAFFIC_BYTES_PER_SYNDROME = {0: (286.208e3 + 1.536e3) / 8192, 2: (286.208e3 + 0.0) / 8192}


# sources of the headline kernel (decode_exact_kernel<9, *>): its plan, layout and templates (the
# host-side code object declared beside them in mld_internal.h does not enter the kernel)
TRAFFIC_SOURCES = ("mld_plan.h", "mld_exact_impl.cuh", "mld_exact.h", "mld_exact.cu")


def kernel_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for name in TRAFFIC_SOURCES:
        f = os.path.join(ROOT, "paper_2605_17230_gb300", "csrc", name)
        h.update(name.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _measured_peaks():
    """The driver-written measured peaks of this machine's GPUs, if present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def wilson_interval(k, n, z=1.959963984540054):
    """Wilson score interval of a binomial proportion k/n (95% by default)."""
    if n == 0:
        return (0.0, 1.0)
    ph = k / n
    den = 1.0 + z * z / n
    c = (ph + z * z / (2 * n)) / den
    h = z * ((ph * (1 - ph) / n + z * z / (4 * n * n)) ** 0.5) / den
    return (max(0.0, c - h), min(1.0, c + h))


def _env_int(k, dflt):
    try:
        return int(os.environ.get(k, dflt))
    except ValueError:
        return dflt


def workload(B_local, b0):
    n = D * D
    noise = synth.depolarizing(n, P).astype(np.float32)
    E = synth.sample_errors(D, noise, B_local, seed=SEED, b0=b0)
    return noise, synth.syndromes_of(D, E)


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({nm for r in rows for nm, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(sample=B):
    """The FP64 oracle (exact dense contraction, OpenMP over syndromes) on
    the host cores, on a bounded sample of the same workload; the same on one
    core, and the oracle's FP64 boundary-MPS mode (the plain method of Sec.
    3.2.1 in numpy, at the same chi) on a few syndromes."""
    import oracle
    import oracle.mps as omps
    noise, syn = workload(sample, 0)
    oracle.decode(D, noise, syn[:64])                  # warm-up
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.decode(D, noise, syn, threads=cores)
    dt = time.perf_counter() - t
    one = min(sample, 2048)
    t = time.perf_counter()
    oracle.decode(D, noise, syn[:one], threads=1)
    dt1 = time.perf_counter() - t
    nm = 4
    t = time.perf_counter()
    omps.decode_mps(D, noise.astype(np.float64), syn[:nm], CHI, xl_column=D - 1)
    dtm = time.perf_counter() - t
    return {"value": sample / dt, "unit": "syndromes/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample} of the {B} d=9 p=0.10 syndromes (rank 0's batch), exact FP64 dense "
                      f"contraction, {dt:.1f} s wall on {cores} threads",
            "one_core_value": one / dt1, "one_core_sample": f"first {one} syndromes, 1 thread",
            "mps_mode_value": nm / dtm,
            "mps_mode_sample": f"first {nm} syndromes, FP64 boundary MPS at chi={CHI} (numpy QR/SVD), 1 process"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    sample = args.ref_sample
    noise, syn = workload(sample, 0)
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.decode(D, noise, syn[:256], threads=cores)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.decode(D, noise, syn, threads=cores)
    dt = time.perf_counter() - t
    v = args.steps * sample / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "syndromes/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"d={D} chi=exact p={P} depolarizing; sample of "
                                                        f"{sample} syndromes per step", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "syndromes/s", "cores": cores, "kind": "oracle",
                             "sample": f"{sample} syndromes per step"},
            "e2e": {"value": v, "unit": "syndromes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


MIXED_CHI = {3: 16, 5: 16, 7: 16, 9: 32, 11: 32, 13: 64}


# what a mixed-precision request runs at each d of the mixed batch
PRODUCT_PATH = {
    0: "FP32 FFMA products (the split-TF32 path is slower at this d; a mixed request runs the FP32 kernel)",
    9: "split-TF32 mma.sync tensor-core products (hi.hi + hi.lo + lo.hi) for data-site products of at "
       "least 32x16x32, FP32 elsewhere",
    11: "dense-state FP32 column transfer (untruncated chi; the faster exact kernel at this d, 2.6M "
        "against 2.1M syndromes/s for the split-TF32 boundary-MPS kernel; a mixed request runs the same "
        "kernel)",
    13: "dense-state FP32 column transfer (untruncated chi; no product is MMA-shaped; a mixed request "
        "runs the same kernel)",
}


def run_mixed(args):
    """Mixed batch (1,048,576 syndromes, d uniform over 3..13, p ~ U[0.02, 0.18]
    per syndrome, chi by d) decoded by one CUDA-graph launch."""
    import torch
    import paper_2605_17230_gb300 as mld
    total = args.mixed_total
    ds = sorted(MIXED_CHI)
    per = total // len(ds)
    items_by_prec, host = {}, []
    codes = {d: mld.Code(d) for d in ds}
    for d in ds:
        p = synth.per_syndrome_depolarizing(per, seed=synth.config_seed(2, d, 0.0), lo=0.02, hi=0.18)
        E = synth.sample_errors(d, p, per, seed=synth.config_seed(2, d, 0.1))
        host.append((d, p, synth.syndromes_of(d, E)))
    for prec in (mld.MLD_FP32, mld.MLD_MIXED_TF32):
        items = []
        for d, p, syn in host:
            items.append((codes[d], torch.tensor(p.astype(np.float32), device="cuda"),
                          torch.tensor(syn.view(np.int64), device="cuda"), MIXED_CHI[d], prec,
                          torch.empty((per, 4), dtype=torch.float64, device="cuda"),
                          torch.empty((per,), dtype=torch.uint8, device="cuda")))
        items_by_prec[prec] = items
    res = {}
    for prec, items in items_by_prec.items():
        g = mld.Graph(mld.make_jobs(items))
        for _ in range(max(1, args.warmup)):
            g.launch()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g.launch()
        e1.record()
        torch.cuda.synchronize()
        res[prec] = (e0.elapsed_time(e1) / args.steps, g)
    import oracle
    per_d = {}
    for k, (d, p, syn) in enumerate(host):
        a = items_by_prec[mld.MLD_FP32][k][5].cpu().numpy()
        b = items_by_prec[mld.MLD_MIXED_TF32][k][5].cpu().numpy()
        # error of both precisions against the FP64 oracle on a sample of this distance's syndromes
        ns = 256
        ref, _ = oracle.decode(d, p[:ns].astype(np.float32).astype(np.float64), syn[:ns],
                               threads=os.cpu_count() or 1)
        fin = np.isfinite(ref)
        # this distance alone: one mld_decode per precision on the same batch
        rate = {}
        for prec in (mld.MLD_FP32, mld.MLD_MIXED_TF32):
            it = items_by_prec[prec][k]
            codes[d].decode(it[1], it[2], MIXED_CHI[d], prec)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            codes[d].decode(it[1], it[2], MIXED_CHI[d], prec)
            e1.record()
            torch.cuda.synchronize()
            rate[prec] = per / (e0.elapsed_time(e1) / 1e3)
        per_d[str(d)] = {"chi": MIXED_CHI[d], "max_abs_dlogP_mixed_vs_fp32": float(np.abs(a - b).max()),
                         "max_abs_dlogP_fp32_vs_oracle": float(np.abs(a[:ns][fin] - ref[fin]).max()),
                         "max_abs_dlogP_mixed_vs_oracle": float(np.abs(b[:ns][fin] - ref[fin]).max()),
                         "oracle_sample": ns,
                         "mixed_product_path": PRODUCT_PATH.get(d, PRODUCT_PATH[0]),
                         "fp32_syndromes_per_s_alone": rate[mld.MLD_FP32],
                         "mixed_syndromes_per_s_alone": rate[mld.MLD_MIXED_TF32]}
    ms32, msm = res[mld.MLD_FP32][0], res[mld.MLD_MIXED_TF32][0]
    line = {"metric": "syndromes/s, mixed d=3..13 batch in one graph launch", "workload": "mixed",
            "value": per * len(ds) / (msm / 1e3), "unit": "syndromes/s", "fp32_value": per * len(ds) / (ms32 / 1e3),
            "ms_per_launch": msm, "fp32_ms_per_launch": ms32, "syndromes": per * len(ds), "steps": args.steps,
            "per_d": per_d, "data": "synthetic",
            "config": {"d": ds, "chi_by_d": MIXED_CHI, "p": "U[0.02, 0.18] per syndrome, depolarizing"}}
    print(json.dumps(line), flush=True)


def _hist_summary(h):
    """Kept-bond statistics from mld_decode_bond_histogram (bin 0: steps that
    ran in the global spill arena)."""
    b = h.copy()
    spilled = int(b[0])
    b[0] = 0
    tot = int(b.sum())
    if tot == 0:
        return None
    ks = np.arange(len(b))
    cdf = np.cumsum(b) / tot
    return {"cuts": tot, "mean": float((b * ks).sum() / tot), "p99": int(np.searchsorted(cdf, 0.99)),
            "max": int(ks[b > 0].max()), "steps_in_spill_arena": spilled}


def _posterior(x):
    return np.exp(x - np.logaddexp.reduce(x, axis=1, keepdims=True))


def run_point(args):
    """One (d, chi, p) point of the untruncated or truncated sweep on its own: --point-batch
    depolarizing-p syndromes (seed config_seed(1, d, p)), FP32 and the mixed request, --warmup
    untimed decodes then --steps timed ones (CUDA events, L2 flushed between them); reports
    syndromes/s per precision and the counted flops rate. The small cases the ncu summaries
    capture run through this."""
    import torch
    import paper_2605_17230_gb300 as mld
    d, chi, p, Bp = args.point_d, args.point_chi, args.point_p, args.point_batch
    noise = synth.depolarizing(d * d, p).astype(np.float32)
    syn = synth.syndromes_of(d, synth.sample_errors(d, noise, Bp, seed=synth.config_seed(1, d, p)))
    code = mld.Code(d)
    if args.point_exact_kernel:
        code.set_exact_kernel(args.point_exact_kernel)
    nz = torch.tensor(noise, device="cuda")
    sy = torch.tensor(syn.view(np.int64), device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    out = {}
    for name, prec in (("fp32", mld.MLD_FP32), ("mixed", mld.MLD_MIXED_TF32)):
        for _ in range(args.warmup):
            code.decode(nz, sy, chi, prec)
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            code.decode(nz, sy, chi, prec)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        st = code.status()
        if st != 0:
            raise RuntimeError("device status: " + mld.mld_status_string(st))
        t = float(np.median(ms))
        out[name] = {"syndromes_per_s": Bp / (t / 1e3), "ms_median": t,
                     "counted_tflops": code.flops(chi, prec) * Bp / t / 1e9}
    code.close()
    print(json.dumps({"metric": "syndromes/s of one decode point", "workload": "point",
                      "config": {"d": d, "chi": chi, "p": p, "syndromes": Bp, "steps": args.steps,
                                 "warmup": args.warmup, "exact_kernel": args.point_exact_kernel},
                      **out, "data": "synthetic"}), flush=True)


def run_large(args):
    """The scale workload: rotated d=17 and 25, depolarizing p=0.12 and biased eta=100 (p=0.12),
    16,384 syndromes per point (seed config_seed(5, d, p)), chi = 32, 64, 128 (--large-p, --large-d,
    --large-chi and --large-noise change the grid; the comparison columns need chi = 128). Every point reports
    syndromes/s, the executed flops rate, the kept-bond histogram of the rank-adaptive truncation,
    the logical-error rate with its 95% Wilson interval, and the largest change of the leading
    coset's ln Z and of the posterior against the chi=128 run of the same syndromes."""
    import torch
    import paper_2605_17230_gb300 as mld
    Bl = args.large_batch
    chis = tuple(sorted(args.large_chi))
    out = []
    for d in args.large_d:
        code = mld.Code(d)
        n = d * d
        pl = args.large_p
        for name, noise in ((f"depolarizing p={pl:g}", synth.depolarizing(n, pl)),
                            (f"biased eta=100 p={pl:g}", synth.biased(n, pl, 100.0))):
            if name.split()[0] not in args.large_noise:
                continue
            noise = noise.astype(np.float32)
            E = synth.sample_errors(d, noise, Bl, seed=synth.config_seed(5, d, pl))
            true = synth.true_class(d, E)
            nz = torch.tensor(noise, device="cuda")
            sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
            res = {}
            for chi in chis[::-1]:
                code.decode(nz, sy[:256], chi)                     # warm-up: workspaces
                torch.cuda.synchronize()
                code.executed_flops()
                code.bond_histogram()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                lp, am = code.decode(nz, sy, chi)
                e1.record()
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                st = code.status()
                if st != 0:
                    raise RuntimeError("device status: " + mld.mld_status_string(st))
                res[chi] = (lp.cpu().numpy(), am.cpu().numpy(), ms, code.executed_flops(), code.bond_histogram())
            ref = res[128][0] if 128 in res else None
            lead = np.argmax(ref, axis=1) if ref is not None else None
            rows = np.arange(Bl)
            for chi in chis:
                lp, am, ms, fl, h = res[chi]
                k = int((am != true).sum())
                rec = {"d": d, "chi": chi, "noise": name, "syndromes": Bl, "ms": ms,
                       "syndromes_per_s": Bl / (ms / 1e3), "executed_tflops": fl / ms / 1e9,
                       "bonds": _hist_summary(h), "ler": k / Bl, "ler_ci95": wilson_interval(k, Bl),
                       "max_abs_dlogP_leading_vs_chi128":
                           None if ref is None else float(np.abs(lp[rows, lead] - ref[rows, lead]).max()),
                       "max_abs_dposterior_vs_chi128":
                           None if ref is None else float(np.abs(_posterior(lp) - _posterior(ref)).max()),
                       "argmax_equals_chi128": None if ref is None else float(np.mean(am == res[128][1]))}
                out.append(rec)
                print(json.dumps(rec), flush=True)
        code.close()
    print(json.dumps({"metric": "syndromes/s at truncating chi (rank-adaptive sweep)", "workload": "large",
                      "points": out, "data": "synthetic", "dtype": "f32",
                      "cutoff": "singular values <= 1e-7 sigma_1 discarded (default)"}), flush=True)


def run_ler(args):
    """Logical-error rates of the d/p grid (d = 5, 7, 9; depolarizing p = 0.05, 0.10, 0.15, 0.19;
    65,536 syndromes each, seed config_seed(1, d, p)): the GPU decoder's LER at every distinct chi of
    {8, 16, 32, exact} (chi >= 2^floor(d/2) is exact, so d = 5, 7 have the exact point only) and the
    FP64 oracle's exact-MLD LER on the same syndromes, each with a 95% Wilson interval, and the
    decisions that differ from the oracle where its two best cosets are more than 1e-4 apart in
    ln Z (must be 0 at exact chi). The paper's optimal threshold of 18.9% (Sec. 2.2, Table 1) is the
    context: below it the LER falls with d, near it the curves meet."""
    import torch
    import oracle
    import paper_2605_17230_gb300 as mld
    Bq = args.ler_batch
    table = []
    for d in (5, 7, 9):
        code = mld.Code(d)
        n = d * d
        exact = 1 << (d // 2)
        chis = sorted({min(c, exact) for c in (8, 16, 32, exact)})
        for p in (0.05, 0.10, 0.15, 0.19):
            noise = synth.depolarizing(n, p).astype(np.float32)
            E = synth.sample_errors(d, noise, Bq, seed=synth.config_seed(1, d, p))
            syn = synth.syndromes_of(d, E)
            true = synth.true_class(d, E)
            ref, am_ref = oracle.decode(d, noise, syn, threads=os.cpu_count() or 1)
            top = np.sort(ref, axis=1)
            clear = top[:, -1] - top[:, -2] > 1e-4
            k_ref = int((am_ref != true).sum())
            nz = torch.tensor(noise, device="cuda")
            sy = torch.tensor(syn.view(np.int64), device="cuda")
            for chi in chis:
                lp, am = code.decode(nz, sy, chi)
                torch.cuda.synchronize()
                am = am.cpu().numpy()
                k = int((am != true).sum())
                rec = {"d": d, "p": p, "chi": chi, "exact": chi >= exact, "syndromes": Bq,
                       "ler_gpu": k / Bq, "ler_gpu_ci95": wilson_interval(k, Bq),
                       "ler_oracle_exact": k_ref / Bq, "ler_oracle_ci95": wilson_interval(k_ref, Bq),
                       "non_tie_decisions_differing_from_oracle": int((am[clear] != am_ref[clear]).sum()),
                       "ties": int((~clear).sum())}
                table.append(rec)
                print(json.dumps(rec), flush=True)
        code.close()
    exact_rows = {(r["d"], r["p"]): r["ler_oracle_exact"] for r in table}
    ordering = {f"p={p}": [exact_rows[(d, p)] for d in (5, 7, 9)] for p in (0.05, 0.10, 0.15, 0.19)}
    print(json.dumps({"metric": "logical-error rates, GPU vs FP64 oracle (exact MLD)", "workload": "ler",
                      "table": table, "oracle_ler_by_d_5_7_9": ordering,
                      "tolerance": "decisions equal to the oracle's wherever its top two cosets differ by "
                                   "more than 1e-4 in ln Z; 0 mismatches required at exact chi",
                      "data": "synthetic"}), flush=True)


def run_grad(args):
    """Adjoint of the sweep on the d=7 workload with per-qubit biased noise:
    gradient of sum_b ln Pr(l_true | s_b) over 65,536 syndromes (and the same
    at d=9, chi=32 over 16,384 syndromes, d=11 chi=32 over 4,096 and d=13
    chi=64 over 1,024, reported as d9_value, d11_value, d13_value)."""
    import torch
    import paper_2605_17230_gb300 as mld

    def one(d, chi, Bg):
        n = d * d
        noise = synth.lognormal_biased(n, seed=3).astype(np.float32)
        E = synth.sample_errors(d, noise, Bg, seed=4)
        syn = synth.syndromes_of(d, E)
        code = mld.Code(d)
        nz = torch.tensor(noise, device="cuda")
        sy = torch.tensor(syn.view(np.int64), device="cuda")
        cls = torch.tensor(synth.true_class(d, E).astype(np.int64), device="cuda")
        lp, _ = code.decode(nz, sy, chi)
        up = torch.zeros_like(lp)
        up.scatter_(1, cls[:, None], 1.0)
        up -= torch.softmax(lp, dim=1)                # d/d lnZ of ln Pr(l_true|s)
        dn = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
        for _ in range(max(1, args.warmup)):
            mld.mld_decode_grad(code.handle, nz, sy, Bg, chi, up, None, dn)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            mld.mld_decode_grad(code.handle, nz, sy, Bg, chi, up, None, dn)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        t0 = torch.cuda.Event(enable_timing=True); t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        for _ in range(args.steps):
            code.decode(nz, sy, chi)
        t1.record()
        torch.cuda.synchronize()
        return ms, Bg / (ms / 1e3), Bg / (t0.elapsed_time(t1) / args.steps / 1e3)

    Bg = args.batch if args.batch != B else 65536
    ms, value, fwd = one(7, 32, Bg)
    line = {"metric": "syndromes/s of the adjoint (d=7, chi=32, per-qubit biased noise)", "workload": "grad",
            "value": value, "unit": "syndromes/s", "ms_per_step": ms, "syndromes": Bg,
            "steps": args.steps, "data": "synthetic", "dtype": "f32 contraction, f64 accumulation",
            "forward_only_value": fwd}
    if args.batch == B:
        _, v9, f9 = one(9, 32, 16384)
        line["d9_value"] = v9
        line["d9_forward_only_value"] = f9
        _, v11, f11 = one(11, 32, 4096)
        line["d11_value"] = v11
        line["d11_forward_only_value"] = f11
        _, v13, f13 = one(13, 64, 1024)
        line["d13_value"] = v13
        line["d13_forward_only_value"] = f13
    print(json.dumps(line), flush=True)


def run_dmle(args):
    """Noise estimation from unlabelled syndromes at scale (Sec. 3.2.4, Eq. 10):
    full-batch Adam on -mean ln sum_l Z_l(s) over 1,048,576 d=9 syndromes drawn
    from per-qubit lognormal biased rates (seed 21), starting from a uniform
    table; a step is one forward sweep, one adjoint sweep and the update."""
    import torch
    import paper_2605_17230_gb300 as mld
    d, chi = 9, 32
    n = d * d
    Bt = args.batch if args.batch != B else 1 << 20
    true = synth.lognormal_biased(n, seed=21)
    E = synth.sample_errors(d, true, Bt, seed=22)
    code = mld.Code(d)
    sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
    mld.estimate_noise(code, sy, chi, steps=max(1, args.warmup))     # warm-up run (own start)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    tab, _, losses = mld.estimate_noise(code, sy, chi, steps=args.steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    p_true = true[:, 1:].sum(axis=1)
    fit = tab.cpu().numpy()[:, 1:].sum(axis=1)
    line = {"metric": "syndromes/s of a full-batch noise-estimation step (d=9, chi=32, forward + adjoint + Adam)",
            "workload": "dmle", "value": Bt / (ms / 1e3), "unit": "syndromes/s", "ms_per_step": ms,
            "syndromes": Bt, "steps": args.steps, "data": "synthetic", "dtype": "f32 contraction, f64 accumulation",
            "rate_error_start": float(np.abs(0.05 - p_true).mean()),
            "rate_error_end": float(np.abs(fit - p_true).mean()),
            "rate_corr_end": float(np.corrcoef(fit, p_true)[0, 1]),
            "loss_first": float(losses[0]), "loss_last": float(losses[-1])}
    print(json.dumps(line), flush=True)


def run_dem(args):
    """Detector-picture decode (Sec. 3.2.2) of a code-capacity error-mechanism
    model at d=9: X, Y and Z mechanisms on every qubit with lognormal rates
    (median 0.03, seed 5), 65,536 syndromes sampled from the mechanisms
    (seed 6); all four classes per syndrome from one sweep. The same model at
    d=11 (16,384 syndromes) is reported as d11_value."""
    import torch
    import paper_2605_17230_gb300 as mld

    def one(d, Bd):
        q, c, p = synth.mechanism_model(d, seed=5)
        E = synth.sample_mechanisms(d, q, c, p, Bd, seed=6)
        sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
        code = mld.Code(d)
        for _ in range(max(1, args.warmup)):
            code.decode_dem(q, c, p, sy)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            lp, am = code.decode_dem(q, c, p, sy)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        true = torch.tensor(synth.true_class(d, E).astype(np.int64), device="cuda")
        ler = float((am.long() != true).float().mean().item())
        code.close()
        return ms, len(p), ler

    Bd = args.batch if args.batch != B else 65536
    ms, nm, ler = one(9, Bd)
    line = {"metric": "syndromes/s of the detector-picture decode (d=9, X/Y/Z mechanisms per qubit, 4 classes)",
            "workload": "dem", "value": Bd / (ms / 1e3), "unit": "syndromes/s", "ms_per_step": ms,
            "syndromes": Bd, "mechanisms": int(nm), "steps": args.steps, "data": "synthetic",
            "dtype": "f32 contraction, f64 ln Z", "logical_error_rate": ler}
    if args.batch == B:
        ms11, nm11, ler11 = one(11, 16384)
        line.update({"d11_value": 16384 / (ms11 / 1e3), "d11_mechanisms": int(nm11),
                     "d11_logical_error_rate": ler11})
    print(json.dumps(line), flush=True)


def _lead_gap(lp, ref):
    """max, p99 and p99.9 of |ln Z_lead(lp) - ln Z_lead(ref)| with lead the
    leading class of ref (torch tensors [B][4])."""
    lead = ref.argmax(dim=1, keepdim=True)
    g = (lp.gather(1, lead) - ref.gather(1, lead)).abs().flatten()
    return {"max": g.max().item(), "p99": g.quantile(0.99).item(), "p999": g.quantile(0.999).item()}


def run_kw(args):
    """Kac-Ward decode (Sec. 3.1.3) under independent X/Z noise with
    px = pz = p on every qubit (default 0.10): syndromes sampled from the
    product table (seed config_seed(7, d, p)); per d the FP32 rate, the FP64
    rate on a quarter of the batch, the logical-error rate, and on the same
    syndromes the boundary-MPS decode (untruncated chi at d <= 13, chi = 32
    above) with its rate and the number of decisions that differ."""
    import torch
    import paper_2605_17230_gb300 as mld

    def timed(fn, steps, before=None):
        for _ in range(max(1, args.warmup)):
            fn()
        torch.cuda.synchronize()
        if before is not None:
            before()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps, out

    default_b = {5: 65536, 7: 65536, 9: 65536, 11: 32768, 13: 32768, 15: 16384, 17: 16384}
    peak, sms = mld.mld_measure_fp32_peak(2.0)
    rows = []
    for d in args.kw_d:
        n, p = d * d, args.kw_p
        Bd = args.kw_batch or default_b.get(d, 4096)
        px = np.full(n, p, np.float32)
        tab = synth.independent_xz(px, px)
        E = synth.sample_errors(d, tab, Bd, seed=synth.config_seed(7, d, p))
        true = torch.tensor(synth.true_class(d, E).astype(np.int64), device="cuda")
        sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
        code = mld.Code(d)
        dpx = torch.tensor(px, device="cuda")
        ms32, (lp, am) = timed(lambda: code.decode_xz(dpx, dpx, sy, mld.MLD_FP32), args.steps,
                               before=code.xz_executed_flops)
        flops = code.xz_executed_flops() / (args.steps * Bd)
        B64 = max(1, Bd // 4)
        ms64, (lp64, am64) = timed(lambda: code.decode_xz(dpx, dpx, sy[:B64], mld.MLD_FP64),
                                   max(1, args.steps // 5))
        if code.status() != 0:
            raise RuntimeError("device status after the Kac-Ward decode")
        row = {"d": d, "p": p, "syndromes": Bd, "fp32_value": Bd / (ms32 / 1e3), "fp32_ms": ms32,
               "fp64_value": B64 / (ms64 / 1e3), "fp64_syndromes": B64,
               "logical_error_rate": float((am.long() != true).float().mean().item()),
               "fp32_fp64_decisions_differ": int((am[:B64] != am64).sum().item()),
               "fp32_vs_fp64_leading_dlnZ": _lead_gap(lp[:B64], lp64),
               "executed_flops_per_syndrome": flops,
               "roofline": {"bound": "alu", "achieved": flops * Bd / (ms32 / 1e3) / 1e12, "peak": peak,
                            "unit": "TFLOP/s", "frac": flops * Bd / (ms32 / 1e3) / 1e12 / peak, "traffic": None}}
        if not args.kw_no_mps:
            chi = 1 << (d // 2) if d <= 13 else 32
            nz = torch.tensor(tab.astype(np.float32), device="cuda")
            code.decode(nz, sy[:256], chi)
            msm, (lpm, amm) = timed(lambda: code.decode(nz, sy, chi), max(1, args.steps // 10))
            row.update({"mps_chi": chi, "mps_value": Bd / (msm / 1e3),
                        "mps_decisions_differ": int((amm != am).sum().item()),
                        "mps_logical_error_rate": float((amm.long() != true).float().mean().item())})
        rows.append(row)
        code.close()
    line = {"metric": "syndromes/s of the Kac-Ward decode (independent X/Z noise, 4 classes)", "workload": "kw",
            "unit": "syndromes/s", "data": "synthetic", "dtype": "complex f32 elimination, f64 ln Z",
            "steps": args.steps, "warmup": args.warmup, "rows": rows,
            "roofline_note": f"achieved = flops executed by the FP32 elimination (counted on the device: 6 per "
                             f"multiplier, 8 per complex multiply-subtract of an updated column) / kernel time; peak = "
                             f"FFMA microbenchmark on {sms} SMs (mld_measure_fp32_peak, 2 s)"}
    print(json.dumps(line), flush=True)


def _crossings(ler, ds, ps):
    """Where the LER curves of consecutive distances cross: the first sign
    change of ler(d2, p) - ler(d1, p) along ps, by linear interpolation."""
    cross = []
    for d1, d2 in zip(ds, ds[1:]):
        diff = [ler[(d2, p)] - ler[(d1, p)] for p in ps]
        pc = None
        for i in range(len(ps) - 1):
            if diff[i] < 0 <= diff[i + 1]:
                pc = ps[i] + (ps[i + 1] - ps[i]) * (-diff[i]) / (diff[i + 1] - diff[i])
                break
        cross.append({"d": [d1, d2], "p_cross": pc})
    return cross


def run_threshold(args):
    """Logical-error rates under depolarizing noise around the optimal
    threshold the paper quotes for it (18.9%, Sec. 3.1.2), decoded by the
    boundary-MPS path: untruncated chi at d <= 13 (2^floor(d/2)), --thr-chi
    above. Per point --thr-batch syndromes (seed config_seed(10, d, p)), the
    LER with its Wilson interval, the decode rate, and the crossings of
    consecutive distances."""
    import torch
    import paper_2605_17230_gb300 as mld

    ps, Bd = args.thr_p, args.thr_batch
    rows, ler = [], {}
    for d in args.thr_d:
        n = d * d
        chi = 1 << (d // 2) if d <= 13 else args.thr_chi
        code = mld.Code(d)
        for p in ps:
            tab = synth.depolarizing(n, p)
            E = synth.sample_errors(d, tab, Bd, seed=synth.config_seed(10, d, p))
            true = synth.true_class(d, E)
            sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
            nz = torch.tensor(tab.astype(np.float32), device="cuda")
            code.decode(nz, sy[:256], chi)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            _, am = code.decode(nz, sy, chi)
            e1.record()
            torch.cuda.synchronize()
            if code.status() != 0:
                raise RuntimeError("device status after the decode")
            k = int((am.cpu().numpy() != true).sum())
            lo, hi = wilson_interval(k, Bd)
            ler[(d, p)] = k / Bd
            rows.append({"d": d, "chi": chi, "p": p, "syndromes": Bd, "logical_error_rate": k / Bd,
                         "ci95": [lo, hi], "syndromes_per_s": Bd / (e0.elapsed_time(e1) / 1e3)})
        code.close()
    line = {"metric": "logical-error rate under depolarizing noise, boundary-MPS MLD", "workload": "threshold",
            "unit": "logical errors per syndrome", "data": "synthetic", "dtype": "f32 sweep, f64 ln Z",
            "paper_threshold": 0.189, "rows": rows, "crossings": _crossings(ler, list(args.thr_d), ps)}
    print(json.dumps(line), flush=True)


def run_kw_threshold(args):
    """Logical-error rates under bit-flip noise (independent X flips with
    probability p on every qubit, no Z errors) decoded exactly by the Kac-Ward
    path, for d in --kw-d and p on a grid around the optimal threshold the
    paper quotes for this channel (10.9%, the random-bond Ising model on the
    Nishimori line; Sec. 3.1.2). Per point --kw-batch syndromes (default
    16,384, seed config_seed(8, d, p)), the LER with its Wilson interval, and
    the crossing of each pair of consecutive distances (linear interpolation
    of the LER difference between grid points)."""
    import torch
    import paper_2605_17230_gb300 as mld

    ps = args.kw_threshold_p
    Bd = args.kw_batch or 16384
    rows, ler = [], {}
    for d in args.kw_d:
        n = d * d
        code = mld.Code(d)
        for p in ps:
            px = np.full(n, p, np.float32)
            tab = synth.independent_xz(px, np.zeros(n))
            E = synth.sample_errors(d, tab, Bd, seed=synth.config_seed(8, d, p))
            true = synth.true_class(d, E)
            sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
            t0 = time.time()
            _, am = code.decode_xz(torch.tensor(px, device="cuda"), None, sy, mld.MLD_FP32)
            torch.cuda.synchronize()
            dt = time.time() - t0
            if code.status() != 0:
                raise RuntimeError("device status after the Kac-Ward decode")
            k = int((am.cpu().numpy() != true).sum())
            lo, hi = wilson_interval(k, Bd)
            ler[(d, p)] = k / Bd
            rows.append({"d": d, "p": p, "syndromes": Bd, "logical_error_rate": k / Bd, "ci95": [lo, hi],
                         "seconds": dt})
        code.close()
    cross = _crossings(ler, list(args.kw_d), ps)
    line = {"metric": "logical-error rate under bit-flip noise, exact MLD (Kac-Ward)", "workload": "kw-threshold",
            "unit": "logical errors per syndrome", "data": "synthetic", "dtype": "complex f32 elimination, f64 ln Z",
            "paper_threshold": 0.109, "rows": rows, "crossings": cross}
    print(json.dumps(line), flush=True)


def run_kw_chi(args):
    """Convergence of the truncated boundary-MPS decode to exact MLD at
    distances the exact contraction cannot reach: independent X/Z noise with
    px = pz = p (default 0.05 and 0.10), --kw-batch syndromes per point
    (default 4,096, seed config_seed(9, d, p)), the Kac-Ward decode (FP64) as
    the exact reference, and the boundary-MPS decode of the product table at
    each chi of --kw-chi with the singular-value cutoff --kw-chi-cutoff:
    decisions that differ from exact MLD, the largest |d ln Z| of the leading
    class, both logical-error rates (Sec. 3.2.1: the bond needed to match
    exact MLD)."""
    import torch
    import paper_2605_17230_gb300 as mld

    Bd = args.kw_batch or 4096
    rows = []
    for d in args.kw_d:
        n = d * d
        code = mld.Code(d)
        for p in args.kw_chi_p:
            px = np.full(n, p, np.float32)
            tab = synth.independent_xz(px, px)
            E = synth.sample_errors(d, tab, Bd, seed=synth.config_seed(9, d, p))
            true = synth.true_class(d, E)
            sy = torch.tensor(synth.syndromes_of(d, E).view(np.int64), device="cuda")
            dpx = torch.tensor(px, device="cuda")
            lpx, amx = code.decode_xz(dpx, dpx, sy, mld.MLD_FP64)
            nz = torch.tensor(tab.astype(np.float32), device="cuda")
            code.set_svd_cutoff(args.kw_chi_cutoff)
            lead = torch.argmax(lpx, dim=1)
            row = {"d": d, "p": p, "syndromes": Bd,
                   "exact_logical_error_rate": float((amx.cpu().numpy() != true).mean()), "chi": []}
            for chi in args.kw_chi:
                code.decode(nz, sy[:256], chi)                 # warm-up: plan and workspaces
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                lpm, amm = code.decode(nz, sy, chi)
                e1.record()
                torch.cuda.synchronize()
                dt = e0.elapsed_time(e1) / 1e3
                dl = (lpm.gather(1, lead[:, None]) - lpx.gather(1, lead[:, None])).abs().max().item()
                row["chi"].append({"chi": chi, "decisions_differ": int((amm != amx).sum().item()),
                                   "max_abs_dlnZ_leading": dl, "seconds": dt, "syndromes_per_s": Bd / dt,
                                   "p99_abs_dlnZ_leading": (lpm.gather(1, lead[:, None]) - lpx.gather(1, lead[:, None]))
                                   .abs().flatten().quantile(0.99).item(),
                                   "logical_error_rate": float((amm.cpu().numpy() != true).mean())})
            if code.status() != 0:
                raise RuntimeError("device status after the decodes")
            rows.append(row)
        code.close()
    line = {"metric": "decisions of the truncated boundary-MPS decode that differ from exact MLD (Kac-Ward)",
            "workload": "kw-chi", "unit": "syndromes", "data": "synthetic", "svd_cutoff": args.kw_chi_cutoff,
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-sample", type=int, default=4096)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch", type=int, default=B, help="syndromes per GPU per step (default: the "
                    "65536 of the workload; smaller values only for profiling captures)")
    ap.add_argument("--workload", default="metric",
                    choices=["metric", "mixed", "grad", "large", "ler", "dmle", "dem", "point", "kw",
                             "kw-threshold", "kw-chi", "threshold"],
                    help="metric: the headline d=9 line (default); mixed: the 1,048,576-syndrome mixed-d "
                         "graph batch; grad: the adjoint on the d=7 workload; dmle: full-batch noise "
                         "estimation from 1,048,576 unlabelled d=9 syndromes; dem: detector-picture decode of "
                         "a d=9 X/Y/Z mechanism model; large: d=17, 25 at chi 32..128 (truncating); "
                         "ler: logical-error rates of the d/p grid against the oracle; point: one (d, chi, p) "
                         "decode point, FP32 and mixed; kw: the Kac-Ward decode under independent X/Z "
                         "noise against the boundary-MPS decode of the same syndromes; kw-threshold: "
                         "logical-error rates under bit-flip noise around the 10.9% threshold, exact; kw-chi: "
                         "truncated boundary-MPS decisions against exact MLD at d=17, 25; threshold: "
                         "logical-error rates under depolarizing noise around the 18.9% threshold")
    ap.add_argument("--kw-d", type=int, nargs="+", default=[9, 13, 17, 25], help="kw: distances")
    ap.add_argument("--kw-p", type=float, default=0.10, help="kw: X and Z flip rate per qubit")
    ap.add_argument("--kw-batch", type=int, default=0, help="kw: syndromes per decode (0: by d)")
    ap.add_argument("--kw-no-mps", action="store_true", help="kw: skip the boundary-MPS comparison")
    ap.add_argument("--kw-chi", type=int, nargs="+", default=[2, 4, 8, 16, 32], help="kw-chi: bond caps")
    ap.add_argument("--thr-d", type=int, nargs="+", default=[9, 13, 17], help="threshold: distances")
    ap.add_argument("--thr-p", type=float, nargs="+", default=[0.170, 0.175, 0.180, 0.185, 0.190, 0.195],
                    help="threshold: depolarizing rates")
    ap.add_argument("--thr-batch", type=int, default=32768, help="threshold: syndromes per point")
    ap.add_argument("--thr-chi", type=int, default=64, help="threshold: bond cap above d = 13")
    ap.add_argument("--kw-chi-p", type=float, nargs="+", default=[0.05, 0.10], help="kw-chi: X and Z flip rates")
    ap.add_argument("--kw-chi-cutoff", type=float, default=1e-7, help="kw-chi: relative singular-value cutoff")
    ap.add_argument("--kw-threshold-p", type=float, nargs="+",
                    default=[0.095, 0.100, 0.105, 0.110, 0.115, 0.120], help="kw-threshold: bit-flip rates")
    ap.add_argument("--large-batch", type=int, default=16384)
    ap.add_argument("--large-d", type=int, nargs="+", default=[17, 25], help="large: distances")
    ap.add_argument("--large-chi", type=int, nargs="+", default=[32, 64, 128],
                    help="large: bond caps (the comparison columns need 128)")
    ap.add_argument("--large-noise", nargs="+", default=["depolarizing", "biased"], help="large: noise models")
    ap.add_argument("--large-p", type=float, default=0.12, help="large: physical error rate")
    ap.add_argument("--ler-batch", type=int, default=65536)
    ap.add_argument("--point-d", type=int, default=13, help="point: distance")
    ap.add_argument("--point-chi", type=int, default=64, help="point: bond cap")
    ap.add_argument("--point-p", type=float, default=0.10, help="point: depolarizing p")
    ap.add_argument("--point-batch", type=int, default=32768, help="point: syndromes per decode")
    ap.add_argument("--point-exact-kernel", type=int, default=0, choices=[0, 1, 2],
                    help="point, untruncated chi: 0 by d, 1 boundary-MPS kernel, 2 dense-state kernel")
    ap.add_argument("--mixed-total", type=int, default=1 << 20)
    args = ap.parse_args()
    rank, world = _env_int("RANK", 0), _env_int("WORLD_SIZE", 1)
    local = _env_int("LOCAL_RANK", 0)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "mixed":
        return run_mixed(args) if rank == 0 else None
    if args.workload == "grad":
        return run_grad(args) if rank == 0 else None
    if args.workload == "dmle":
        return run_dmle(args) if rank == 0 else None
    if args.workload == "dem":
        return run_dem(args) if rank == 0 else None
    if args.workload == "large":
        return run_large(args) if rank == 0 else None
    if args.workload == "ler":
        return run_ler(args) if rank == 0 else None
    if args.workload == "kw":
        return run_kw(args) if rank == 0 else None
    if args.workload == "kw-threshold":
        return run_kw_threshold(args) if rank == 0 else None
    if args.workload == "kw-chi":
        return run_kw_chi(args) if rank == 0 else None
    if args.workload == "threshold":
        return run_threshold(args) if rank == 0 else None
    if args.workload == "point":
        return run_point(args) if rank == 0 else None

    import torch
    import paper_2605_17230_gb300 as mld
    from paper_2605_17230_gb300 import shard
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    # shard: every rank decodes its own contiguous block of syndromes (weak scaling)
    Bn = args.batch
    noise, syn = workload(Bn, rank * Bn)
    code = mld.Code(D)
    dev = torch.device("cuda", local)
    nz = torch.tensor(noise, device=dev)
    sy = torch.tensor(syn.view(np.int64), device=dev)
    logP = torch.empty((Bn, 4), dtype=torch.float64, device=dev)
    am = torch.empty((Bn,), dtype=torch.uint8, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    prec_mixed = mld.MLD_MIXED_TF32

    def step(prec):
        mld.mld_decode(code.handle, nz, mld.MLD_NOISE_TABLE, sy, Bn, CHI, prec, logP, am, stream.cuda_stream)

    # accuracy of the mixed-precision path against the FP32 path on this batch
    step(mld.MLD_FP32)
    lp32 = logP.clone()
    step(prec_mixed)
    torch.cuda.synchronize()
    dlogp = float((logP - lp32).abs().max().item())
    if code.status() != 0:
        raise RuntimeError("device status after the accuracy pass: " + mld.mld_status_string(code.status()))

    def timed(prec, clocks):
        for _ in range(max(3, args.warmup)):
            step(prec)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with Clocks(local) if clocks else _Null() as clk:
            if dist:
                dist.barrier()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.fill_(float(k))                  # evict L2 between timed steps (outside the events)
                ev[k][0].record(stream)
                step(prec)
                ev[k][1].record(stream)
            torch.cuda.synchronize()
            if dist:
                dist.barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        t_local = shard.max_over_ranks(sum(ms) / 1e3, device=dev)
        st = code.status()
        if st != 0:
            raise RuntimeError("device status: " + mld.mld_status_string(st))
        return t_local, ms, (clk.summary() if clocks else None)

    t32, ms32, _ = timed(mld.MLD_FP32, False)
    value32 = world * Bn * args.steps / t32
    t_max, ms, clocks = timed(prec_mixed, True)
    value = world * Bn * args.steps / t_max
    mixed_ok = dlogp <= 1e-3
    if not mixed_ok:                                   # the metric's bound failed: report the FP32 path
        value, t_max, ms, prec_mixed = value32, t32, ms32, mld.MLD_FP32

    # end-to-end through the host-buffer entry point (pinned host memory)
    h_noise = torch.tensor(noise).pin_memory()
    h_syn = torch.tensor(syn.view(np.int64)).pin_memory()
    h_lp = torch.empty((Bn, 4), dtype=torch.float64).pin_memory()
    h_am = torch.empty((Bn,), dtype=torch.uint8).pin_memory()
    import ctypes

    def e2e_step():
        s = mld.load().mld_decode_host(ctypes.c_void_p(code.handle), ctypes.c_void_p(h_noise.data_ptr()),
                                       mld.MLD_NOISE_TABLE, ctypes.c_void_p(h_syn.data_ptr()), Bn, CHI,
                                       prec_mixed, ctypes.c_void_p(h_lp.data_ptr()),
                                       ctypes.c_void_p(h_am.data_ptr()))
        if s != 0:
            raise RuntimeError("mld_decode_host: " + mld.mld_status_string(s))

    for _ in range(2):
        e2e_step()
    e2e_steps = max(3, args.steps // 2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_dt = time.perf_counter() - t0
    e2e_val = world * Bn * e2e_steps / e2e_dt

    # roofline of the dominant kernel (the fused decode kernel): counted flops
    # of the executed schedule / its CUDA-event time (the argmax kernel is
    # < 1% of the step and is included in the timing), against the FP32 FMA
    # rate measured on this GPU by an FFMA microbenchmark (outside the timed
    # region); the tensor fraction sets the same flops against the dense TF32
    # rate (the measured BF16 cuBLAS peak scaled by the nominal TF32/BF16 ratio)
    flops_per_syn = code.flops(CHI, prec_mixed)
    achieved = Bn * flops_per_syn / (statistics.median(ms) / 1e3) / 1e12
    peak, sms = mld.mld_measure_fp32_peak(2.0)
    peaks = _measured_peaks()
    bf16 = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops")
    traffic = (TRAFFIC_BYTES_PER_SYNDROME[prec_mixed] * Bn
               if kernel_sources_sha() == TRAFFIC_SOURCES_SHA and prec_mixed in TRAFFIC_BYTES_PER_SYNDROME
               else None)
    line = {
        "metric": METRIC, "value": value, "unit": "syndromes/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "tf32x3+f32" if prec_mixed == mld.MLD_MIXED_TF32 else "f32", "data": "synthetic",
        "config": {"workload": f"rotated d={D}, depolarizing p={P}, chi={CHI}, {Bn} syndromes per GPU per step, "
                               f"4 cosets + argmax",
                   "global_batch": Bn * world, "l2": "flushed between timed steps (256 MiB write)",
                   "precision": ("mixed: MPO.MPS data-site products on tensor cores from split TF32 operands "
                                 "(hi.hi + hi.lo + lo.hi), FP32 accumulate; everything else FP32")
                   if prec_mixed == mld.MLD_MIXED_TF32 else "fp32 (mixed path failed the 1e-3 bound)"},
        "fp32": {"value": value32, "ms_per_step": 1e3 * t32 / args.steps},
        "mixed_vs_fp32_max_abs_dlogP": dlogp,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"measured: FFMA microbenchmark on {sms} SMs (mld_measure_fp32_peak, 2 s)",
                     "tensor_frac": (achieved / (bf16 * TF32_PER_BF16)) if bf16 else None,
                     "tensor_peak_source": "measured BF16 cuBLAS peak (sustained) x nominal TF32/BF16 1.1/2.25",
                     "note": "achieved = counted flops of the executed sweep schedule / kernel time; traffic = "
                             "DRAM bytes per launch (ncu capture of 8,192 syndromes scaled by the syndrome "
                             "count; null when the kernel sources differ from the captured ones)"},
        "e2e": {"value": e2e_val, "unit": "syndromes/s", "h2d_bytes_per_step": int(h_noise.numel() * 4 +
                                                                                     h_syn.numel() * 8),
                "d2h_bytes_per_step": int(h_lp.numel() * 8 + h_am.numel())},
        "gpu_launches": args.steps * mld.mld_decode_launches(),
        "clocks": clocks,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
