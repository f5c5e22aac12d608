#!/usr/bin/env python
"""Benchmark: exact polynomial-matrix product over F_p on GB300.

Step = one pmat_mul of 32 x 32 . 32 x 32 polynomial matrices of degree < 4096
modulo a random 60-bit prime drawn from seed 0 (uint64 storage; the library
takes it through 5 NTT primes and CRT): forward transforms, pointwise
products, inverse transforms, recombination.  The same sizes modulo
998244353 (uint32, one NTT prime) are reported under "extra".

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  --impl reference times the CPU oracle (plain C,
OpenMP) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pmat-mul & PM-Basis ms, % of HBM/int8 roofline; TC-batched vs plain NTT"
WORKLOAD = "pmat_mul 32x32 . 32x32, degree < 4096, random 60-bit p (seed 0), uint64"
CONFIG = {"workload": WORKLOAD, "m": 32, "n": 32, "k": 32, "deg_bound": 4096, "p_bits": 60, "seed": 0,
          "crt_primes": 5, "transform_len": 8192}
PAPER_CONTEXT = {"ms": 2000.0, "hardware": "Intel i7-4790, 1 thread, NTL 11.3.1",
                 "workload": "m = 32, degree 4096, random 60-bit prime (product table of Sec. 2)"}
L2_FLUSH_BYTES = 256 << 20
# the pointwise kernel of the tuned form, keyed as in profiles/traffic.json: form 1 runs the
# 4 x 8 thread-tile instance that the committed capture measured; other forms have no entry
PW_KERNEL = {1: ("k_pointwise", "pointwise.cu"), 6: ("k_pointwise<4>", "pointwise.cu"),
             2: ("k_pointwise_tc", "tc_pointwise.cu")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the timings of the drivers (see --extra)")
    ap.add_argument("--extra-only", action="store_true",
                    help="diagnostic: run only the --extra workloads (no headline step) and print their timings")
    ap.add_argument("--extra", default="vandermonde,pm_basis,resultant,batched,inverse,solve,slices,intbasis,linsolve,"
                                         "villard",
                    help="comma-separated subset of vandermonde, pm_basis, resultant, batched, inverse, solve, slices, "
                         "intbasis, linsolve, villard")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers
def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(ms_step: float, world: int) -> float:
    """Whole-job ms per product: every rank computes one product per step (replicas), and the
    step takes the slowest rank's time."""
    return ms_step / world


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def sha(path):
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def traffic_for(kernel: str, src_file: str):
    """dram bytes per launch from the committed ncu summary, if taken on the current kernel source."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t.get(kernel)
        if e and e.get("source_sha") == sha(os.path.join(ROOT, "paper_1905_04356_gb300", "csrc", src_file)):
            return e.get("dram_bytes_per_launch")
    except Exception:
        pass
    return None


def inst_for(kernel: str, src_file: str):
    """warp instructions per launch from the committed ncu summary, if taken on the current kernel source."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
        e = t.get(kernel)
        if e and e.get("source_sha") == sha(os.path.join(ROOT, "paper_1905_04356_gb300", "csrc", src_file)):
            return e.get("inst_executed_per_launch")
    except Exception:
        pass
    return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)
def oracle_sample(W, rows: int):
    """Time the oracle on the first `rows` rows of A (rows x 32 of the 32 x 32 output entries)."""
    import oracle
    A = W["A"][:rows]
    t0 = time.perf_counter()
    oracle.pmat_mul(W["p"], A, W["B"])
    dt = time.perf_counter() - t0
    return dt * 1000.0 * (W["A"].shape[0] / rows), dt, oracle.max_threads()


def cpu_baseline(W, budget_s=15.0):
    ms1, dt1, cores = oracle_sample(W, 1)
    rows = max(1, min(32, int(budget_s / max(dt1, 1e-3))))
    if rows > 1:
        ms, dt, cores = oracle_sample(W, rows)
    else:
        ms, dt = ms1, dt1
    return {"value": round(ms, 1), "unit": "ms", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{rows} of 32 output rows ({rows * 32} of 1024 entries, all 8191 coefficients), "
                      f"{dt:.1f} s of CPU time, scaled to the full product"}


def run_reference(args, rank):
    if rank != 0:
        return
    import synth
    W = synth.product_c2(0)
    for _ in range(args.warmup):
        oracle_sample(W, 1)
    vals, cores = [], 1
    for _ in range(args.steps):
        ms, _, cores = oracle_sample(W, 1)
        vals.append(ms)
    v = statistics.median(vals)
    sample = "1 of 32 output rows (32 of 1024 entries, all coefficients) per step, scaled to the full product"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(v, 2), "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(v, 2), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic", "config": CONFIG,
        "cpu_baseline": {"value": round(v, 2), "unit": "ms", "cores": cores, "cpu_model": cpu_model(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": round(v, 2), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------- other workloads (reported under "extra")
def extra_workloads(ctx, s, which=("vandermonde", "pm_basis", "resultant", "batched", "inverse", "solve", "slices",
                                   "intbasis", "linsolve", "villard"), reps=3):
    """PM-Basis (F 32x16, order 8192, 60-bit p), 512 batched uneven products, resultants
    (deg_x = deg_y = 150, 1 prime and 16 primes), the truncated inverse of a 32x32 matrix of
    degree < 4096 mod x^4096 and the lifted series solution of A v = b mod x^32768 (same A, b of
    degree < 4096; 60-bit p), six high-order lifting slices of the same A^-1, PM-IntBasis (E 32x16
    at 8192 geometric points, 60-bit p), the lifting solver A u = f b (16x16, length 256, 60-bit
    p), the Villard-variant resultant (deg 150 / 150, 1 prime): ms per call, CUDA events on the
    stream."""
    import numpy as np
    import torch
    import synth
    from paper_1905_04356_gb300 import pmat

    def ev_ms(fn, n):
        fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        for _ in range(n):
            fn()
        b.record(s)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    def stage_split(fn, n=3):
        """Per-stage device time of one call (events around each stage on the stream): the
        median over n stage-timed calls, so that one disturbed call does not skew the split;
        with the product work counters of one call."""
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 1)
        ctx.stage_times()
        ctx.work(reset=True)
        runs = []
        for _ in range(n):
            fn()
            runs.append(ctx.stage_times())
        wk = ctx.work(reset=True)
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 0)
        ctx.sync()
        st = {k: statistics.median(r[k][0] for r in runs) for k in runs[0] if runs[0][k][1]}
        return st, {k: v // n for k, v in wk.items()}

    def pm_basis():
        W = synth.pmbasis_c3(0)
        F = pmat.to_device(W["F"])
        run = lambda: pmat.pm_basis(ctx, W["p"], F, W["d"], W["shift"])  # noqa: E731
        out = {"pm_basis_32x16_d8192_ms": round(ev_ms(run, reps), 2)}
        # the threshold tuner on the same shape (seeded pseudo-random input); the call above used T = 32
        T, ns = pmat.tune_basis(ctx, W["p"], 32, 16, W["d"], reps=1)
        out["pm_basis_tuned_threshold"] = {"T": T, "ms": round(ns / 1e6, 2)}
        if T != 32:
            out["pm_basis_32x16_d8192_tuned_T_ms"] = round(ev_ms(run, reps), 2)
        ctx.set_option(pmat.PM_OPT_THRESHOLD, 32)
        st, wk = stage_split(run)
        out["pm_basis_stage_ms"] = {k: round(v, 2) for k, v in st.items()}
        out["pm_basis_leaf_us_per_order_step"] = round(st["leaf"] * 1000 / W["d"], 2)
        # the product work of one call (library counters) over the product stages' time
        prod_ms = sum(st[k] for k in ("fwd_ntt", "pointwise", "inv_ntt", "crt"))
        pk = peaks()
        out["pm_basis_product_work"] = {
            "bytes": wk["bytes"], "pointwise_macs": wk["macs"], "butterflies": wk["butterflies"],
            "product_stage_ms": round(prod_ms, 2),
            "compulsory_GBps": round(wk["bytes"] / (prod_ms * 1e-3) / 1e9, 1),
            "compulsory_frac_hbm": round(wk["bytes"] / (prod_ms * 1e-3) / 1e9 / (pk["hbm_gbs"] if pk else 6800.0), 4),
            "gmacs_per_s": round(wk["macs"] / (prod_ms * 1e-3) / 1e9, 1)}
        return out

    def resultant():
        R = synth.resultant_c5(0, nprimes=16)
        f1, g1 = pmat.to_device(np.stack(R["f"][:1])), pmat.to_device(np.stack(R["g"][:1]))
        f16, g16 = pmat.to_device(np.stack(R["f"])), pmat.to_device(np.stack(R["g"]))
        return {"resultant_150_1prime_ms": round(
                    ev_ms(lambda: pmat.bivariate_resultant(ctx, R["primes"][:1], f1, g1), reps), 2),
                "resultant_150_16primes_ms": round(
                    ev_ms(lambda: pmat.bivariate_resultant(ctx, R["primes"], f16, g16), 2), 2)}

    def batched():
        items = synth.batch_c4(0)
        dev = [(it["p"], pmat.to_device(it["A"]), pmat.to_device(it["B"])) for it in items]
        outs = [torch.empty((it["m"], it["k"], 2 * it["d"] - 1), dtype=dev[i][1].dtype, device="cuda")
                for i, it in enumerate(items)]
        run = lambda: pmat.pmat_mul_batched(ctx, dev, outs)  # noqa: E731
        ms_model = ev_ms(run, 2)
        # autotuned tiles: the tuner times every pointwise form and tile of each product's shape
        # (before the timing; later products of a tuned shape take its choice)
        t0 = time.time()
        forms = {}
        for it in items:
            f = pmat.tune_product(ctx, it["p"], it["A"].dtype.itemsize, it["m"], it["n"], it["k"], it["d"], it["d"],
                                  reps=1)[0]
            forms[f] = forms.get(f, 0) + 1
        tune_s = time.time() - t0
        torch.cuda.synchronize()
        n0 = ctx.launches()
        ms = ev_ms(run, 2)
        out = {"batched_512_ms": round(ms, 2), "batched_512_launches_per_call": (ctx.launches() - n0) // 3,
               "batched_512_untuned_ms": round(ms_model, 2),
               "batched_512_autotune": {"shapes": len(items), "seconds": round(tune_s, 1), "forms_chosen": forms}}
        st, wk = stage_split(lambda: pmat.pmat_mul_batched(ctx, dev, outs))
        out["batched_512_stage_ms"] = {k: round(v, 2) for k, v in st.items()}
        pk = peaks()
        out["batched_512_work"] = {"bytes": wk["bytes"], "pointwise_macs": wk["macs"], "butterflies": wk["butterflies"],
                                   "compulsory_frac_hbm": round(wk["bytes"] / (ms * 1e-3) / 1e9 /
                                                                (pk["hbm_gbs"] if pk else 6800.0), 4),
                                   "gmacs_per_s": round(wk["macs"] / (ms * 1e-3) / 1e9, 1)}
        return out

    def inverse():
        W = synth.inverse_w(0)
        A = pmat.to_device(W["A"])
        X = torch.empty((32, 32, W["t"]), dtype=A.dtype, device="cuda")
        run = lambda: pmat.pmat_inv_trunc(ctx, W["p"], A, W["t"], out=X)  # noqa: E731
        out = {"inv_trunc_32x32_t4096_ms": round(ev_ms(run, reps), 3)}
        out["inv_trunc_stage_ms"] = {k: round(v, 3) for k, v in stage_split(run)[0].items()}
        return out

    def solve():
        W = synth.solve_w(0)
        A, b = pmat.to_device(W["A"]), pmat.to_device(W["b"])
        v = torch.empty((32, 1, W["N"]), dtype=A.dtype, device="cuda")
        run = lambda: pmat.pmat_solve_series(ctx, W["p"], A, b, W["N"], out=v)  # noqa: E731
        out = {"solve_series_32x32_d4096_N32768_ms": round(ev_ms(run, reps), 3)}
        out["solve_series_stage_ms"] = {k: round(v, 3) for k, v in stage_split(run)[0].items()}
        # the same series by high-order lifting (3 slices, 3 levels of 8 residues), the paper's
        # other lifting column
        v2 = torch.empty_like(v)
        run2 = lambda: pmat.pmat_solve_series_hol(ctx, W["p"], A, b, W["N"], out=v2)  # noqa: E731
        out["solve_series_hol_32x32_d4096_N32768_ms"] = round(ev_ms(run2, reps), 3)
        out["solve_series_hol_stage_ms"] = {k: round(v3, 3) for k, v3 in stage_split(run2)[0].items()}
        out["solve_series_hol_equals_dixon"] = bool(torch.equal(v, v2))
        return out

    def slices():
        W = synth.inverse_w(0)
        A = pmat.to_device(W["A"])
        S = torch.empty((6, 32, 32, 2 * 4096 - 1), dtype=A.dtype, device="cuda")
        run = lambda: pmat.pmat_inv_slices(ctx, W["p"], A, 6, out=S)  # noqa: E731
        out = {"inv_slices_32x32_d4096_K6_ms": round(ev_ms(run, reps), 3)}
        ctx.sync()
        return out

    def intbasis():
        W = synth.intbasis_w(0)
        E = pmat.to_device(W["E"])
        m, _, sigma = W["E"].shape
        P = torch.empty((m, m, sigma + 1), dtype=E.dtype, device="cuda")
        run = lambda: pmat.pm_intbasis(ctx, W["p"], E, W["c"], W["q"], W["shift"], out=P)  # noqa: E731
        out = {"pm_intbasis_32x16_s8192_ms": round(ev_ms(run, reps), 2)}
        out["pm_intbasis_stage_ms"] = {k: round(v, 2) for k, v in stage_split(run)[0].items()}
        return out

    def linsolve():
        W = synth.linsolve_w(0)
        A, b = pmat.to_device(W["A"]), pmat.to_device(W["b"])
        run = lambda: pmat.pmat_solve(ctx, W["p"], A, b)  # noqa: E731
        out = {"solve_16x16_d256_ms": round(ev_ms(run, reps), 2)}
        out["solve_stage_ms"] = {k: round(v, 2) for k, v in stage_split(run)[0].items()}
        return out

    def villard():
        R = synth.resultant_c5(0, nprimes=1)
        f1, g1 = pmat.to_device(np.stack(R["f"][:1])), pmat.to_device(np.stack(R["g"][:1]))
        run = lambda: pmat.bivariate_resultant_villard(ctx, R["primes"][:1], f1, g1)  # noqa: E731
        out = {"resultant_villard_150_1prime_ms": round(ev_ms(run, reps), 2)}
        out["resultant_villard_stage_ms"] = {k: round(v, 2) for k, v in stage_split(run)[0].items()}
        return out

    def vandermonde():
        """Products by Vandermonde-matrix evaluation / interpolation (dense tensor-core products
        mod 998244353) next to the NTT path on the same inputs, at the product table's m = 128,
        d = 1024 and m = 512, d = 128 and at 32 x 32, d = 4096; outputs compared; the GEMM
        stages' issued MMA throughput against the fp16 rate measured in this run."""
        res = {}
        peak = pmat.mma_rate(0, 128, 4096)
        for (mm, dd) in ((128, 1024), (512, 128), (32, 4096)):
            g = synth.rng(mm + dd)
            Ah = synth.uniform(g, (mm, mm, dd), synth.P998, np.uint32)
            Bh = synth.uniform(g, (mm, mm, dd), synth.P998, np.uint32)
            A, B = pmat.to_device(Ah), pmat.to_device(Bh)
            del Ah, Bh
            C1 = torch.empty((mm, mm, 2 * dd - 1), dtype=torch.int32, device="cuda")
            C2 = torch.empty_like(C1)
            vd = lambda: pmat.pmat_mul_vdm(ctx, synth.P998, A, B, out=C1)  # noqa: E731
            nt = lambda: pmat.pmat_mul(ctx, synth.P998, A, B, out=C2)     # noqa: E731
            # the NTT path with the CUDA-core pointwise form, then the Vandermonde path with it
            ctx.set_option(pmat.PM_OPT_POINTWISE, 1)
            t_nt = ev_ms(nt, 2)
            stc, _ = stage_split(nt, 2)
            t_vd = ev_ms(vd, 2)
            st, _ = stage_split(vd, 2)
            ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
            L = 1 << max(5, (2 * dd - 2).bit_length())
            nks = lambda K: (K + 15) // 16                                    # noqa: E731
            tiles = lambda M, N: ((M + 127) // 128) * ((N + 31) // 32)       # noqa: E731
            mma = 2 * 128 * 128 * 16 * 4
            e = mm * mm
            eval_fl = 2 * tiles(e, L) * nks(dd) * mma
            interp_fl = tiles(e, 2 * dd - 1) * nks(L) * mma
            torch.cuda.synchronize()
            key = f"m{mm}_d{dd}"
            res[key] = {"ntt_cuda_core_pointwise_ms": round(t_nt, 3), "vdm_ms": round(t_vd, 3),
                        "outputs_equal": bool(torch.equal(C1, C2)),
                        "cuda_core_pointwise_stage_ms": round(stc["pointwise"], 3),
                        "vdm_stage_ms": {k2: round(v, 3) for k2, v in st.items()},
                        "eval_gemm_tflops": round(eval_fl / (st["fwd_ntt"] * 1e-3) / 1e12, 1),
                        "interp_gemm_tflops": round(interp_fl / (st["inv_ntt"] * 1e-3) / 1e12, 1),
                        "eval_tensor_frac": round(eval_fl / (st["fwd_ntt"] * 1e-3) / 1e12 / peak, 4)}
            if mm >= 64:
                # the pointwise stage as dense tensor-core products per point, on the NTT path
                # and on the Vandermonde path (every stage on the tensor cores)
                C3 = torch.empty_like(C1)
                ctx.set_option(pmat.PM_OPT_POINTWISE, 3)
                nt3 = lambda: pmat.pmat_mul(ctx, synth.P998, A, B, out=C3)  # noqa: E731
                t_nt3 = ev_ms(nt3, 2)
                st3, _ = stage_split(nt3, 2)
                t_vd3 = ev_ms(vd, 2)
                ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
                t_auto = ev_ms(nt, 2)
                torch.cuda.synchronize()
                res[key].update({"ntt_tensor_core_pointwise_ms": round(t_nt3, 3), "vdm_tensor_core_pointwise_ms": round(t_vd3, 3),
                                 "tensor_core_pointwise_stage_ms": round(st3["pointwise"], 3),
                                 "pointwise_speedup": round(stc["pointwise"] / st3["pointwise"], 3),
                                 "auto_mode_ms": round(t_auto, 3),
                                 "tensor_core_outputs_equal": bool(torch.equal(C3, C2) and torch.equal(C1, C2))})
                del C3
            del A, B, C1, C2
            torch.cuda.empty_cache()
        # the dense tensor-core pointwise form at m = 512, d = 128 modulo a 60-bit prime (5 CRT primes)
        g = synth.rng(512128)
        p60 = synth.random_prime(g, 60)
        A = pmat.to_device(synth.uniform(g, (512, 512, 128), p60, np.uint64))
        B = pmat.to_device(synth.uniform(g, (512, 512, 128), p60, np.uint64))
        C1 = torch.empty((512, 512, 255), dtype=torch.int64, device="cuda")
        C2 = torch.empty_like(C1)
        ctx.set_option(pmat.PM_OPT_POINTWISE, 1)
        t_cc = ev_ms(lambda: pmat.pmat_mul(ctx, p60, A, B, out=C1), 2)
        st_cc, _ = stage_split(lambda: pmat.pmat_mul(ctx, p60, A, B, out=C1), 2)
        ctx.set_option(pmat.PM_OPT_POINTWISE, 3)
        t_tc = ev_ms(lambda: pmat.pmat_mul(ctx, p60, A, B, out=C2), 2)
        st_tc, _ = stage_split(lambda: pmat.pmat_mul(ctx, p60, A, B, out=C2), 2)
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
        torch.cuda.synchronize()
        p60_res = {"ntt_cuda_core_pointwise_ms": round(t_cc, 3), "ntt_tensor_core_pointwise_ms": round(t_tc, 3),
                   "cuda_core_pointwise_stage_ms": round(st_cc["pointwise"], 3),
                   "tensor_core_pointwise_stage_ms": round(st_tc["pointwise"], 3),
                   "pointwise_speedup": round(st_cc["pointwise"] / st_tc["pointwise"], 3),
                   "outputs_equal": bool(torch.equal(C1, C2))}
        del A, B, C1, C2
        torch.cuda.empty_cache()
        return {"vandermonde_p998": res, "dense_tensor_core_pointwise_p60_m512_d128": p60_res,
                "mma_peak_tflops_n128": round(peak, 1)}

    out = {}
    with torch.cuda.stream(s):
        for name, fn in (("vandermonde", vandermonde), ("pm_basis", pm_basis), ("resultant", resultant), ("batched", batched),
                         ("inverse", inverse), ("solve", solve), ("slices", slices), ("intbasis", intbasis),
                         ("linsolve", linsolve), ("villard", villard)):
            if name in which:
                out.update(fn())
    return out


# ---------------------------------------------------------------- GPU arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import numpy as np
    import torch
    import synth
    from paper_1905_04356_gb300 import Context, build, pmat

    torch.cuda.set_device(local)
    if args.extra_only:
        build.build()
        s0 = torch.cuda.Stream()
        c0 = Context(local, stream=s0)
        print(json.dumps({"extra_only": extra_workloads(c0, s0, tuple(args.extra.split(",")))}), flush=True)
        c0.close()
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()

    W = synth.product_c2(0)
    W998 = synth.product_c2(0, ntt_prime=True)
    p, Ah, Bh = W["p"], W["A"], W["B"]
    m, n, dA = Ah.shape
    k, dB = Bh.shape[1], Bh.shape[2]
    lenC = dA + dB - 1
    s = torch.cuda.Stream()
    ctx = Context(local, stream=s)
    with torch.cuda.stream(s):
        A, B = pmat.to_device(Ah), pmat.to_device(Bh)
        Cd = torch.empty((m, k, lenC), dtype=torch.int64, device="cuda")
        A2, B2 = pmat.to_device(W998["A"]), pmat.to_device(W998["B"])
        C2 = torch.empty((m, k, lenC), dtype=torch.int32, device="cuda")
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()

    def step(i):
        pmat.pmat_mul(ctx, p, A, B, out=Cd)

    def timed(fn, K, events=True):
        ts = []
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        for i in range(K):
            flush.add_(1)                      # L2 flush, outside the per-step events
            ev[i][0].record(s)
            fn(i)
            ev[i][1].record(s)
        torch.cuda.synchronize()
        for a, b in ev:
            ts.append(a.elapsed_time(b))
        return ts

    with torch.cuda.stream(s):
        # the autotuner picks the pointwise form and block tile of this shape (before any timing)
        tuned = pmat.tune_product(ctx, p, 8, m, n, k, dA, dB, reps=3)
        for i in range(args.warmup):
            step(i)
        torch.cuda.synchronize()
        # ---- timed region
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(local)
        n0 = ctx.launches()
        t_wall = time.perf_counter()
        ts = timed(step, args.steps)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
        launches = ctx.launches() - n0
        if dist:
            dist.barrier()
        ck = clocks.stop()
        ms_step = max_over_ranks(sum(ts) / len(ts), dist, "cuda")

        # ---- per-stage times (events on the launching stream) for the roofline
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 1)
        ctx.stage_times()
        timed(step, max(5, args.steps // 2))
        st = ctx.stage_times()
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 0)

        # ---- the same step captured once in a CUDA graph and replayed (L2 flushed between
        #      replays, outside the events)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            pmat.pmat_mul(ctx, p, A, B, out=Cd)
        for _ in range(3):
            graph.replay()
        ts_graph = timed(lambda i: graph.replay(), args.steps)

        # ---- the same step with the tensor-core pointwise form (8-bit limbs in bf16 on tcgen05,
        #      fp32 accumulation in tensor memory, limb recombination on the CUDA cores): its time,
        #      its pointwise stage, and exact equality with the CUDA-core output
        Ctc = torch.empty_like(Cd)
        ctx.set_option(pmat.PM_OPT_POINTWISE, 2)
        for _ in range(3):
            pmat.pmat_mul(ctx, p, A, B, out=Ctc)
        ts_tc = timed(lambda i: pmat.pmat_mul(ctx, p, A, B, out=Ctc), args.steps)
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 1)
        ctx.stage_times()
        timed(lambda i: pmat.pmat_mul(ctx, p, A, B, out=Ctc), 5)
        st_tc = ctx.stage_times()
        ctx.set_option(pmat.PM_OPT_STAGE_TIMING, 0)
        ctx.set_option(pmat.PM_OPT_POINTWISE, 0)
        pmat.pmat_mul(ctx, p, A, B, out=Cd)
        torch.cuda.synchronize()
        tc_equal = bool(torch.equal(Ctc, Cd))

        # ---- same sizes modulo 998244353 (one NTT prime, uint32)
        for _ in range(3):
            pmat.pmat_mul(ctx, W998["p"], A2, B2, out=C2)
        ts998 = timed(lambda i: pmat.pmat_mul(ctx, W998["p"], A2, B2, out=C2), args.steps)

        # ---- the 4x4 . 4x4, length-256 product mod 998244353 (latency-bound: reported in us)
        W1 = synth.product_c1(0)
        A1, B1 = pmat.to_device(W1["A"]), pmat.to_device(W1["B"])
        C1 = torch.empty((4, 4, 511), dtype=A1.dtype, device="cuda")
        for _ in range(3):
            pmat.pmat_mul(ctx, W1["p"], A1, B1, out=C1)
        ts_c1 = timed(lambda i: pmat.pmat_mul(ctx, W1["p"], A1, B1, out=C1), args.steps)

        # ---- end to end: pmat_mul_host on pinned host buffers, every host<->device copy
        #      inside the timed region (overlapped with the stages by the library)
        Ap = torch.from_numpy(Ah.view(np.int64)).pin_memory()
        Bp = torch.from_numpy(Bh.view(np.int64)).pin_memory()
        Cp = torch.empty((m, k, lenC), dtype=torch.int64).pin_memory()

        def e2e_step(i):
            pmat.pmat_mul_host(ctx, p, Ap, Bp, out=Cp)
            ctx.host_join()                     # the step's download inside its own events

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize()
        ts_lat = timed(e2e_step, args.steps)   # one call at a time: latency
        # K calls back to back (each call's download overlaps the next call's upload and work),
        # joined once: every copy of every step is inside the events
        ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ea.record(s)
        for i in range(args.steps):
            pmat.pmat_mul_host(ctx, p, Ap, Bp, out=Cp)
        ctx.host_join()
        eb.record(s)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(ea.elapsed_time(eb) / args.steps, dist, "cuda")
        e2e_latency_ms = max_over_ranks(sum(ts_lat) / len(ts_lat), dist, "cuda")
        h2d = Ah.nbytes + Bh.nbytes
        d2h = m * k * lenC * 8

    # ---- roofline of the dominant kernel.  Algorithmic bytes = the product's compulsory I/O (A and
    #      B read once, C written once): the transform-domain intermediates are the method's own
    #      choice, so a kernel's staged bytes (its own reads and writes of them) are a diagnostic.
    K, L = 5, 8192
    eA, eB, eC = m * n, n * k, m * k
    pw_kernel, pw_src = PW_KERNEL.get(int(tuned[0]), ("pointwise form %d" % int(tuned[0]), "pointwise.cu"))
    compulsory = (eA * dA + eB * dB) * 8 + eC * lenC * 8
    staged = {   # bytes each stage's kernel reads + writes (one launch per stage here)
        "fwd_ntt": (eA * dA + eB * dB) * 8 + K * (eA + eB) * L * 4,
        "pointwise": K * (eA + eB) * L * 4 + K * eC * L * 4,
        "inv_ntt": K * eC * L * 4 + K * eC * lenC * 4,
        "crt": K * eC * lenC * 4 + eC * lenC * 8,
    }
    kname = {"fwd_ntt": ("k_ntt_fwd_block", "ntt.cu"), "pointwise": (pw_kernel, pw_src),
             "inv_ntt": ("k_ntt_inv_block", "ntt.cu"), "crt": ("k_crt", "pointwise.cu")}
    stages = {k2: v for k2, v in st.items() if v[1] > 0}
    dom = max(stages, key=lambda x: stages[x][0])
    dom_ms = stages[dom][0] / stages[dom][1]
    pk = peaks()
    peak = pk["hbm_gbs"] if pk else 6800.0
    achieved = compulsory / (dom_ms * 1e-3) / 1e9
    staged_gbs = staged[dom] / (dom_ms * 1e-3) / 1e9
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    clk = ck.get("sm_mhz") or (pk["sm_max_mhz"] if pk else 2070.0)
    issue_peak = sms * 4 * clk * 1e6                 # warp instructions per second (one per SMSP per clock)
    inst = inst_for(*kname[dom])
    roof = {"bound": "hbm", "kernel": kname[dom][0], "achieved": round(achieved, 1), "peak": peak,
            "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": traffic_for(*kname[dom]),
            "algorithmic_bytes_per_launch": compulsory,
            "algorithmic_bytes": "compulsory I/O of the product: A and B read once, C written once",
            "launch_ms": round(dom_ms, 4),
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if pk else "fallback",
            "staged_bytes_per_launch": staged[dom], "staged_GBps": round(staged_gbs, 1),
            "staged_frac": round(staged_gbs / peak, 4),
            "issue": {"warp_instructions_per_launch": inst, "sms": sms, "sm_mhz": clk,
                      "peak_warp_instructions_per_s": issue_peak,
                      "frac": round(inst / (dom_ms * 1e-3) / issue_peak, 4) if inst else None,
                      "source": "instruction count from the committed ncu summary of the same kernel source, "
                                "time from this run's CUDA events"}}
    def tc_report(ts_tc, st_tc, st_cc):
        """The tensor-core pointwise form on the same step: its pointwise stage against the
        CUDA-core one, and its tensor throughput against the measured fp16 MMA rate.  Issued MMA
        flops count every 128 x 128 x 16 instruction (four points share the 128 rows, one point
        per lane quarter); useful flops count the 16 digit products of every output."""
        tc_pw = st_tc["pointwise"][0] / max(1, st_tc["pointwise"][1])
        cc_pw = st_cc["pointwise"][0] / max(1, st_cc["pointwise"][1])
        ksteps = (n + 15) // 16
        issued = K * (L // 4) * 4 * 4 * ksteps * 2 * 128 * 128 * 16
        useful = K * L * 16 * m * n * k * 2
        peak_n128 = pmat.mma_rate(local, 128, 4096)
        peak_n256 = pmat.mma_rate(local, 256, 4096)
        tf = issued / (tc_pw * 1e-3) / 1e12
        return {"step_ms": round(sum(ts_tc) / len(ts_tc), 4), "pointwise_ms": round(tc_pw, 4),
                "cuda_core_pointwise_ms": round(cc_pw, 4), "speedup": round(cc_pw / tc_pw, 3),
                "outputs_equal": tc_equal, "mma_issued_tflops": round(tf, 1),
                "mma_useful_tflops": round(useful / (tc_pw * 1e-3) / 1e12, 1),
                "mma_peak_tflops_n128": round(peak_n128, 1), "mma_peak_tflops_n256": round(peak_n256, 1),
                "tensor_frac": round(tf / peak_n128, 4),
                "peak_source": "measured in this run: pm_mma_rate, dense tcgen05.mma kind::f16 of 128 x N x 16",
                "dtype": "fp16 digits (balanced radix 256), fp32 accumulation"}

    value = job_value(ms_step, world)
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": dict(CONFIG, l2="256 MiB buffer written between steps, outside the per-step events",
                       replicas=world),
        "roofline": roof,
        "e2e": {"value": round(job_value(e2e_ms, world), 4), "unit": "ms", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": ck,
        "extra": {
            "stage_ms_per_step": {k2: round(v[0] / max(5, args.steps // 2), 4) for k2, v in stages.items()},
            "step_compulsory_bytes": compulsory,
            "step_compulsory_GBps": round(compulsory / (ms_step * 1e-3) / 1e9, 1),
            "step_compulsory_frac_hbm": round(compulsory / (ms_step * 1e-3) / 1e9 / peak, 4),
            "graph_replay_ms_per_step": round(sum(ts_graph) / len(ts_graph), 4),
            "e2e_single_call_latency_ms": round(e2e_latency_ms, 4),
            "tensor_core_vs_cuda_core": tc_report(ts_tc, st_tc, stages),
            "autotune": {"form": {1: "CUDA-core block tile", 2: "tensor-core digits, four points per MMA",
                                   3: "streaming", 4: "matrix-vector",
                                   5: "tensor-core dense products per point",
                                   6: "CUDA-core block tile, 4 x 4 thread tiles"}.get(tuned[0], tuned[0]),
                         "block_tile": [tuned[1], tuned[2]], "pointwise_us": round(tuned[3] / 1000, 1),
                         "candidates": tuned[4]},
            "c2_p998_ms": round(sum(ts998) / len(ts998), 4),
            "c1_4x4_d256_p998_us": round(1000 * sum(ts_c1) / len(ts_c1), 1),
            "wall_s_timed_region": round(t_wall, 3),
            "paper_context": PAPER_CONTEXT,
        },
    }
    if not args.no_extra:
        out["extra"].update(extra_workloads(ctx, s, tuple(args.extra.split(","))))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(W)
    if rank == 0:
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
