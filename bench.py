"""Benchmark of the CASCI hot path on CAS(14,14) (7 alpha + 7 beta electrons in
14 orbitals, 11,778,624 determinants; seeded synthetic integrals, 28 factors,
seed 2).

One step = one Davidson-Liu solve of the lowest root from the unit-vector
guess to an FP64 residual that puts the energy within 1e-8 Eh (tol 1e-5,
energy error ~ |r|^2 / gap), followed by the spin-free 1- and 2-RDMs of the
root.  ``value`` is the sigma throughput of the whole step: determinants x
sigma vectors built during the step / step time (det/s).

Contract: prints one JSON line (rank 0).  --impl reference times the CPU
oracle (the plain Slater-Condon program under oracle/) on a bounded sample of
output determinants of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth_inputs as si  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0
# FP64 FMA pipe: nominal GB300 FP64 rate (1.25 TFLOP/s = 152 SMs x 2 DFMA/clk x 2 flop x ~2.06 GHz)
FP64_PEAK_TFLOPS = 1.25

WORKLOADS = {
    "cas1414": si.CAS1414,
    "cas1212": si.CAS1212,
    "cas88": si.CAS88,
}
METRIC = "CASCI H*C det/s and Davidson time-to-1e-8 Eh, CAS(14,14), mixed vs FP64, 1 GB300"


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p.get("hbm_gbs", FALLBACK_HBM_GBS), p.get("bf16_tflops", FALLBACK_BF16_TFLOPS), \
            p.get("bf16_tflops_sustained", FALLBACK_BF16_TFLOPS), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, FALLBACK_BF16_TFLOPS, 1700.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ oracle arm
def oracle_sigma_rate(cfg, seconds=10.0, seed=21):
    """Oracle direct sigma on a bounded random sample of output determinants;
    returns (det/s, rows, wall s, threads)."""
    import oracle
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    Na, Nb = si.n_strings(n, na), si.n_strings(n, nb)
    C = si.random_vectors(1, Na, Nb, seed=7).reshape(1, -1)
    rng = np.random.default_rng(seed)
    # calibrate: per-call set-up cost + per-row cost from two probe sizes
    t = []
    for m in (256, 4096):
        probe = rng.integers(0, Na * Nb, size=m)
        t0 = time.perf_counter()
        oracle.sigma(n, na, nb, h, eri, C, rows=probe)
        t.append(time.perf_counter() - t0)
    per_row = max((t[1] - t[0]) / 3840.0, t[1] / 4096.0 * 0.5, 1e-7)
    nrows = int(max(4096, min(5_000_000, max(seconds - t[0], 0.5) / per_row)))
    rows = rng.integers(0, Na * Nb, size=nrows)
    t0 = time.perf_counter()
    oracle.sigma(n, na, nb, h, eri, C, rows=rows)
    dt = time.perf_counter() - t0
    return nrows / dt, nrows, dt, oracle.num_threads()


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sigma_rate(cfg, seconds=2.0)
    rates = []
    t_all = 0.0
    nthreads = 1
    rows_tot = 0
    for _ in range(args.steps):
        r, rows, dt, nthreads = oracle_sigma_rate(cfg, seconds=args.ref_seconds)
        rates.append(r)
        t_all += dt
        rows_tot += rows
    value = rows_tot / t_all
    sample = (f"oracle direct sigma on {rows_tot} random output determinants of {args.workload} "
              f"over {args.steps} steps")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "det/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_all / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": args.workload, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": "det/s", "cores": nthreads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "det/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


# ------------------------------------------------------------------ GPU arm
def kernel_flops(ctx_info, name, nvec):
    """Algorithmic FLOPs of one sigma vector through kernel `name`."""
    nd, nka, nkb, nnz_a, nnz_b = ctx_info
    if name == "ab_fp64":
        return 2.0 * nd * nka * nkb * nvec
    if name == "ss_spmm":
        return 2.0 * nd * (nnz_a + nnz_b) / 2.0 * nvec
    return None


def run_ours(args):
    import torch
    import paper_2405_10197_gb300 as fg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    cfg = WORKLOADS[args.workload]
    n, na, nb = cfg["norb"], cfg["nalpha"], cfg["nbeta"]
    h, eri = si.integrals(n, cfg["n_l"], cfg["seed"])
    mode = {"fp64": fg.FORTE_FP64, "tf32": fg.FORTE_TF32, "bf16x2": fg.FORTE_BF16X2}[args.precision]
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    prob = fg.CASProblem(n, na, nb, h, eri, precision=mode, stream=stream)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    nd = prob.ndet
    nroots = 1
    tol = args.tol

    g1 = torch.empty(n, n, dtype=torch.float64, device="cuda")
    g2 = torch.empty((n,) * 4, dtype=torch.float64, device="cuda")
    root = torch.empty(nroots, prob.na, prob.nb, dtype=torch.float64, device="cuda")

    def step():
        fg.forte_davidson(prob.ctx, nroots, tol, allow_not_converged=True)
        fg.forte_get_roots(prob.ctx, nroots, root)
        fg.forte_rdms(prob.ctx, root[0], g1, g2, n)

    # reference energy (FP64, tight), outside every timed region
    E_ref = None
    if args.ref_energy:
        fg.forte_set_precision(prob.ctx, fg.FORTE_FP64)
        fg.forte_davidson(prob.ctx, 1, 1e-8, allow_not_converged=True)
        E_ref = float(fg.forte_get_roots(prob.ctx, 1)[0][0])
        fg.forte_set_precision(prob.ctx, mode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    s0 = fg.forte_get_counters(prob.ctx)
    clocks = ClockSampler(dev)
    clocks.start()
    fg.forte_profile_enable(prob.ctx, 1)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dav_ms = []
    energies = []
    ev0.record(stream)
    for _ in range(args.steps):
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        fg.forte_davidson(prob.ctx, nroots, tol, allow_not_converged=True)
        d1.record(stream)
        E, rn, it = fg.forte_get_roots(prob.ctx, nroots, root)
        fg.forte_rdms(prob.ctx, root[0], g1, g2, n)
        energies.append(float(E[0]))
        dav_ms.append((d0, d1, it, float(rn[0])))
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    fg.forte_profile_enable(prob.ctx, 0)
    t_ms = ev0.elapsed_time(ev1)
    s1 = fg.forte_get_counters(prob.ctx)
    nsig64, nsigm = s1[0] - s0[0], s1[1] - s0[1]
    prof = fg.profile_table(prob.ctx)
    launches = sum(v[0] for v in prof.values())

    if dist:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
    units = nd * (nsig64 + nsigm) * world
    value = units / (t_ms / 1000.0)

    # roofline of the dominant kernel
    hbm, bf16, bf16s, peak_src = peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    dom_name, (dom_n, dom_ms) = dom
    nka = prob.norb * 0  # placeholder replaced below
    nk = lambda ne: ne * (n - ne) + ne  # noqa: E731
    info = (nd, nk(na), nk(nb), None, None)
    roof = None
    if dom_name == "ab_fp64":
        flops = 2.0 * nd * nk(na) * nk(nb) * nsig64
        ach = flops / (dom_ms / 1000.0) / 1e12
        roof = {"kernel": dom_name, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "peak_source": "nominal FP64 pipe rate (152 SMs x 2 DFMA/clk x 2 x ~2.06 GHz)",
                "launches": dom_n, "avg_ms": dom_ms / max(dom_n, 1)}
    else:
        roof = {"kernel": dom_name, "bound": None, "achieved": None, "peak": None, "unit": None,
                "frac": None, "traffic": None, "launches": dom_n, "avg_ms": dom_ms / max(dom_n, 1)}

    dav_times = [a.elapsed_time(b) for (a, b, _, _) in dav_ms]
    dav_iters = [x[2] for x in dav_ms]
    out = {
        "metric": METRIC, "value": value, "unit": "det/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if mode == fg.FORTE_FP64 else args.precision,
        "data": "synthetic",
        "config": {"workload": f"CAS(14,14) 7a7b 11,778,624 dets seed 2 (n_L 28)"
                   if args.workload == "cas1414" else args.workload,
                   "precision": args.precision, "nroots": nroots, "tol": tol,
                   "step": "Davidson to tol + 1-/2-RDM", "l2": "inputs larger than L2 (94 MB vectors, >2 GB subspace)",
                   "parallelism": f"replicas{world}"},
        "davidson": {"ms": dav_times, "iterations": dav_iters, "energy": energies,
                     "E_ref_fp64": E_ref,
                     "energy_err": [abs(e - E_ref) for e in energies] if E_ref is not None else None,
                     "sigma_vectors_fp64": nsig64, "sigma_vectors_mixed": nsigm},
        "setup_s": t_setup,
        "roofline": roof,
        "kernels": {k: {"launches": v[0], "ms": v[1]} for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "gpu_launches": launches,
        "clocks": clk,
    }

    # end to end through the C ABI with host buffers
    if args.e2e_steps > 0:
        import paper_2405_10197_gb300 as fg2
        h_pin = torch.tensor(h).pin_memory()
        eri_pin = torch.tensor(eri).pin_memory()
        E_host = np.zeros(1)
        g1_host = torch.empty(n, n, dtype=torch.float64).pin_memory()
        g2_host = torch.empty((n,) * 4, dtype=torch.float64).pin_memory()
        e2e_t = []
        e2e_units = 0
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = fg2.forte_cas_create(n, na, nb, h_pin.numpy(), eri_pin.numpy())
            fg2.forte_set_stream(ctx, stream)
            fg2.forte_set_precision(ctx, mode)
            fg2.forte_davidson(ctx, nroots, tol, allow_not_converged=True)
            E_host[:], _, _ = fg2.forte_get_roots(ctx, nroots, root)
            fg2.forte_rdms(ctx, root[0], g1, g2, n)
            g1_host.copy_(g1, non_blocking=True)
            g2_host.copy_(g2, non_blocking=True)
            torch.cuda.synchronize()
            c = fg2.forte_get_counters(ctx)
            fg2.forte_destroy(ctx)
            e2e_t.append(time.perf_counter() - t0)
            e2e_units += nd * (c[0] + c[1])
        out["e2e"] = {"value": e2e_units * world / sum(e2e_t), "unit": "det/s",
                      "h2d_bytes_per_step": 8 * (n * n + n ** 4),
                      "d2h_bytes_per_step": 8 * (nroots + n * n + n ** 4),
                      "steps": args.e2e_steps, "s_per_step": sum(e2e_t) / len(e2e_t),
                      "includes": "forte_cas_create (string tables, CSR, H_II) + Davidson + RDMs + D2H"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, rows, dt, thr = oracle_sigma_rate(cfg, seconds=args.ref_seconds)
        out["cpu_baseline"] = {"value": r, "unit": "det/s", "cores": thr, "kind": "oracle",
                               "sample": f"oracle direct sigma on {rows} random output determinants "
                                         f"({dt:.1f} s)"}
    if rank == 0:
        print(json.dumps(out))
    prob.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cas1414")
    ap.add_argument("--precision", choices=["fp64", "tf32", "bf16x2"], default="fp64")
    ap.add_argument("--tol", type=float, default=1e-5)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--ref-seconds", type=float, default=10.0)
    ap.add_argument("--ref-energy", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
