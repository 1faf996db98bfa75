#!/usr/bin/env python
"""Throughput benchmark of the density-matrix solve D = f(Hp) on GB300.

Default workload (one GPU): the single gapped zero-temperature solve, n=4096,
N_e=3500, occupied eigenvalues uniform in [-3, -0.01] Ha, empty in
[0.01, 1.0] Ha, Hp = Q diag(lambda) Q^T with Q from QR of a seeded Gaussian,
mixed precision (split-FP16 tensor-core products, FP64 polish).  One "step" is
one complete solve (bounds, X0, every expansion product, output, tr(Hp D)).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  `value` is solves/s with Hp and D resident in
HBM; `e2e` is the same through the C ABI with pinned HOST buffers (Hp copied
in and D copied out inside the timed region).  With N > 1 (torchrun), every
rank solves its own independent problems (replicas; no collective on the data
path) and `value` is the total over ranks.  `--impl reference` times the CPU
oracle (FP64 SP2 on the host cores) on a bounded sample of the same workload.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import hp_synth  # noqa: E402

METRIC = "fermi_expansion_solves_per_s"
UNIT = "solves/s"


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


WORKLOADS = {
    "gapped_n4096": dict(make=lambda: hp_synth.workload_n4096(), precision="mixed"),
    "gapped_n256_fp64": dict(make=lambda: hp_synth.workload_n256(), precision="fp64"),
    # larger single solves (generated on the GPU: the CPU QR would take minutes)
    "gapped_n8192": dict(make=lambda: hp_synth.gapped(8192, 6963, (-3.0, -0.01), (0.01, 1.0), 1005,
                                                        device="cuda", name="gapped_n8192"),
                         precision="mixed"),
    "gapped_n16384": dict(make=lambda: hp_synth.gapped(16384, 13926, (-3.0, -0.01), (0.01, 1.0), 1004,
                                                         device="cuda", name="gapped_n16384"),
                          precision="mixed"),
    "fermi_n16384": dict(make=lambda: hp_synth.workload_n16384_ft(device="cuda"), precision="mixed"),
    # the paper's own synthetic Hamiltonian (Sec. IV), N_e = 0.9 n: a continuous band, gap ~1.4/n
    "paper_matrix_n8192": dict(make=lambda: hp_synth.paper_matrix(8192, device="cuda"), precision="mixed"),
    # many problems per step (see bench_batch / bench_serve)
    "ragged_batch64": dict(make=None, precision="mixed"),
    "serve_poisson": dict(make=None, precision="mixed"),
}


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms."""

    def __init__(self, device):
        self.device = device
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4)
                          if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def sp2_products_on_spectrum(lam, emin, emax, ne, tol):
    """Number of SP2 products the plain FP64 recursion takes on this Hp: the
    branch rule only sees traces, so the scalar recursion on the exact
    eigenvalues reproduces the matrix recursion's decisions."""
    x = (emax - lam) / (emax - emin)
    t1 = x.sum()
    for it in range(1, 400):
        t2 = float(np.dot(x, x))
        x = x * x if abs(t2 - ne) <= abs(2 * t1 - t2 - ne) else 2 * x - x * x
        t1n = x.sum()
        if abs(t1n - t1) <= tol * ne and abs(t1n - float(np.dot(x, x))) <= 1e-9:
            return it
        t1 = t1n
    return 400


def cpu_oracle_sample(p, products_per_solve, max_seconds=20.0):
    """Time FP64 SP2 products of the CPU oracle on this workload; extrapolate
    to a full solve.  Returns (solves/s, threads, sample description)."""
    import oracle
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    t0 = time.perf_counter()
    oracle.sp2(p.H, p.ne, tol=1e-300, max_iter=1)
    per = time.perf_counter() - t0
    k = 1
    if per * 2 < max_seconds:
        t0 = time.perf_counter()
        oracle.sp2(p.H, p.ne, tol=1e-300, max_iter=2)
        per = (time.perf_counter() - t0) / 2
        k = 2
    solve_s = per * products_per_solve
    return (1.0 / solve_s, threads,
            "%d FP64 SP2 product(s) of the n=%d workload on %d host threads, %.2f s each; "
            "solve = %d products (scalar SP2 count on the exact spectrum)"
            % (k, p.n, threads, per, products_per_solve))


def reference_arm(args, p, wl_name):
    """--impl reference: the oracle on the host cores, bounded sample per step."""
    import oracle
    lo, hi = oracle.gershgorin(p.H)
    prods = sp2_products_on_spectrum(p.lam, lo, hi, p.ne, 5e-8)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    for _ in range(args.warmup):
        oracle.sp2(p.H, p.ne, tol=1e-300, max_iter=1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sp2(p.H, p.ne, tol=1e-300, max_iter=1)
        times.append(time.perf_counter() - t0)
    per = statistics.mean(times)
    value = 1.0 / (per * prods)
    sample = ("each step = 1 FP64 SP2 product of the CPU oracle (n=%d, %d threads); "
              "solve = %d products" % (p.n, threads, prods))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": wl_name, "n": p.n, "n_e": p.ne, "kT": 0.0,
                                             "parallelism": "replicas" if args.gpus > 1 else "single"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def traffic_record(kernel_name, src_file):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel's
    source has not changed since it was measured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path)).get(kernel_name)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    h = hashlib.sha256(open(os.path.join(ROOT, "paper_2301_04642_gb300", "csrc", src_file), "rb")
                       .read()).hexdigest()
    return rec.get("bytes_per_launch") if rec.get("src_sha256") == h else None


def job_rate(torch, dist, device, steps, t_ms):
    """Whole-job solves/s of the replicas: every rank solved `steps` problems
    and the job lasted as long as its slowest rank (the maximum over ranks of
    the timed region).  Returns (rate, slowest t_ms)."""
    world = 1
    if dist is not None:
        tt = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms = float(tt.item())
        world = dist.get_world_size()
    return world * steps / (t_ms / 1e3), t_ms


def reference_occupations(lam, ne, kT):
    """Occupations of the constructed spectrum: the N_e lowest states at zero
    temperature, Fermi-Dirac with mu from bisection on sum f = N_e otherwise."""
    import numpy as np
    lam = np.asarray(lam, dtype=np.float64)
    if kT == 0.0:
        return (np.arange(lam.size) < int(ne)).astype(np.float64)
    lo, hi = lam.min() - 40 * kT, lam.max() + 40 * kT
    for _ in range(200):
        mu = 0.5 * (lo + hi)
        f = 0.5 * (1.0 - np.tanh((lam - mu) / (2.0 * kT)))
        if f.sum() > ne:
            hi = mu
        else:
            lo = mu
    return 0.5 * (1.0 - np.tanh((lam - 0.5 * (lo + hi)) / (2.0 * kT)))


def probe_errors(torch, D, Q, lam, f, ne, kT, res, nprobe=4, seed=7):
    """Error of a solve against the constructed D_ref = Q diag(f) Q^T, on this
    GPU in FP64: ||D - D_ref||_F / sqrt(N_e) and ||D^2 - D||_F estimated with
    Gaussian probes (E ||A v||^2 = ||A||_F^2), and |E_band - sum f lambda| / N_e."""
    import numpy as np
    dev = D.device
    Qd = Q.to(dev, torch.float64) if torch.is_tensor(Q) else torch.from_numpy(np.asarray(Q)).to(dev)
    fd = torch.from_numpy(np.asarray(f, dtype=np.float64)).to(dev)
    g = torch.Generator(device=dev).manual_seed(seed)
    V = torch.randn(D.shape[0], nprobe, dtype=torch.float64, device=dev, generator=g)
    DV = D @ V
    err = DV - Qd @ (fd[:, None] * (Qd.T @ V))
    out = {"eps1_probe": float(torch.sqrt((err ** 2).sum() / nprobe)) / math.sqrt(ne),
           "e_err_per_electron": abs(res["e_band"] - float(np.dot(np.asarray(f), np.asarray(lam)))) / ne}
    if kT == 0.0:
        out["idem_probe"] = float(torch.sqrt(((D @ DV - DV) ** 2).sum() / nprobe))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gapped_n4096", choices=sorted(WORKLOADS))
    ap.add_argument("--no-baselines", action="store_true")
    ap.add_argument("--precision", default=None, choices=["mixed", "try_fp16", "fp32", "fp64"],
                    help="override the workload's precision schedule")
    ap.add_argument("--tiles", default="auto", choices=["auto", "256", "128"],
                    help="tensor-core tile width: autotuned per size (untimed, before the warm-up) or fixed")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    wl = WORKLOADS[args.workload]
    if args.precision:
        wl = dict(wl, precision=args.precision)

    if args.impl == "reference":
        if rank != 0:
            return
        if wl["make"] is None or args.workload in ("gapped_n8192", "gapped_n16384", "fermi_n16384",
                                                   "paper_matrix_n8192"):
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle arm is timed on the "
                              "single-solve workloads gapped_n4096 and gapped_n256_fp64"}), flush=True)
            return
        reference_arm(args, wl["make"](), args.workload)
        return

    import torch
    import paper_2301_04642_gb300 as fe

    if args.workload == "ragged_batch64":
        return bench_batch(args, torch, fe)
    if args.workload == "serve_poisson":
        return bench_serve(args, torch, fe)

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    peaks, peak_kind = load_peaks()

    p = wl["make"]()
    n = p.n
    prec = wl["precision"]
    kT = float(getattr(p, "kT", 0.0) or 0.0)
    H = p.H.to(dev) if torch.is_tensor(p.H) else torch.from_numpy(p.H).to(dev)
    D = torch.empty_like(H)
    stream = torch.cuda.Stream(device=dev)
    ctx = fe.Context(device=local_rank, stream=stream.cuda_stream)
    tiles = apply_tiles(ctx, [n], prec, args.tiles)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MiB > L2

    def one():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        return ctx.solve(H, p.ne, kT=kT, tol=p.tol, D=D, precision=prec)

    for _ in range(args.warmup):
        r = one()
    iters = r["iters"]

    # ---- timed region: K solves, inputs resident in HBM
    lat = []
    l0 = ctx.launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            r = one()
            lat.append(r["ms"])
            assert r["status"] == 0, r
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
    launches = ctx.launch_count() - l0
    phases = ctx.phase_ms()  # the last timed solve: set-up, step loop, output
    t_ms = e0.elapsed_time(e1)
    # the last timed solve's error against the constructed reference (outside the timing)
    torch.cuda.synchronize()
    if p.Q is None:
        # a matrix given by a formula: the reference eigenpairs come from
        # cuSOLVER syevd (FP64) on this GPU, outside the timing
        lam_ref, Q_ref = torch.linalg.eigh(H)
        accuracy = probe_errors(torch, D, Q_ref, lam_ref.cpu().numpy(),
                                reference_occupations(lam_ref.cpu().numpy(), p.ne, kT), p.ne, kT, r)
        accuracy["reference"] = "cuSOLVER syevd (FP64) eigenpairs"
        gap_at_ne = float(lam_ref[int(p.ne)] - lam_ref[int(p.ne) - 1]) if 0 < p.ne < n else None
        del Q_ref
    else:
        accuracy = probe_errors(torch, D, p.Q, p.lam, reference_occupations(p.lam, p.ne, kT), p.ne, kT, r)
        gap_at_ne = None
    value, t_ms = job_rate(torch, dist, dev, args.steps, t_ms)

    # ---- end to end through the C ABI with pinned host buffers
    Hh = (p.H.cpu() if torch.is_tensor(p.H) else torch.from_numpy(p.H)).pin_memory()
    Dh = torch.empty_like(Hh).pin_memory()
    for _ in range(2):
        ctx.solve(Hh.numpy(), p.ne, kT=kT, tol=p.tol, D=Dh.numpy(), precision=prec)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        re = ctx.solve(Hh.numpy(), p.ne, kT=kT, tol=p.tol, D=Dh.numpy(), precision=prec)
        _ = re["e_band"]
    f1.record(stream)
    torch.cuda.synchronize()
    te_ms = f0.elapsed_time(f1)
    e2e, te_ms = job_rate(torch, dist, dev, args.steps, te_ms)

    # ---- per-kernel times (one profiled solve, CUDA events on the launch stream)
    ctx.profile(True)
    rp = one()
    prof = ctx.profile_read()
    steps_ms = ctx.profile_steps()
    ctx.profile(False)
    # zero temperature: the first iters_by_phase[0] tensor-core steps are
    # single FP16 products, the next iters_by_phase[1] split ones
    n_single = rp["iters_by_phase"][0] if kT == 0.0 else 0
    single_ms = float(sum(steps_ms[:n_single]))
    tc_split_ms = prof["tc_ms"] - single_ms
    tc_n = max(prof["tc_launches"] - n_single, 1)
    fp_n = max(prof["fp64_launches"], 1)
    tc_avg = tc_split_ms / tc_n
    fp_avg = prof["fp64_ms"] / fp_n
    # algorithmic work per launch (upper triangle incl. diagonal: n^2 (n+1) flops per product)
    sym_flops = float(n) * n * (n + 1)
    # the FP64-accurate steps: the digit-product kernel (mixed) or the SIMT FP64 kernel (fp64)
    fp_name = "k_digit_mma" if prec != "fp64" else "k_fp64_step"
    kernels = {
        "k_sym_mma": {"launches": prof["tc_launches"] - n_single, "ms_total": tc_split_ms, "ms_avg": tc_avg,
                      "algorithmic_flops": 3 * sym_flops,
                      "achieved_tflops": 3 * sym_flops / (tc_avg * 1e-3) / 1e12 if tc_split_ms > 0 else 0},
        fp_name: {"launches": prof["fp64_launches"], "ms_total": prof["fp64_ms"],
                  "ms_avg": fp_avg, "fp64_equivalent_flops": sym_flops,
                  "fp64_equivalent_tflops": sym_flops / (fp_avg * 1e-3) / 1e12 if prof["fp64_ms"] else 0},
    }
    if fp_name == "k_digit_mma":
        # 28 FP16 digit products per FP64-accurate product (levels a + c <= 6 of 7 digits)
        kernels[fp_name]["algorithmic_flops"] = 28 * sym_flops
        kernels[fp_name]["achieved_tflops"] = (28 * sym_flops / (fp_avg * 1e-3) / 1e12
                                               if prof["fp64_ms"] else 0)
        kernels[fp_name]["includes"] = "k_digit_prep (digit split of X) + k_digit_mma"
    else:
        kernels[fp_name]["algorithmic_flops"] = sym_flops
        kernels[fp_name]["achieved_tflops"] = kernels[fp_name]["fp64_equivalent_tflops"]
    tc_names = ["k_sym_mma", fp_name]
    if n_single:
        # the same kernel on one FP16 slice per operand: one product per chunk
        avg1 = single_ms / n_single
        kernels["k_sym_mma_fp16"] = {"launches": n_single, "ms_total": single_ms, "ms_avg": avg1,
                                     "algorithmic_flops": sym_flops,
                                     "achieved_tflops": sym_flops / (avg1 * 1e-3) / 1e12}
        tc_names.append("k_sym_mma_fp16")
    kernels["share_of_solve"] = {k: kernels[k]["ms_total"] / prof["solve_ms"] for k in tc_names}
    if kernels["k_sym_mma"]["ms_total"] >= kernels[fp_name]["ms_total"] or fp_name == "k_digit_mma":
        # every kernel of the mixed schedules runs on the tensor cores; the
        # dominant one is reported
        kname = max(tc_names, key=lambda k: kernels[k]["ms_total"])
        peak = peaks["bf16_tflops_sustained"]
        ach = kernels[kname]["achieved_tflops"]
        roof = {"kernel": kname, "bound": "tensor", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic_record(kname, "k_digit.cu" if kname == "k_digit_mma" else "k_mma.cu"),
                "peak_source": "%s bf16 dense sustained (fp16 dense has the same rate)" % peak_kind}
    else:
        peak = 1.25  # FP64 nominal of GB300 (no FP64 tensor path)
        ach = kernels["k_fp64_step"]["achieved_tflops"]
        roof = {"kernel": "k_fp64_step", "bound": "alu", "achieved": ach, "peak": peak,
                "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": traffic_record("k_fp64_step", "k_fp64.cu"),
                "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": {"mixed": "f16x2+f16digits", "try_fp16": "f16+f16x2+f16digits",
                                                       "fp32": "f16x2"}.get(prec, "f64"),
           "data": "synthetic",
           "config": {"workload": args.workload, "n": n, "n_e": p.ne, "kT": kT,
                      "precision": prec, "parallelism": "replicas" if world > 1 else "single",
                      "l2": "256 MiB buffer written before every step; working set > 129 MB L2",
                      "tiles": tiles, "gap_at_ne": gap_at_ne},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "phases_ms": phases,
           "effective_tflops": iters * 2.0 * n ** 3 * value / 1e12,
           "products_per_solve": iters, "iters_by_phase": r["iters_by_phase"],
           "accuracy": dict({"trace_err": abs(r["trace"] - p.ne)}, **accuracy),
           "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 8 * n * n,
                   "d2h_bytes_per_step": 8 * n * n},
           "gpu_launches": launches, "roofline": roof, "kernels": kernels,
           "clocks": clk.summary()}

    small_zero_t = n <= 4096 and kT == 0.0 and p.Q is not None  # plain FP64 / syevd / CPU arms only where they finish
    if rank == 0 and not args.no_baselines and small_zero_t:
        base = {}
        # the same expansion with every product in FP64 on this GPU
        t0 = time.perf_counter()
        r64 = ctx.solve(H, p.ne, tol=p.tol, D=D, precision="fp64")
        f_ref = reference_occupations(p.lam, p.ne, 0.0)
        torch.cuda.synchronize()
        base["fp64_gpu_sp2"] = {"solves_per_s": 1e3 / r64["ms"], "products": r64["iters"],
                                "accuracy": probe_errors(torch, D, p.Q, p.lam, f_ref, p.ne, 0.0, r64)}
        # the other precision schedules of the configuration (FP32-class split
        # products without the FP64-accurate polish; single-FP16 bulk until
        # RelTr < 5e-4, then split, then polish), each with its error
        for name in ("fp32", "try_fp16"):
            rs = ctx.solve(H, p.ne, tol=p.tol, D=D, precision=name, check=False)
            torch.cuda.synchronize()
            base["schedule_" + name] = {"solves_per_s": 1e3 / rs["ms"], "status": rs["status"],
                                        "iters_by_phase": rs["iters_by_phase"],
                                        "accuracy": probe_errors(torch, D, p.Q, p.lam, f_ref, p.ne, 0.0, rs)}
        # cuSOLVER syevd (torch.linalg.eigh, FP64) + D = V_occ V_occ^T
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record()
        w, V = torch.linalg.eigh(H)
        Vo = V[:, : int(p.ne)]
        Dsy = Vo @ Vo.T
        g1.record()
        torch.cuda.synchronize()
        base["cusolver_syevd"] = {"solves_per_s": 1e3 / g0.elapsed_time(g1)}
        base["speedup_vs_fp64_gpu_sp2"] = value / world / base["fp64_gpu_sp2"]["solves_per_s"]
        base["speedup_vs_cusolver_syevd"] = value / world / base["cusolver_syevd"]["solves_per_s"]
        out["baselines_same_gpu"] = base
        del Dsy, V
    if rank == 0:
        if small_zero_t:
            import oracle
            lo, hi = oracle.gershgorin(p.H)
            prods = sp2_products_on_spectrum(p.lam, lo, hi, p.ne, 5e-8)
            v, thr, sample = cpu_oracle_sample(p, prods)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": thr, "kind": "oracle", "sample": sample}
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


def apply_tiles(ctx, sizes, prec, mode):
    """Tile widths of the tensor-core products for these sizes: 'auto' runs
    the library's autotuner on them (outside the timed region), '256' / '128'
    fix the width.  Returns the config record."""
    if prec == "fp64":
        return None
    sizes = sorted(set(int(n) for n in sizes))
    if mode == "auto":
        ents = ctx.autotune(sizes, precision=prec, reps=2)
        return {"mode": "autotuned", "narrow_sizes": sum(e["bn"] == 128 for e in ents),
                "sizes": len(ents),
                "table": [[e["n"], e["bn"], round(e["ms_256"], 4), round(e["ms_128"], 4)] for e in ents]}
    for n in sizes:
        ctx.set_tile_width(n, int(mode), prec)
    return {"mode": "fixed", "bn": int(mode)}


def _kernel_times(ctx, n_list):
    """Per-kernel CUDA-event times of the last profiled solve or batch."""
    prof = ctx.profile_read()
    return {"k_sym_mma_ms": prof["tc_ms"], "k_sym_mma_launches": prof["tc_launches"],
            "fp64_accurate_ms": prof["fp64_ms"], "fp64_accurate_launches": prof["fp64_launches"],
            "solve_ms": prof["solve_ms"]}


def bench_batch(args, torch, fe):
    """64 gapped problems, n log-uniform in [512, 6144], in one fe_solve_batch."""
    dev = torch.device("cuda", 0)
    sizes = hp_synth.ragged_batch_sizes()
    probs = [hp_synth.ragged_member(i, device="cuda") for i in range(len(sizes))]
    items = []
    for p in probs:
        H = p.H.to(dev) if torch.is_tensor(p.H) else torch.from_numpy(p.H).to(dev)
        items.append(dict(H=H, ne=p.ne, tol=p.tol, D=torch.empty_like(H), precision="mixed"))
    stream = torch.cuda.Stream(device=dev)
    ctx = fe.Context(device=0, stream=stream.cuda_stream)
    if args.tiles == "auto":
        # tuned on the batch itself (outside the timed region): per-size
        # timings do not carry over to a launch that holds every problem's tiles
        trials = ctx.autotune_batch(items, reps=2)
        widths = [ctx.tile_width(n) for n in sizes]
        tiles = {"mode": "autotuned on the batch", "narrow_problems": sum(w == 128 for w in widths),
                 "trial_batch_ms": [round(t, 3) for t in trials]}
    else:
        tiles = apply_tiles(ctx, sizes, "mixed", args.tiles)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def one():
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        return ctx.solve_batch(items)

    for _ in range(args.warmup):
        rc, res = one()
    l0 = ctx.launch_count()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            rc, res = one()
            assert rc == 0
        e1.record(stream)
        torch.cuda.synchronize()
    t_ms = e0.elapsed_time(e1)
    launches = ctx.launch_count() - l0
    phases = ctx.phase_ms()  # the last timed batch: set-up, step loop, output
    ctx.profile(True)
    one()
    kern = _kernel_times(ctx, sizes)
    ctx.profile(False)
    products = sum(float(n) ** 3 * r["iters"] * 2.0 for n, r in zip(sizes, res))
    value = len(items) * args.steps / (t_ms / 1e3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f16x2+f16digits", "data": "synthetic",
           "config": {"workload": "ragged_batch64", "problems": len(items), "n_min": min(sizes),
                      "n_max": max(sizes), "n_e": "round(0.85 n)", "parallelism": "single",
                      "l2": "256 MiB buffer written before every step", "tiles": tiles},
           "effective_tflops": products * args.steps / (t_ms / 1e3) / 1e12,
           "max_trace_err": max(abs(r["trace"] - p.ne) for r, p in zip(res, probs)),
           "phases_ms": phases,
           "gpu_launches": launches, "kernels": kern, "clocks": clk.summary(), "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    ctx.close()


def bench_serve(args, torch, fe):
    """Continuous batching: Poisson arrivals of mixed zero-T / finite-T requests
    (by default n log-uniform in [1024, 8192] at 20/s: the sub-capacity variant
    of the serving configuration; FE_SERVE_NMAX=32768 FE_SERVE_RATE=200 asks for
    the full one), submitted at their arrival times; latency = submit to done."""
    dev = torch.device("cuda", 0)
    rate = float(os.environ.get("FE_SERVE_RATE", "20"))
    count = int(os.environ.get("FE_SERVE_COUNT", "40"))
    nmin = int(os.environ.get("FE_SERVE_NMIN", "1024"))
    nmax = int(os.environ.get("FE_SERVE_NMAX", "8192"))
    u = hp_synth.uniform(3000, 4 * count)
    reqs = []
    for k in range(count):
        n = int(round(math.exp(math.log(nmin) + u[4 * k] * (math.log(nmax) - math.log(nmin)))))
        n = max(64, n)
        ne = round(0.85 * n)
        if u[4 * k + 1] < 0.7:
            gap = 0.01 + 0.09 * u[4 * k + 2]
            p = hp_synth.gapped(n, ne, (-3.0, -gap / 2), (gap / 2, 1.0), 3100 + k, device="cuda")
            kT = 0.0
        else:
            kT = 0.001 + 0.009 * u[4 * k + 2]
            p = hp_synth.smeared(n, float(ne), kT, -2.0, 1.0, 3100 + k, device="cuda")
        H = p.H.to(dev) if torch.is_tensor(p.H) else torch.from_numpy(p.H).to(dev)
        reqs.append((n, ne, kT, p.tol, H, torch.empty_like(H)))
    gaps = [-math.log(max(1e-12, 1.0 - x)) / rate for x in hp_synth.uniform(3001, count)]
    ctx = fe.Context(device=0)
    torch.cuda.synchronize()
    # warm the kernels and slots on the first request
    t = ctx.submit(reqs[0][4], reqs[0][1], kT=reqs[0][2], tol=reqs[0][3], D=reqs[0][5])
    ctx.wait(t)
    l0 = ctx.launch_count()
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        tickets = []
        due = t0
        for (n, ne, kT, tol, H, D), g in zip(reqs, gaps):
            due += g
            while time.perf_counter() < due:
                time.sleep(0.0002)
            tickets.append(ctx.submit(H, ne, kT=kT, tol=tol, D=D))
        res = [ctx.wait(tk, timeout_s=1800) for tk in tickets]
        t1 = time.perf_counter()
    launches = ctx.launch_count() - l0
    lat = [r["ms"] for r in res]
    ok = sum(1 for r in res if r["status"] == 0)
    value = ok / (t1 - t0)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": count, "warmup": 1,
           "ms_per_step": (t1 - t0) * 1e3 / count, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f16x2+f16digits", "data": "synthetic",
           "config": {"workload": "serve_poisson", "requests": count, "rate_per_s": rate,
                      "n": "log-uniform [%d, %d]" % (nmin, nmax), "mix": "70% gapped, 30% finite T",
                      "parallelism": "single"},
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "completed_ok": ok, "gpu_launches": launches, "clocks": clk.summary(), "cpu_baseline": None}
    print(json.dumps(out), flush=True)
    ctx.close()


if __name__ == "__main__":
    main()
