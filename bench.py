#!/usr/bin/env python
"""Benchmark of the GD-lambda-AMG hot path on one GB300 (or N replicas).

Metric: seconds to the k smallest-|lambda| eigenpairs of Q = Gamma5 D at
eigen-residual 1e-8 (mixed precision: FP32 inner solves, FP64 outer).  The
timed step is the 16 x 8^3 workload (k = 50, two-level MG, 2^4 aggregates,
Nv = 8, SAP 2^4, 4 targets per outer iteration): multigrid setup +
eigensolve from the resident gauge field.
Also reported: the same step in plain FP64; the end-to-end time through the
C ABI from host buffers; the fine-stencil bandwidth on a 64 x 32^3 lattice;
the live roofline of the dominant kernel (HBM and, for the SAP block solves,
FP32 ALU against the measured FMA peak); the 64 x 32^3 three-level workload
(mixed precision, timed once after a warm-up; 16 pairs by default so that the
run ends within minutes, --large-k 100 for the workload's 100, --only-large
for that measurement alone); and the CPU oracle timed on per-operation
samples on the host's cores.  Prints one JSON line (rank 0).

usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "sec to k smallest-|lambda| of Q at res 1e-8, mixed vs FP64; stencil HBM GB/s"
WORKLOAD = "c2_16x8c3"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gdlamg", choices=["gdlamg", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-stencil", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-clocks", action="store_true",
                    help="no nvidia-smi clock sampling (profiling runs under ncu)")
    ap.add_argument("--smoother-sweep", action="store_true",
                    help="shifted-solve iterations and time vs tau for SAP / GMRES smoothing and the "
                         "D - tau Gamma5 / Q - tau forms on an 8^4 field, then exit")
    ap.add_argument("--ablation", action="store_true",
                    help="GD-lambda-AMG variants on the workload (k = 20): default, no interpolation "
                         "updates, Rayleigh-Ritz extraction; then exit")
    ap.add_argument("--local-coherence", action="store_true",
                    help="lc(v) of all 3072 eigenvectors of the 4^4 Q for the 128 interpolation sets "
                         "of 24 consecutive eigenpairs (block averages), then exit")
    ap.add_argument("--large", action="store_true",
                    help="study: 100 pairs of the 32x16^3 workload (4^4 aggregates, Nv 20, 16 targets per "
                         "iteration), mixed precision")
    ap.add_argument("--large-blocks", default="",
                    help="comma-separated targets per outer iteration for --large (default: the workload's 16)")
    ap.add_argument("--gradient", action="store_true",
                    help="eigenvalue derivatives of the 20 smallest |lambda| on a 16^4 field along 16 su(3) "
                         "directions, checked by central differences of Rayleigh quotients; then exit")
    ap.add_argument("--only-stencil", action="store_true",
                    help="run and print only the fine-stencil bandwidth measurement")
    ap.add_argument("--k", type=int, default=None,
                    help="eigenpairs per step instead of the workload's (short profiling runs)")
    ap.add_argument("--coarse-stencil", action="store_true",
                    help="run and print only the coarse-stencil comparison (tensor cores vs FMA units)")
    ap.add_argument("--no-coarse-stencil", action="store_true")
    ap.add_argument("--sap-bench", action="store_true",
                    help="run and print only the SAP block-solve measurement (32x16^3, 2 and 16 right-hand "
                         "sides, FP32 and FP16 block basis)")
    ap.add_argument("--no-large-workload", action="store_true",
                    help="skip the 64 x 32^3 three-level measurement")
    ap.add_argument("--large-workload", default="c4_64x32c3")
    ap.add_argument("--large-k", type=int, default=16,
                    help="eigenpairs of the large-workload measurement (the workload lists 100; "
                         "the default run times 16 so that it ends within minutes)")
    ap.add_argument("--only-large", action="store_true",
                    help="run only the large-workload measurement and print it")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--oracle-ops", action="store_true", help=argparse.SUPPRESS)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """Max of a per-rank float over all ranks of the default process group
    (the whole-job time of N replicas); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu capture of each kernel as it stands now, for the roofline's
# "traffic"; a kernel that changes is taken out of this table until it is
# captured again (the field is then null).  coarse_gmres_f32: two launches of
# coarse_gmres_kernel<float2, float> in the 16 x 8^3 step (k = 4, 4 targets),
# dram__bytes.sum.per_second x gpu__time_duration.sum = 9.808 and 9.820 MB
# (profiles/coarse_gmres_f32_c2_16x8c3.md).  sap_block_f32: two launches of
# sap_chi_kernel<float, float2> in the same step (four block solves per CTA),
# 6.8831 and 6.8836 MB read, 0 written (profiles/sap_chi_f32_c2_16x8c3.md).
NCU_TRAFFIC = {"coarse_gmres_f32": 9.814e6, "sap_block_f32": 6.8833e6}

# Work model of the SAP block solves for the FP32-ALU roofline, per block
# site and GMRES step j (0-based) of a block solve of k steps: the Dirichlet
# block operator (clover 504 + diagonal and shift 48 + 168 per in-block hop;
# 2^4 blocks have 4 in-block hops per site), 192 (j + 1) for the Gram-Schmidt
# inner products and updates, 72 for the norm and scaling and 96 for the
# solution update.  Summed over j: k (op + 168) + 192 k (k + 1) / 2, with the
# two sums read from the library's SAP work counters.
def sap_flops(site_steps, site_steps_tri, block=(2, 2, 2, 2)):
    hops = sum(2.0 * (b - 1) / b for b in block)
    op = 504.0 + 48.0 + 168.0 * hops
    return site_steps * (op + 168.0) + 192.0 * site_steps_tri


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, enabled=True):
        self.idx = gpu_index
        self.enabled = enabled
        self.proc = None
        self.file = None

    def start(self):
        if not self.enabled:
            return
        try:
            self.file = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = [r.split(",") for r in open(self.file.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- CPU oracle sample
# Operation counts of one GPU eigensolve of each workload (FGMRES iterations
# summed over targets, outer iterations; from the GPU bench line), used to
# scale the oracle's per-operation times to one eigensolve when no GPU run
# of the same process provides them (the reference arm).
REF_COUNTS = {"c2_16x8c3": dict(inner=3303, outer=168, block=4)}


def oracle_ops(w):
    """Time the oracle (FP64 numpy) on per-operation samples of the workload,
    in this process: one Q apply, the Galerkin build of P and D_c, one
    two-level MG cycle (SAP, Table 2 parameters), and one Gram-Schmidt pass
    of a vector against 50 orthonormal basis vectors (dot products + update,
    twice)."""
    from oracle.dirac import WilsonClover
    from oracle import mg
    from paper_2004_08146_gb300 import synth
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    op = WilsonClover(U, w["m0"], w["csw"])
    psi = synth.spinor(dims, w["seed"] + 11)
    t0 = time.perf_counter()
    for _ in range(3):
        op.Q(psi)
    t_apply = (time.perf_counter() - t0) / 3
    h = mg.TwoLevelMG(op, w["agg"], w["sap"], w["nv"], smoother="sap", form="g5")
    vecs = synth.spinor(dims, w["seed"] + 12, nvec=w["nv"])
    t0 = time.perf_counter()
    h.set_vectors(vecs)
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    h.cycle(psi, 0.05)
    t_cycle = time.perf_counter() - t0
    B = synth.complex_gaussian((op.n, 50), w["seed"] + 13)
    B, _ = np.linalg.qr(B)
    v = psi.reshape(-1)
    t0 = time.perf_counter()
    for _ in range(2):
        v = v - B @ (B.conj().T @ v)
    t_gs = time.perf_counter() - t0
    return dict(t_apply=t_apply, t_build=t_build, t_cycle=t_cycle, t_gs=t_gs)


def oracle_estimate(w, ops, inner, outer, block):
    """One eigensolve from per-operation times: the setup (setup_iters Galerkin
    builds, setup_iters x Nv cycles), every FGMRES iteration (one cycle and
    one Q apply) and every added basis vector (Gram-Schmidt and one Q apply)."""
    setup = 6 * ops["t_build"] + 6 * w["nv"] * ops["t_cycle"]
    return setup + inner * (ops["t_cycle"] + ops["t_apply"]) + outer * block * (ops["t_gs"] + ops["t_apply"])


def oracle_sample_subprocess(workload, k=None):
    """oracle_ops of the workload in a child process with one BLAS/OpenMP
    thread, so the timing uses exactly one host core."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-ops", "--workload", workload]
    if k is not None:
        cmd += ["--k", str(k)]
    t0 = time.perf_counter()
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    wall = time.perf_counter() - t0
    if out.returncode != 0:
        raise RuntimeError("oracle sample failed: " + out.stderr[-400:])
    ops = json.loads(out.stdout.strip().splitlines()[-1])
    ops["wall_s"] = wall
    return ops


def cpu_baseline_line(w, ops, inner, outer, block, counts_from):
    est = oracle_estimate(w, ops, inner, outer, block)
    return {"value": est, "unit": "s", "cores": 1, "kind": "oracle", "host_cpu_count": os.cpu_count(),
            "sample": (f"FP64 numpy oracle on one host core, per-operation samples of the {w['name']} workload: "
                       f"Q apply {ops['t_apply']:.3f} s, Galerkin build {ops['t_build']:.2f} s, two-level cycle "
                       f"{ops['t_cycle']:.2f} s, Gram-Schmidt against 50 vectors {ops['t_gs']:.3f} s; value = "
                       f"6 builds + 6 x Nv cycles + {inner} FGMRES iterations x (cycle + apply) + {outer} x {block} "
                       f"added vectors x (Gram-Schmidt + apply), counts from {counts_from}"),
            "per_op_s": {k: round(v, 4) for k, v in ops.items() if k.startswith("t_")}}


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from paper_2004_08146_gb300 import workloads
    w = workloads.get(args.workload)
    w["name"] = args.workload
    c = REF_COUNTS[args.workload]
    samples, walls = [], []
    for i in range(args.warmup + args.steps):
        ops = oracle_sample_subprocess(args.workload)
        if i >= args.warmup:
            samples.append(oracle_estimate(w, ops, c["inner"], c["outer"], c["block"]))
            walls.append(ops["wall_s"])
    val = float(np.mean(samples))
    cpu = cpu_baseline_line(w, ops, c["inner"], c["outer"], c["block"], "the GPU bench's recorded counts")
    cpu["value"] = val
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            # each step is one timed per-operation sample; its wall time is the step time
            "ms_per_step": float(np.mean(walls)) * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, w["dims"])), "k": w["k"]},
            "cpu_baseline": cpu,
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.oracle_ops:
        from paper_2004_08146_gb300 import workloads
        print(json.dumps(oracle_ops(workloads.get(args.workload))), flush=True)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2004_08146_gb300 import qcd, synth, workloads

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    devn = torch.device("cuda", local)
    w = workloads.get(args.workload)
    if args.k is not None:
        w["k"] = args.k
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    n = int(np.prod(dims)) * 12
    stream = torch.cuda.Stream(devn)
    sp = stream.cuda_stream
    if args.gradient:
        print(json.dumps({"gradient": gradient_study(qcd, synth, torch, devn, stream)}), flush=True)
        return
    if args.large:
        for b in [int(x) for x in args.large_blocks.split(",")] if args.large_blocks else [None]:
            print(json.dumps({"large": large_study(qcd, synth, torch, devn, stream, b)}), flush=True)
        return
    if args.local_coherence:
        print(json.dumps({"local_coherence": local_coherence_study(qcd, synth, torch, devn, stream)}), flush=True)
        return
    if args.ablation:
        print(json.dumps({"ablation": ablation(qcd, synth, torch, devn, stream, w, U, dims, n)}), flush=True)
        return
    if args.smoother_sweep:
        print(json.dumps({"smoother_sweep": smoother_sweep(qcd, synth, torch, devn, stream)}), flush=True)
        return
    if args.only_stencil:
        peak, _ = measured_peaks()
        print(json.dumps({"stencil": stencil_bench(qcd, synth, torch, devn, stream, peak)}), flush=True)
        return
    if args.coarse_stencil:
        print(json.dumps({"coarse_stencil": coarse_stencil_bench(qcd, synth, torch, devn, stream)}), flush=True)
        return
    if args.sap_bench:
        print(json.dumps({"sap": sap_bench(qcd, synth, torch, devn, stream)}), flush=True)
        return
    if args.only_large:
        print(json.dumps({"large_workload": large_workload(qcd, synth, torch, devn, stream, workloads,
                                                           args.large_workload, args.large_k)}), flush=True)
        return

    def make(precision):
        p = workload_params(qcd, w, precision=precision)
        ctx = qcd.Context(params=p, stream=sp)
        ctx.qcd_set_gauge(U, dims, w["m0"], w["csw"])
        return ctx

    V = torch.zeros(w["k"] * n, dtype=torch.complex128, device=devn)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=devn)   # > L2 (129 MB)

    def step(ctx):
        if w["use_mg"]:
            ctx.qcd_mg_setup(w["nv"], w["agg"])
        rc, lam, info = ctx.qcd_eigs(w["k"], 1e-8, V)
        if rc != qcd.QCD_OK:
            raise RuntimeError(f"eigensolve did not converge: {info.locked} locked")
        return lam, info

    def timed_steps(ctx, K, W, profile=None):
        infos = []
        for _ in range(W):
            step(ctx)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        ms = []
        for i in range(K):
            # the last timed step is the profiler range (ncu --profile-from-start off)
            last = profile and i == K - 1
            with torch.cuda.stream(stream):
                flush.fill_(1.0)            # evict L2 between steps (outside the timed interval)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            if last:
                torch.cuda.synchronize()
                torch.cuda.profiler.start()
            e0.record(stream)
            lam, info = step(ctx)
            e1.record(stream)
            e1.synchronize()
            if last:
                torch.cuda.profiler.stop()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        return ms, infos, lam

    # ---- mixed precision: find the dominant kernel in a warm-up step
    ctx = make(qcd.QCD_MIXED)
    step(ctx)
    qcd.qcd_stats_reset(1)
    step(ctx)
    st = qcd.qcd_stats_read()
    dom = max(st, key=lambda s: s["total_ms"])
    # ---- timed region: launch counts for all kernels, events on the dominant one
    clocks = ClockSampler(local, enabled=not args.no_clocks)
    qcd.qcd_stats_reset(2, dom["name"])
    clocks.start()
    ms, infos, lam = timed_steps(ctx, args.steps, max(0, args.warmup - 2), profile=True)
    clk = clocks.stop()
    st_timed = {s["name"]: s for s in qcd.qcd_stats_read()}
    torch.cuda.synchronize()
    sap_work = qcd.qcd_stats_sap_work()
    qcd.qcd_stats_reset(0)
    launches = sum(s["launches"] for s in st_timed.values())
    # warm-up steps ran inside the accounting window too: count only the timed share
    n_steps_in_window = args.steps + max(0, args.warmup - 2)
    launches_timed = int(round(launches * args.steps / n_steps_in_window))
    d = st_timed[dom["name"]]
    peak, peak_kind = measured_peaks()
    achieved = d["timed_bytes"] / (d["total_ms"] * 1e-3) / 1e9 if d["total_ms"] > 0 else 0.0
    step_s = max_over_ranks(sum(ms) / len(ms) / 1e3, devn)

    # ---- FP64 comparison (same workload, same tolerance)
    fp64 = None
    if not args.no_fp64:
        ctx64 = make(qcd.QCD_FP64)
        ms64, infos64, lam64 = timed_steps(ctx64, 1, 1)
        fp64 = {"value": ms64[0] / 1e3, "unit": "s", "outer": infos64[0].outer, "inner": infos64[0].inner,
                "max_abs_dlambda_vs_mixed": float(np.max(np.abs(lam64 - lam)) / np.max(np.abs(lam)))}
        ctx64.close()

    # ---- end to end through the C ABI from host buffers
    e2e_s = None
    if not args.no_e2e:
        ctx_e = qcd.Context(params=workload_params(qcd, w, precision=qcd.QCD_MIXED), stream=sp)
        Vh = torch.empty(w["k"] * n, dtype=torch.complex128).pin_memory()
        e2e, e2e_info = [], []
        for i in range(1 + max(1, min(args.steps, args.e2e_steps))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx_e.qcd_set_gauge(U, dims, w["m0"], w["csw"])
            lam_e, info_e = step(ctx_e)
            stream.synchronize()                  # V is written on the library's stream
            Vh.copy_(V, non_blocking=True)
            torch.cuda.current_stream(devn).synchronize()
            if i > 0:
                e2e.append(time.perf_counter() - t0)
                e2e_info.append({"outer": info_e.outer, "inner": info_e.inner})
        ctx_e.close()
        e2e_s = float(np.mean(e2e))

    # ---- fine-stencil bandwidth, 64 x 32^3 (inputs far larger than L2)
    stencil = None
    if not args.no_stencil and rank == 0:
        stencil = stencil_bench(qcd, synth, torch, devn, stream, peak)

    # ---- SAP block solves against the FP32 ALU peak (work counted from the steps taken)
    alu = None
    if d["name"].startswith("sap_block_f32") and d["total_ms"] > 0:
        fp32_peak = qcd.qcd_fma_peak(qcd.QCD_FP32)
        sflops = sap_flops(*sap_work, block=w["sap"])
        alu = {"kernel": d["name"], "bound": "alu", "achieved": sflops / (d["total_ms"] * 1e-3) / 1e12,
               "peak": fp32_peak, "unit": "TFLOP/s", "peak_kind": "measured FP32 FMA probe (qcd_fma_peak)",
               "frac": sflops / (d["total_ms"] * 1e-3) / 1e12 / fp32_peak,
               "site_steps": sap_work[0]}
    fp64_peak = qcd.qcd_fma_peak(qcd.QCD_FP64)
    fp64_tc_peak = qcd.qcd_fma_peak(2)

    coarse = None
    if not args.no_coarse_stencil and rank == 0:
        coarse = coarse_stencil_bench(qcd, synth, torch, devn, stream)

    # ---- the 64 x 32^3 three-level workload, 100 pairs, mixed precision
    large = None
    if not args.no_large_workload and rank == 0:
        large = large_workload(qcd, synth, torch, devn, stream, workloads, args.large_workload, args.large_k)

    cpu = None
    if not args.no_cpu and rank == 0 and ws == 1:
        w["name"] = args.workload
        ops = oracle_sample_subprocess(args.workload)
        cpu = cpu_baseline_line(w, ops, int(np.mean([i.inner for i in infos])), int(np.mean([i.outer for i in infos])),
                                w.get("block", qcd.default_params().block), "this run's GPU steps")

    if rank == 0:
        info = infos[-1]
        line = {
            "metric": METRIC, "value": step_s, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "lattice": "x".join(map(str, dims)), "k": w["k"],
                       "mg": f"2-level, {w['agg']} aggregates, Nv={w['nv']}, SAP {w['sap']}",
                       "targets_per_iteration": w.get("block", 2),
                       "precision": "FP32 inner / FP64 outer", "tol": 1e-8, "m0": w["m0"], "csw": w["csw"],
                       "eps": w["eps"], "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "e2e": None if e2e_s is None else {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(U.nbytes),
                                               "d2h_bytes_per_step": int(V.numel() * 16 + 8 * w["k"]),
                                               "steps": len(e2e), "iterations": e2e_info},
            "gpu_launches": launches_timed,
            "roofline": {"kernel": dom["name"], "bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                         "traffic": NCU_TRAFFIC.get(dom["name"]), "launches_timed": d["timed"],
                         "avg_launch_us": d["total_ms"] * 1e3 / max(1, d["timed"]),
                         "share_of_step": d["total_ms"] / (sum(ms) * n_steps_in_window / args.steps)},
            "eig": {"outer": info.outer, "inner": info.inner, "locked": info.locked, "updates": info.updates,
                    "max_residual": info.max_residual, "min_abs_lambda": float(np.min(np.abs(lam))),
                    "max_abs_lambda": float(np.max(np.abs(lam)))},
            "alu_roofline": alu,
            "fp64_fma_peak_tflops": fp64_peak,
            "fp64_tensor_peak_tflops": fp64_tc_peak,
            "fp64": fp64,
            "stencil": stencil,
            "coarse_stencil": coarse,
            "large_workload": large,
            "clocks": clk,
            "cpu_baseline": None if cpu is None else {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "kernel_share_warmup": {s["name"]: round(s["total_ms"], 3) for s in
                                    sorted(st, key=lambda s: -s["total_ms"])[:8]},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def workload_params(qcd, w, **kw):
    """Library parameters of a workload: Table 2 defaults plus the workload's
    MG and outer-iteration shape."""
    p = dict(use_mg=w["use_mg"], sap_block=w["sap"])
    for key in ("block", "m_min", "m_max", "update_every", "levels", "nv2", "agg2", "sap_half", "coarse_maxiter"):
        if key in w:
            p[key] = w[key]
    p.update(kw)
    return qcd.default_params(**p)


def large_workload(qcd, synth, torch, devn, stream, workloads, name, k):
    """The 64 x 32^3 workload (2.1 M sites, 25 M unknowns; eps 0.6, c_sw 1.9),
    three-level MG (4^4 then 2^4 aggregates, Nv = nv2 = 24), k pairs at
    residual 1e-8 (the workload lists 100), 16 targets per outer iteration,
    mixed precision: one warm-up setup and a 2-pair solve, then one timed
    setup + eigensolve of k pairs (CUDA events on the library's stream, every
    kernel timed by the library's accounting, clocks sampled)."""
    w = workloads.get(name)
    w["k"] = int(k)
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    n = 12 * int(np.prod(dims))
    p = workload_params(qcd, w, max_outer=2000)
    ctx = qcd.Context(params=p, stream=stream.cuda_stream)
    t0 = time.perf_counter()
    ctx.qcd_set_gauge(U, dims, w["m0"], w["csw"])
    t_gauge = time.perf_counter() - t0
    V = torch.zeros(w["k"] * n, dtype=torch.complex128, device=devn)
    ctx.qcd_mg_setup(w["nv"], w["agg"])                  # warm-up
    ctx.qcd_eigs(2, 1e-8, V)
    torch.cuda.synchronize()
    clocks = ClockSampler(devn.index or 0)
    qcd.qcd_stats_reset(1)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.qcd_mg_setup(w["nv"], w["agg"])
    e1.record(stream)
    rc, lam, info = ctx.qcd_eigs(w["k"], 1e-8, V)
    e2.record(stream)
    e2.synchronize()
    clk = clocks.stop()
    st = qcd.qcd_stats_read()
    torch.cuda.synchronize()
    sap_work = qcd.qcd_stats_sap_work()
    qcd.qcd_stats_reset(0)
    ctx.close()
    top = sorted(st, key=lambda r: -r["total_ms"])[:12]
    sap = [r for r in st if r["name"] == "sap_block_f32"]
    out = {"workload": name, "lattice": "x".join(map(str, dims)), "unknowns": n, "k": w["k"],
           "mg": f"{w.get('levels', 2)}-level, {w['agg']} then {w.get('agg2')} aggregates, Nv={w['nv']}, "
                 f"nv2={w.get('nv2')}, SAP {w['sap']}",
           "targets_per_iteration": w["block"], "m_min": w["m_min"], "m_max": w["m_max"], "m0": w["m0"],
           "csw": w["csw"], "eps": w["eps"], "precision": "FP32 inner / FP64 outer",
           "converged": bool(info.converged), "rc": rc,
           "value": (e0.elapsed_time(e2)) / 1e3, "unit": "s", "setup_s": e0.elapsed_time(e1) / 1e3,
           "eigs_s": e1.elapsed_time(e2) / 1e3, "set_gauge_s": t_gauge,
           "outer": info.outer, "inner": info.inner, "locked": info.locked, "updates": info.updates,
           "coarse_iterations": info.coarse_iterations, "max_residual": info.max_residual,
           "min_abs_lambda": float(np.nanmin(np.abs(lam))), "max_abs_lambda": float(np.nanmax(np.abs(lam))),
           "clocks": clk, "kernel_ms": {r["name"]: round(r["total_ms"], 1) for r in top},
           "gpu_launches": int(sum(r["launches"] for r in st))}
    if sap and sap[0]["total_ms"] > 0:
        fl = sap_flops(*sap_work, block=w["sap"])
        peak = qcd.qcd_fma_peak(qcd.QCD_FP32)
        out["sap_alu"] = {"achieved": fl / (sap[0]["total_ms"] * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                          "frac": fl / (sap[0]["total_ms"] * 1e-3) / 1e12 / peak}
    return out


def gradient_study(qcd, synth, torch, devn, stream):
    """Differentiation workload: 16^4 field (eps 0.5, csw 1.5, m0 of the
    workload table), the 20 smallest-|lambda| eigenpairs from the GPU
    eigensolver (two-level MG, 4^4 aggregates, Nv = 8), then d lambda_k / d eps along 16 random su(3)
    directions X (U -> exp(i eps X) U).  Each derivative is checked against
    the central difference (h = 1e-6) of the Rayleigh quotient v_k^H Q(U(+-h)) v_k,
    whose derivative at eps = 0 is the same Hellmann-Feynman expression.  The
    per-link forces of all 20 eigenvalues are timed once and contracted with
    every direction against the directional derivatives."""
    from paper_2004_08146_gb300 import workloads
    w = workloads.get("c5_16c4")
    dims, m0, csw = tuple(w["dims"]), w["m0"], w["csw"]
    k, ndir, h = w["k"], 16, 1e-6
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    n = 12 * int(np.prod(dims))
    p = qcd.default_params(sap_block=w["sap"])
    ctx = qcd.Context(params=p, stream=stream.cuda_stream)
    ctx.qcd_set_gauge(U, dims, m0, csw)
    V = torch.zeros(k * n, dtype=torch.complex128, device=devn)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.qcd_mg_setup(w["nv"], w["agg"])      # 4^4 aggregates: a 4^4 coarse lattice
    rc, lam, info = ctx.qcd_eigs(k, 1e-8, V)
    torch.cuda.synchronize()
    t_eigs = time.perf_counter() - t0
    Vm = V.view(k, n)
    ctx_fd = qcd.Context(params=qcd.default_params(precision=qcd.QCD_FP64), stream=stream.cuda_stream)
    QV = torch.empty_like(Vm)
    worst, t_der = 0.0, 0.0

    def moved(X, eps):   # exp(i eps X) U to O(eps^3) ~ 1e-18 for eps = 1e-6
        X2 = np.einsum('...ab,...bc->...ac', X, X)
        E = np.eye(3) + 1j * eps * X - 0.5 * eps * eps * X2
        return np.einsum('...ab,...bc->...ac', E, U)

    def rayleigh(Um):
        ctx_fd.qcd_set_gauge(Um, dims, m0, csw)
        for j in range(k):
            ctx_fd.qcd_apply_Q(Vm[j], QV[j], 0.0)
        torch.cuda.synchronize()      # the library's stream is not torch's
        return np.array([torch.vdot(Vm[j], QV[j]).real.item() / torch.vdot(Vm[j], Vm[j]).real.item()
                         for j in range(k)])

    # per-link forces of all k eigenvalues (gauge-field layout per eigenvector)
    nl = 36 * int(np.prod(dims))
    F = torch.empty(k * nl, dtype=torch.complex128, device=devn)
    ctx.qcd_eig_force(k, V, F)                  # warm-up (buffers)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ctx.qcd_eig_force(k, V, F)
    torch.cuda.synchronize()
    t_force = time.perf_counter() - t1
    Fm = F.view(k, -1, 3, 3)
    worst_force = 0.0
    for d in range(ndir):
        X = synth.su3_directions(dims, 2000 + d, 1)[0]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        der = ctx.qcd_eig_derivative(X, k, V)
        t_der += time.perf_counter() - t1
        fd = (rayleigh(moved(X, h)) - rayleigh(moved(X, -h))) / (2 * h)
        worst = max(worst, float(np.max(np.abs(der - fd) / np.maximum(np.abs(fd), 1e-3))))
        # sum_{x,mu} tr(X F_k) must reproduce the directional derivative
        Xt = torch.from_numpy(np.ascontiguousarray(X).reshape(-1, 3, 3)).to(devn)
        con = (Xt.unsqueeze(0) * Fm.transpose(-1, -2)).sum(dim=(1, 2, 3)).real.cpu().numpy()
        worst_force = max(worst_force, float(np.max(np.abs(con - der) / np.maximum(np.abs(der), 1e-3))))
    ctx.close()
    ctx_fd.close()
    return {"lattice": "16^4", "m0": m0, "k": k, "directions": ndir, "eigs_s": t_eigs, "converged": bool(info.converged),
            "min_abs_lambda": float(np.min(np.abs(lam))), "derivative_s_per_direction": t_der / ndir,
            "max_rel_dev_from_central_difference": worst, "h": h,
            "force_s_per_eigenvector": t_force / k,
            "max_rel_dev_force_contraction_vs_derivative": worst_force}


def large_study(qcd, synth, torch, devn, stream, block=None):
    """The 32x16^3 workload (1,572,864 unknowns; eps 0.6, csw 1.7, m0 from the
    dense-proxy tuning): 100 eigenpairs to residual 1e-8, mixed precision,
    two-level MG with 4^4 aggregates and Nv = 20, SAP on 2^4 blocks with an
    FP16-stored block basis, 16 targets per outer iteration (m_min 30,
    m_max 50; ``block`` overrides the 16), P rebuilt every 20 locks.
    Reported: setup and eigensolver times, iteration counts, residuals, and
    the largest deviation of V^H V from the identity."""
    from paper_2004_08146_gb300 import workloads
    w = workloads.get("c3_32x16c3")
    dims = tuple(w["dims"])
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    n = 12 * int(np.prod(dims))
    k = w["k"]
    block = w["block"] if block is None else block
    p = workload_params(qcd, w, block=block, max_outer=4000)
    ctx = qcd.Context(params=p, stream=stream.cuda_stream)
    ctx.qcd_set_gauge(U, dims, w["m0"], w["csw"])
    V = torch.zeros(k * n, dtype=torch.complex128, device=devn)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.qcd_mg_setup(w["nv"], w["agg"])
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    rc, lam, info = ctx.qcd_eigs(k, 1e-8, V)
    torch.cuda.synchronize()
    t_eigs = time.perf_counter() - t0
    Vm = V.view(k, n)
    orth = float((Vm.conj() @ Vm.T - torch.eye(k, dtype=V.dtype, device=devn)).abs().max().item())
    ctx.close()
    return {"workload": "c3_32x16c3", "lattice": "32x16^3", "unknowns": n, "k": k, "block": block,
            "nv": w["nv"], "aggregates": list(w["agg"]), "m0": w["m0"], "sap_half": w.get("sap_half", 0),
            "setup_s": t_setup, "setup_plus_eigs_s": t_eigs, "converged": bool(info.converged),
            "locked": info.locked, "outer": info.outer, "inner": info.inner, "updates": info.updates,
            "coarse_iterations": info.coarse_iterations, "max_residual": info.max_residual,
            "min_abs_lambda": float(np.min(np.abs(lam))), "max_abs_lambda": float(np.max(np.abs(lam))),
            "max_abs_VhV_minus_I": orth}


def local_coherence_study(qcd, synth, torch, devn, stream):
    """The 4^4 local-coherence study of Sec. 3 for Q: the full spectrum
    (dense eigendecomposition on the host, 3072 eigenpairs ordered on the real
    line) is cut into 128 interpolation sets of 24 consecutive eigenpairs; for
    each set P is built from its vectors (2^4 aggregates) and lc(v) of every
    eigenvector is computed on the GPU.  Reported: 16 x 16 block averages of
    the 128 x 3072 matrix (rows: sets from most negative to most positive),
    and the averages the paper discusses."""
    dims = (4, 4, 4, 4)
    U = synth.gauge_field(dims, 0.3, 1001)
    ctx = qcd.Context(params=qcd.default_params(precision=qcd.QCD_FP64, sap_block=(2, 2, 2, 2)),
                      stream=stream.cuda_stream)
    ctx.qcd_set_gauge(U, dims, -0.2, 1.0)
    # dense Q from the library's own operator, columns Q e_i in batches of 16;
    # its full eigendecomposition (numpy, host) only generates the study's inputs
    N = 12 * int(np.prod(dims))
    Qd = np.zeros((N, N), dtype=np.complex128)
    E = torch.zeros(16 * N, dtype=torch.complex128, device=devn)
    out = torch.empty_like(E)
    for c0 in range(0, N, 16):
        E.zero_()
        for j in range(16):
            E[j * N + c0 + j] = 1.0
        torch.cuda.synchronize()      # E is written on torch's stream, read on the library's
        ctx.qcd_apply(qcd.QCD_OP_Q, qcd.QCD_FP64, 16, E, out, [0.0] * 16)
        torch.cuda.synchronize()
        Qd[:, c0:c0 + 16] = out.cpu().numpy().reshape(16, N).T
    w, Y = np.linalg.eigh(0.5 * (Qd + Qd.conj().T))
    Yd = torch.from_numpy(np.ascontiguousarray(Y.T)).to(devn)
    nset, per = N // 24, 24
    lc = np.zeros((nset, N))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(nset):
        ctx.qcd_mg_update_from_eigvecs(Yd[s * per:(s + 1) * per], per)
        lc[s] = ctx.qcd_local_coherence(N, Yd)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    ctx.close()
    blocks = lc.reshape(16, nset // 16, 16, N // 16).mean(axis=(1, 3))
    order = np.argsort(np.abs(w))
    small = np.zeros(N, dtype=bool)
    small[order[:N // 10]] = True                        # 10 % smallest |lambda|
    central = [s for s in range(nset) if small[s * per:(s + 1) * per].all()]
    outer = [0, nset - 1]
    return {"lattice": "4^4", "sets": nset, "per_set": per, "seconds_gpu": secs,
            "mean_lc": float(lc.mean()), "no_coherence_lc": 0.5, "no_coherence_lc2": 768 / 3072,
            "mean_lc_small10_vs_central_sets": float(lc[np.ix_(central, np.where(small)[0])].mean()),
            "mean_lc_small10_vs_outermost_sets": float(lc[np.ix_(outer, np.where(small)[0])].mean()),
            "mean_lc_outside_own_set_small10": float(np.mean([lc[s][small & (np.arange(N) // per != s)].mean()
                                                              for s in central])),
            "block_means_16x16": np.round(blocks, 3).tolist()}


def ablation(qcd, synth, torch, devn, stream, w, U, dims, n):
    """The variants of Sec. 4 on the workload: harmonic Ritz extraction with
    interpolation updates after every lock (the method), without updates, and
    with Rayleigh-Ritz extraction; 20 eigenpairs, at most 600 outer iterations."""
    k = 20
    rows = []
    for name, kw in (("harmonic+updates", {}), ("harmonic, no updates", {"update_every": 0}),
                     ("rayleigh-ritz+updates", {"extraction": qcd.QCD_EXTRACT_RITZ})):
        p = qcd.default_params(use_mg=w["use_mg"], sap_block=w["sap"], max_outer=600, **kw)
        ctx = qcd.Context(params=p, stream=stream.cuda_stream)
        ctx.qcd_set_gauge(U, dims, w["m0"], w["csw"])
        V = torch.zeros(k * n, dtype=torch.complex128, device=devn)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.qcd_mg_setup(w["nv"], w["agg"])
        rc, lam, info = ctx.qcd_eigs(k, 1e-8, V)
        torch.cuda.synchronize()
        rows.append({"variant": name, "converged": bool(info.converged), "locked": info.locked,
                     "outer": info.outer, "inner": info.inner, "updates": info.updates,
                     "coarse_iterations": info.coarse_iterations, "s": time.perf_counter() - t0})
        ctx.close()
    return {"workload": "c2_16x8c3", "k": k, "rows": rows}


def smoother_sweep(qcd, synth, torch, devn, stream):
    """Iterations and time of one shifted solve (Q - tau) x = b to 1e-8 relative
    residual against the shift tau, for the SAP and the GMRES smoother and for
    the two forms of the correction equation (Sec. 2 last paragraph, Sec. 3):
    8^4 field with the 16x8^3 workload's eps, csw and m0, two-level MG with 2^4
    aggregates, Nv = 8, SAP on 2^4 blocks."""
    dims = (8, 8, 8, 8)
    U = synth.gauge_field(dims, 0.5, 1005)
    m0, csw = -0.85, 1.5
    b = torch.from_numpy(synth.spinor(dims, 1006).reshape(-1)).to(devn)
    rows = []
    for sm_name, sm in (("sap", qcd.QCD_SMOOTHER_SAP), ("gmres", qcd.QCD_SMOOTHER_GMRES)):
        for form_name, form in (("D-tau*G5", qcd.QCD_OP_D), ("Q-tau", qcd.QCD_OP_Q)):
            p = qcd.default_params(smoother=sm, correction_form=form, sap_block=(2, 2, 2, 2))
            ctx = qcd.Context(params=p, stream=stream.cuda_stream)
            ctx.qcd_set_gauge(U, dims, m0, csw)
            ctx.qcd_mg_setup(8, (2, 2, 2, 2))
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            ctx.qcd_shifted_solve(b, x, 0.0, 1e-8)            # warm-up
            # shifts across the wanted part of the spectrum (the 50 smallest
            # |lambda| of the 16x8^3 workload reach 0.25); beyond it the
            # two-level solver stops converging for every smoother and form
            for tau in (0.0, 0.05, 0.1, 0.15, 0.2, 0.25):
                x.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rc, info = ctx.qcd_shifted_solve(b, x, tau, 1e-8)
                torch.cuda.synchronize()
                rows.append({"smoother": sm_name, "form": form_name, "tau": tau, "converged": rc == qcd.QCD_OK,
                             "fgmres_iterations": info.iterations, "refinements": info.refinements,
                             "residual": info.residual, "ms": (time.perf_counter() - t0) * 1e3})
            ctx.close()
    return {"lattice": "8^4", "eps": 0.5, "csw": csw, "m0": m0, "tol": 1e-8, "rows": rows}


def coarse_stencil_bench(qcd, synth, torch, devn, stream, reps=20):
    """The coarse stencil of the 32 x 16^3 field with 4^4 aggregates and
    Nv = 24 (512 coarse sites, 2 Nv = 48, the size of the 64 x 32^3
    workload's level 2 and 1/16 of its level 1) on 16 right-hand sides in one
    apply, FP32 data: tensor cores (3xTF32 mma.sync) against the FMA units.
    Flops 8 x 9 x (2 Nv)^2 per site and right-hand side; bytes: the stencil
    blocks once plus the vectors in and out."""
    dims, nv, nrhs = (32, 16, 16, 16), 24, 16
    U = synth.gauge_field(dims, 0.6, 1004)
    out = {"lattice": "32x16^3", "aggregates": [4, 4, 4, 4], "nv": nv, "nrhs": nrhs}
    for tensor in (1, 0):
        ctx = qcd.Context(params=qcd.default_params(setup_iters=1, coarse_tensor=tensor), stream=stream.cuda_stream)
        ctx.qcd_set_gauge(U, dims, -0.85, 1.9)
        ctx.qcd_mg_setup(nv, (4, 4, 4, 4))
        info = ctx.qcd_mg_info()
        nco = info["coarse_sites"] * 2 * nv
        x = torch.randn(nrhs * nco, dtype=torch.complex64, device=devn)
        y = torch.empty_like(x)
        taus = [0.01] * nrhs
        torch.cuda.synchronize()
        for _ in range(3):
            ctx.qcd_coarse_apply(qcd.QCD_OP_D, qcd.QCD_FP32, nrhs, x, y, taus)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.qcd_coarse_apply(qcd.QCD_OP_D, qcd.QCD_FP32, nrhs, x, y, taus)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        sites = info["coarse_sites"]
        flops = 8.0 * 9 * (2 * nv) ** 2 * sites * nrhs
        nbytes = 8.0 * (9 * (2 * nv) ** 2 * sites + 2 * nrhs * nco)
        out["tensor" if tensor else "fma"] = {"us_per_apply": t * 1e6, "tflops": flops / t / 1e12,
                                               "gbs": nbytes / t / 1e9}
        ctx.close()
    return out


def sap_bench(qcd, synth, torch, devn, stream, reps=5):
    """SAP smoothing (Eq. 2.10, 2^4 blocks, block GMRES to 1e-1 or 10 steps,
    D - tau Gamma5 form) on the 32 x 16^3 field (eps 0.6, c_sw 1.7, m0 -1.1;
    inputs larger than L2) with 2 and 16 right-hand sides, FP32 with the
    block basis in FP32 and in FP16: per launch of the block-solve kernel
    (one colour) its CUDA-event time, the block solves and GMRES steps it ran,
    and the counted block-solve arithmetic against the measured FP32 FMA
    peak."""
    dims = (32, 16, 16, 16)
    U = synth.gauge_field(dims, 0.6, 1003)
    V = int(np.prod(dims))
    peak = qcd.qcd_fma_peak(qcd.QCD_FP32)
    out = {"lattice": "32x16^3", "block": [2, 2, 2, 2], "fp32_fma_peak_tflops": peak}
    for nrhs in (2, 16):
        b = torch.randn(nrhs * V * 12, dtype=torch.complex64, device=devn)
        taus = [0.01 * j for j in range(nrhs)]
        for half in (0, 1):
            ctx = qcd.Context(params=qcd.default_params(sap_half=half), stream=stream.cuda_stream)
            ctx.qcd_set_gauge(U, dims, -1.1, 1.7)
            x = torch.zeros_like(b)
            ctx.qcd_sap(qcd.QCD_OP_D, qcd.QCD_FP32, nrhs, b, x, taus, 1, 0.1)     # warm-up
            torch.cuda.synchronize()
            qcd.qcd_stats_reset(1)
            for _ in range(reps):
                x.zero_()
                ctx.qcd_sap(qcd.QCD_OP_D, qcd.QCD_FP32, nrhs, b, x, taus, 1, 0.1)
            torch.cuda.synchronize()
            st = {r["name"]: r for r in qcd.qcd_stats_read()}
            work = qcd.qcd_stats_sap_work()
            name = "sap_block_f32h" if half else "sap_block_f32"
            r = st[name]
            fl = sap_flops(*work)
            out[f"nrhs{nrhs}_{'fp16' if half else 'fp32'}_basis"] = {
                "us_per_launch": r["total_ms"] * 1e3 / max(1, r["launches"]), "launches": r["launches"],
                "block_solves_per_launch": V // 16 // 2 * nrhs,
                "gmres_steps_per_solve": work[0] / (r["launches"] * (V // 2) * nrhs),
                "tflops": fl / (r["total_ms"] * 1e-3) / 1e12, "frac_fp32_fma": fl / (r["total_ms"] * 1e-3) / 1e12 / peak}
            ctx.close()
    qcd.qcd_stats_reset(0)
    return out


def stencil_bench(qcd, synth, torch, devn, stream, peak):
    """Fine Wilson-clover stencil (D - tau Gamma5) on a 64 x 32^3 field (inputs
    far larger than L2): FP32 and FP64 with one right-hand side, and FP32 with
    8 and 16 right-hand sides in one launch (links and clover read once per
    group of right-hand sides).  Algorithmic bytes per site and right-hand side:
    in + out spinor (48 reals) plus links and clover (144 reals) over the
    right-hand sides that share them -- 768 B (FP32) and 1536 B (FP64) at one
    right-hand side, (48 + 144 / nrhs) x 4 B in FP32 with nrhs of them."""
    dims = (64, 32, 32, 32)
    U = synth.gauge_field(dims, 0.6, 1004)
    ctx = qcd.Context(stream=stream.cuda_stream)
    ctx.qcd_set_gauge(U, dims, -0.5, 1.9)
    V = int(np.prod(dims))
    out = {"lattice": "64x32^3", "sites": V}
    for prec, name, dt, real, nrhs in ((1, "fp32", torch.complex64, 4, 1), (0, "fp64", torch.complex128, 8, 1),
                                       (1, "fp32_nrhs8", torch.complex64, 4, 8),
                                       (1, "fp32_nrhs16", torch.complex64, 4, 16)):
        x = torch.randn(V * 12 * nrhs, dtype=dt, device=devn)
        y = torch.empty_like(x)
        taus = [0.0] * nrhs
        for _ in range(3):
            ctx.qcd_apply(qcd.QCD_OP_D, prec, nrhs, x, y, taus)
        reps = 20 if nrhs == 1 else 5
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            ctx.qcd_apply(qcd.QCD_OP_D, prec, nrhs, x, y, taus)
        e1.record(stream)
        e1.synchronize()
        t = e0.elapsed_time(e1) / reps * 1e-3
        bps = (48.0 + 144.0 / nrhs) * real          # per site and right-hand side
        gbs = bps * V * nrhs / t / 1e9
        out[name] = {"nrhs": nrhs, "us_per_apply": t * 1e6, "gbs": gbs, "frac_hbm": gbs / peak,
                     "gflops": 1824 * V * nrhs / t / 1e9, "bytes_per_site_rhs": bps}
        del x, y
    ctx.close()
    return out


if __name__ == "__main__":
    main()
