#!/usr/bin/env python
"""KKT solves/s and p99 latency of the parallel Riccati tree on one GB300,
against the plain per-instance serial Riccati recursion on the same GPU, at a
relative KKT residual <= 1e-8.

Workloads (seeded, synthetic; shapes and distributions of the paper's MHE
problems):
  batch (default)  4096 MHE instances, nx ~ U{6, 12, 24}, nw = ny = nx / 2,
                   UFTOC horizon N ~ U[32, 2048]; FP32 tree + refinement
                   against the FP64 KKT residual.
  long             one instance nx = 20, nw = ny = 10, N = 131072, FP64.
A step is the whole hot path over the workload: per shape bucket the stage
assembly (Section II) and the factor + solve + refinement of the tree.

Arms: default = the CUDA library; --impl reference = the serial FP64 CPU
oracle on a bounded sample of the same workload (host cores).
"""
from __future__ import annotations

import argparse
import json
import os

# the host pipeline of the end-to-end arm runs a stream per piece and shape bucket (up to
# ~30): give them as many hardware work queues as the device offers, so that streams do
# not share a queue and wait on each other's unrelated work (set before CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1510_03110_gb300 import synth  # noqa: E402

METRIC = "KKT solves/s and p99 latency vs plain batched serial Riccati, same GPU, rel-res<=1e-8"
RELRES_BAR = 1e-8
LONG_N = 131072   # horizon of the long workload (--N)


def flops_leaf_stage(n, m):
    """Algorithm 4 per stage (matrix and vector part), the count used for the roofline."""
    return 6 * n ** 3 + 12 * n ** 2 * m + 6 * n * m ** 2 + m ** 3 / 3.0


def pass_model(ph, lvl, n, m, q, prec, N, serial=False, df=False):
    """Algorithmic work of one full pass of a level-0 kernel over a bucket:
    (bound, work, unit) with work in TFLOP or GB.  The counts:
      reduce  Algorithm 4 per stage (flops_leaf_stage; the arrival stage has width n)
      resid   FP64 FMAs of the KKT rows per stage: dynamics A x + B w, costate
              A^T lam + B^T lam, and Q z in the MHE factors (FP32_IR: C x, V u, S^T w,
              C^T e, W w, S u) or with the assembled Q (FP64); the double-float form (default
              in the mixed precisions) by its bytes instead: the stage matrices as pairs,
              l, a and the iterate in FP64, the FP32 correction rows written
      prep    bytes: FP64 A, B, C, R, a, y~, w~ read; FP32 A, B, Q, a, l and FP64 l written, and with
              the double-float residual the float pairs of A, B, C, R (FP64 mode: C, R, y~, w~ read,
              FP64 Q, l written)
      rhs     bytes: stored P, chol(G), K and FP32 A, B, a, l read per stage
      down    bytes: stored K, k, L and FP32 A, B, Q, a, l read; x, w, lam written (FP32)
              and accumulated into FP64 z"""
    stages = int(np.sum(N))
    inst = len(N)
    if lvl != 0:
        return None
    if ph == "reduce":
        f = flops_serial_stage if serial else flops_leaf_stage   # a serial plan runs Algorithms 1-2 only
        fl = stages * f(n, m) - inst * (f(n, m) - f(n, n))
        return ("alu", fl / 1e12, "TFLOP/s")
    if ph == "resid":
        if prec == 1 and df:
            # double-float residual (FP32 pipes): bound by memory; its algorithmic bytes are the
            # stage matrices (float pairs: 8 bytes a value as in FP64), l, a and the iterate's
            # x_t, w_t, lambda_t, lambda_t+1, x_t+1 in FP64, and the FP32 correction rows written
            b = 8 * (n * n + n * m + q * n + (m + q) ** 2) + 8 * (n + m + n) + 8 * (4 * n + m) + 4 * (2 * n + m)
            return ("hbm", b * stages / 1e9, "GB/s")
        qz = (2 * n * q + q * q + q * m + m * m + m * q) if prec == 1 else (n + m) ** 2
        fma = qz + 2 * (n * n + n * m)
        return ("alu", 2.0 * fma * stages / 1e12, "TFLOP/s")
    if ph == "prep":
        if prec == 1:
            b = 8 * (n * n + n * m + q * n + (m + q) ** 2 + n + q + m) + 4 * (n * n + n * m + (n + m) ** 2 + 2 * n + m) \
                + 8 * (n + m)
            if df:   # the residual's float pairs: lo of A, B; hi and lo of C, R
                b += 4 * (n * n + n * m + 2 * q * n + 2 * (m + q) ** 2)
        else:
            b = 8 * (q * n + (m + q) ** 2 + q + m) + 8 * ((n + m) ** 2 + n + m)
        return ("hbm", b * stages / 1e9, "GB/s")
    ts = 4 if prec == 1 else 8
    if ph == "rhs":
        return ("hbm", ts * (2 * n * n + m * m + 2 * m * n + 2 * n + m) * stages / 1e9, "GB/s")
    if ph == "down":
        b = ts * (2 * m * n + m + n * n + n * m + (n + m) ** 2 + 2 * n + m + 3 * n + m)
        if prec == 1:
            b += 2 * 8 * (2 * n + m)
        return ("hbm", b * stages / 1e9, "GB/s")
    return None


def flops_serial_stage(n, m):
    """Algorithms 1-3 per stage."""
    return 4 * n ** 3 + 6 * n ** 2 * m + 4 * n * m ** 2 + m ** 3 / 3.0


# ---------------------------------------------------------------- workload

def make_workload(name):
    if name == "batch":
        w = synth.batch_uneven(seed=3)
        desc = dict(workload="batched uneven MHE instances", instances=4096, nx="U{6,12,24}",
                    nw_ny="nx/2", N="U[32,2048] (UFTOC horizon)", precision="FP32 tree + FP64 refinement",
                    seed=3, l2="inputs larger than L2 (tens of GB resident)")
        buckets = []
        for n, b in sorted(w["buckets"].items()):
            buckets.append(dict(n=n, m=b["m"], q=b["q"], N=b["N"], pool=b["pool"], idx=b["idx"], x0=b["x0"]))
        return desc, buckets, 1   # prec FP32_IR
    if name == "profile":
        # a small case of the same kernels for ncu captures: 192 instances of nx = 24
        w = synth.batch_uneven(seed=5, count=192, nx_choices=(24,))
        desc = dict(workload="profile case: 192 batched uneven MHE instances", instances=192, nx=24,
                    nw_ny=12, N="U[32,2048] (UFTOC horizon)", precision="FP32 tree + FP64 refinement",
                    seed=5, l2="inputs larger than L2 (a few GB)")
        b = w["buckets"][24]
        return desc, [dict(n=24, m=12, q=12, N=b["N"], pool=b["pool"], idx=b["idx"], x0=b["x0"])], 1
    if name in ("xl", "xl_profile"):
        # 256 instances of nx = 64, nw = ny = 32, N = 1024 (262,144 stages); stages drawn from a seeded pool of
        # 2048 independent stages (the eigenvalue scaling of 64 x 64 draws dominates generation time).
        # xl_profile: 32 instances of N = 256, the ncu case of the same kernels
        rng = np.random.default_rng(5)
        count, N, n, m = (256, 1024, 64, 32) if name == "xl" else (32, 256, 64, 32)
        pool = synth.stage_pool(np.random.default_rng([5, n]), n, m, m, 2048)
        idx = rng.integers(0, 2048, size=count * (N - 1))
        x0 = rng.standard_normal((count, n))
        desc = dict(workload=f"{count} MHE instances of nx=64, nw=ny=32, N={N}", instances=count, nx=n, nw_ny=m,
                    N=N, precision="FP32 tree (128-thread teams) + FP64 refinement", seed=5,
                    l2="inputs larger than L2 (26 GB resident)")
        return desc, [dict(n=n, m=m, q=m, N=np.full(count, N, dtype=np.int64), pool=pool, idx=idx, x0=x0)], 1
    if name == "long":
        N = LONG_N
        p = synth.mhe_instance(1, 20, 10, 10, N)
        pool = {k: p[k] for k in ("A", "B", "C", "R", "a", "yt", "wt")}
        desc = dict(workload="long-horizon single MHE instance", instances=1, nx=20, nw=10, ny=10,
                    N=N, precision="FP64", seed=1,
                    l2="inputs larger than L2" if N * 8400 > 129e6 else "inputs smaller than L2 (L2 not flushed)")
        return desc, [dict(n=20, m=10, q=10, N=np.array([N]), pool=pool,
                           idx=np.arange(N - 1), x0=p["x0"][None, :])], 0
    raise SystemExit(f"unknown workload {name}")


def to_device(bk):
    """Pool -> device, expanded to every stage by an index gather (column-major blocks)."""
    import torch
    dev = "cuda"
    idx = torch.from_numpy(np.asarray(bk["idx"], dtype=np.int64)).to(dev)
    out = {}
    for k in ("A", "B", "C", "R"):
        pool = torch.from_numpy(synth.colmajor(bk["pool"][k]).reshape(len(bk["pool"][k]), -1)).to(dev)
        out[k] = pool.index_select(0, idx).contiguous()
        del pool
    for k in ("a", "yt", "wt"):
        pool = torch.from_numpy(np.ascontiguousarray(bk["pool"][k])).to(dev)
        out[k] = pool.index_select(0, idx).contiguous()
        del pool
    n, m = bk["n"], bk["m"]
    S = int(len(bk["idx"]))
    out["x0"] = torch.from_numpy(np.ascontiguousarray(bk["x0"]).reshape(-1)).to(dev)
    out["P0inv"] = torch.eye(n, dtype=torch.float64, device=dev).reshape(1, -1).repeat(len(bk["N"]), 1).contiguous()
    out["S"] = S
    return out


# ---------------------------------------------------------------- clocks

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(parts)
            except Exception:
                pass
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                    reasons=sorted(reasons), samples=len(rows))


def clocks_check(clk):
    """The timing rule on clocks: a run that saw a hardware or thermal slowdown, or
    SM clocks well below their maximum with no reason given (a leftover clock
    lock), is not a valid measurement; the power cap is kept and noted."""
    if not clk or not clk.get("samples"):
        return "no clock samples"
    bad = [r for r in clk["reasons"] if r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")]
    if bad:
        return "rejected: " + ", ".join(bad)
    sm, mx = clk.get("sm_mhz"), clk.get("sm_max_mhz")
    if sm and mx and sm < 0.9 * mx and not clk["reasons"]:
        return "rejected: SM clock %.0f of %.0f MHz with no reason active" % (sm, mx)
    return "ok (sw_power_cap active, noted)" if "sw_power_cap" in clk["reasons"] else "ok"


# ---------------------------------------------------------------- GPU arm

def peaks():
    p = {}
    try:
        p = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(p.get("sm_max_mhz", 2070.0))
    return dict(hbm_gbs=float(p.get("hbm_gbs", 6800.0)), sm_max_mhz=sm_max,
                src="measured" if p else "fallback",
                # ALU peaks from unit counts x clock: 152 SMs x 128 FP32 lanes x 2 flop x clock;
                # FP64: the part's nominal 1.25 TFLOP/s
                fp32_tflops=152 * 128 * 2 * sm_max * 1e6 / 1e12, fp64_tflops=1.25,
                bf16_tflops=float(p.get("bf16_tflops", 1900.0)))


# FP64 and FP32 FMA throughput of the GPU (the ALU roofline denominators next to the
# measured HBM and BF16 peaks): every thread runs eight independent FMA chains, 8 CTAs
# of 256 threads per SM, best of two timed runs after a warm-up (CUDA events).
ALU_PROBE = r"""
#include <cstdio>
#include <cuda_runtime.h>
template <typename T>
__global__ void k_fma(T* out, int iters, T a, T b)
{
    T x0 = threadIdx.x, x1 = x0 + 1, x2 = x0 + 2, x3 = x0 + 3, x4 = x0 + 4, x5 = x0 + 5, x6 = x0 + 6, x7 = x0 + 7;
    for (int i = 0; i < iters; ++i) {
        x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
        x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = x0 + x1 + x2 + x3 + x4 + x5 + x6 + x7;
}
template <typename T>
static double tflops(int blocks, int threads, int iters)
{
    T* out = nullptr;
    if (cudaMalloc(&out, sizeof(T) * blocks * threads) != cudaSuccess) return -1.0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0);
        k_fma<T><<<blocks, threads>>>(out, iters, (T)0.999999, (T)1e-7);
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaFree(out);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return 2.0 * 8.0 * (double)iters * blocks * threads / (best * 1e-3) / 1e12;
}
int main()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = sms * 8, threads = 256;
    const double f64 = tflops<double>(blocks, threads, 20000);
    const double f32 = tflops<float>(blocks, threads, 160000);
    const cudaError_t err = cudaGetLastError();
    printf("{\"fp64_tflops\": %.4f, \"fp32_tflops\": %.4f, \"sm_count\": %d, \"status\": \"%s\"}\n", f64, f32,
           sms, cudaGetErrorString(err));
    return err == cudaSuccess ? 0 : 1;
}
"""


def run_alu_peaks():
    """Compile and run the FMA probe (one GPU); prints its JSON line."""
    from paper_1510_03110_gb300.build import ARCH, nvcc
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "alu_peaks.cu"), os.path.join(d, "alu_peaks")
        open(src, "w").write(ALU_PROBE)
        subprocess.run([nvcc(), "-O3", *ARCH, "-o", exe, src], check=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        sys.stdout.write(r.stdout)
        sys.stderr.write(r.stderr)
        return r.returncode


def read_traffic():
    """DRAM bytes per stage of the leaf reduction from the committed ncu summary (or None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                try:
                    out[k.strip()] = float(v.split()[0])
                except Exception:
                    pass
    return out


def run_gpu(args):
    import torch
    from paper_1510_03110_gb300 import build, mhe
    build.build()
    torch.cuda.set_device(0)
    desc, buckets, prec = make_workload(args.workload)
    # the Solver's precision: MHE_TF32_IR puts the reductions' stage products on the tensor cores
    sprec = prec
    if prec == 1 and (args.prec == "tf32" or (args.prec == "auto" and args.workload in ("xl", "xl_profile"))):
        sprec = mhe.MHE_TF32_IR
        desc["precision"] = ("FP32 tree (128-thread teams), stage products F, G, H on the tensor cores "
                             "(tcgen05 kind::tf32, operands split hi + lo, FP32 accumulation) + FP64 refinement")
    elif prec == 1 and args.prec == "bf16":
        sprec = mhe.MHE_BF16_IR
        desc["precision"] = ("FP32 tree (128-thread teams), stage products F, G, H on the tensor cores "
                             "(tcgen05 kind::f16, BF16 operands split hi + mid + lo, FP32 accumulation) "
                             "+ FP64 refinement")
    t0 = time.time()
    for bk in buckets:
        bk["dev"] = to_device(bk)
    gen_s = time.time() - t0
    refine_tol = args.refine_tol
    max_refine = 16 if prec == 1 else 2
    solvers, plans = [], []
    stream = torch.cuda.current_stream()
    bstreams = [torch.cuda.Stream() for _ in buckets]
    t_tune = time.time()
    for bk in buckets:
        plan = dict(leaf_len=16 if prec == 0 else 8, branching=8 if prec == 0 else 4, top_len=4)
        if bk["n"] in args.serial_nx:
            plan = dict(leaf_len=plan["leaf_len"], branching=plan["branching"], top_len=int(np.max(bk["N"])) + 1)
        elif args.plan:
            lf, br, tp = (int(v) for v in args.plan.split(","))
            plan = dict(leaf_len=lf, branching=br, top_len=tp)
        elif args.autotune:
            # the library's autotuner on the first instances of the bucket (a contiguous prefix)
            d = bk["dev"]
            # a prefix of the bucket; nx = 64 tunes on the whole batch (its instances fill the SMs, which
            # changes the best plan, and 256 instances are a small batch)
            k = min(len(bk["N"]), args.tune_instances if bk["n"] < 48 else len(bk["N"]))
            S = int(np.sum(bk["N"][:k] - 1))
            n, m = bk["n"], bk["m"]
            dims, _keep = mhe.make_dims(n, m, bk["N"][:k], sprec, 0, 0, 0, refine_tol, max_refine)
            Qp = torch.empty(max(S, 1), (n + m) ** 2, dtype=torch.float64, device="cuda")
            lp = torch.empty(max(S, 1), n + m, dtype=torch.float64, device="cuda")
            if S > 0:
                mhe.mhe_assemble(n, m, bk["q"], d["C"][:S].contiguous(), d["R"][:S].contiguous(),
                                 d["yt"][:S].contiguous(), d["wt"][:S].contiguous(), Qp, lp)
            r = mhe.mhe_autotune(dims, d["A"][:S].contiguous(), d["B"][:S].contiguous(), Qp,
                                 d["P0inv"][:k].contiguous(), lp, d["a"][:S].contiguous(),
                                 d["x0"][:k * n].contiguous())
            del Qp, lp
            plan = dict(leaf_len=r["leaf_len"], branching=r["branching"], top_len=r["top_len"],
                        down_pass=r["down_pass"], team=r["team"])
        plans.append(dict(nx=bk["n"], **plan))
        s = mhe.Solver(bk["n"], bk["m"], bk["N"], prec=sprec, refine_tol=refine_tol,
                       max_refine=max_refine, stream=bstreams[len(solvers)],
                       fp64_masters=args.fp64_masters and prec == 1, **plan)
        mhe.mhe_set_double_float_residual(s.ctx, not args.fp64_residual)
        s.out = s.outputs()
        solvers.append(s)
    tune_s = time.time() - t_tune

    def step(ss, timing=False):
        # one stream per shape bucket, forked from and joined back into the timed stream:
        # the buckets' kernels overlap (one bucket's tails and small upper levels leave SMs idle)
        fork = torch.cuda.Event()
        fork.record(stream)
        for bk, s, st in zip(buckets, ss, bstreams):
            d = bk["dev"]
            st.wait_event(fork)
            # steps a0..a7 from the MHE data (stage assembly inside the library)
            s.estimate(bk["q"], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"],
                       out=s.out)
        for st in bstreams:
            stream.wait_stream(st)

    def step_serial(ss):
        # the same step with the buckets one after another
        prev = torch.cuda.Event()
        prev.record(stream)
        for bk, s, st in zip(buckets, ss, bstreams):
            d = bk["dev"]
            st.wait_event(prev)
            s.estimate(bk["q"], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"], d["x0"], d["P0inv"],
                       out=s.out)
            prev = torch.cuda.Event()
            prev.record(st)
        stream.wait_event(prev)

    for _ in range(args.warmup):
        step(solvers)
    torch.cuda.synchronize()
    launches0 = sum(mhe.mhe_launch_count(s.ctx) for s in solvers) + mhe.mhe_assemble_count()
    clocks = Clocks()
    clocks.start()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # per-pass CUDA events on the contexts' stream during the timed steps (the roofline's durations)
    for s in solvers:
        mhe.mhe_timing_read(s.ctx)
        mhe.mhe_timing_enable(s.ctx, True)
    torch.cuda.synchronize()
    t_host = time.time()
    torch.cuda.nvtx.range_push("timed")
    for i in range(args.steps):
        evs[i][0].record(stream)
        step(solvers)
        evs[i][1].record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    wall = time.time() - t_host
    clk = clocks.stop()
    if clk:
        clk["rule"] = clocks_check(clk)
    launches = sum(mhe.mhe_launch_count(s.ctx) for s in solvers) + mhe.mhe_assemble_count() - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms = sum(step_ms) / len(step_ms)
    instances = int(sum(len(bk["N"]) for bk in buckets))
    infos = np.concatenate([s.infos() for s in solvers])
    relres_max = float(np.max(infos["relres"]))
    ok = bool(np.all(infos["status"] == 0) and relres_max <= RELRES_BAR)

    # per-pass timing of the timed steps: the dominant kernel and its roofline
    passes = []
    for bk, s in zip(buckets, solvers):
        for (ph, lvl, calls, tms, tmax) in mhe.mhe_timing_read(s.ctx):
            passes.append(dict(nx=bk["n"], phase=ph, level=lvl, calls=calls // args.steps,
                               ms=tms / args.steps, ms_max=tmax))
        mhe.mhe_timing_enable(s.ctx, False)
    pk = peaks()
    traffic = read_traffic()
    kern = {"reduce": "k_level<{t},{n},{m},0,%s>" % {2: "REDUCE_TC", 3: "REDUCE_BF"}.get(sprec, "REDUCE"),
            "rhs": "k_level<{t},{n},{m},0,RHS>",
            "down": "k_level<{t},{n},{m},0,DOWN>",
            "resid": "k_resid<{n},{m},{t},{y}>" if (args.fp64_residual or prec == 0) else "k_resid_df<{n},{m},{y}>",
            "prep": "k_prep<{n},{m},{q}>" if prec == 1 else "k_assemble<{n},{m},{q}>"}

    def roof(r):
        bk = [b for b in buckets if b["n"] == r["nx"]][0]
        n, m, q = bk["n"], bk["m"], bk["q"]
        pl = [p for p in plans if p["nx"] == n][0]
        mod = pass_model(r["phase"], r["level"], n, m, q, prec, bk["N"], serial=pl["top_len"] > int(np.max(bk["N"])),
                         df=not args.fp64_residual)
        if mod is None:
            return None
        bound, work, unit = mod
        full_ms = r["ms_max"]   # the longest pass covers every instance
        achieved = work / (full_ms * 1e-3)
        if bound == "hbm":
            peak, src = pk["hbm_gbs"], "HBM copy bandwidth, %s" % pk["src"]
        elif r["phase"] == "resid" or prec == 0:
            peak, src = pk["fp64_tflops"], "FP64: nominal 1.25 TFLOP/s of the part (a DFMA probe reaches 1.256)"
        else:
            peak, src = pk["fp32_tflops"], "FP32: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % pk["sm_max_mhz"]
        tkey = f"{r['phase']}_nx{n}_{'fp32' if prec == 1 else 'fp64'}_bytes_per_stage"
        tr = traffic.get(tkey)
        name = kern[r["phase"]].format(t="float" if prec == 1 else "double", n=n, m=m, q=q,
                                       y=(q if prec == 1 else 0))
        out = dict(bound=bound, kernel=name, achieved=round(achieved, 3), peak=round(peak, 2), unit=unit,
                   frac=round(achieved / peak, 4), traffic=(tr * int(np.sum(bk["N"])) if tr else None),
                   peak_src=src, work_per_launch=work, ms_per_launch=round(full_ms, 4),
                   launches_per_step=r["calls"], ms_per_step=round(r["ms"], 4))
        if r["phase"] == "reduce" and sprec in (2, 3) and n == 64:
            # the tensor pipe's view: MMA flops issued per stage (M = 128 rows; TF32: N = 2k + k per
            # product for the hi/lo split, against TF32 = the measured BF16 peak x 1.1 / 2.25; BF16:
            # N = 2k + k + 2k + k for the three-way split, against the measured BF16 peak)
            mma = (3 if sprec == 2 else 6) * 2 * 128 * n * (n + (n + m)) * int(np.sum(bk["N"]))
            tf = pk["bf16_tflops"] * (1.1 / 2.25 if sprec == 2 else 1.0)
            out["tensor"] = dict(mma_tflop_per_launch=mma / 1e12, achieved=round(mma / 1e12 / (full_ms * 1e-3), 2),
                                 peak=round(tf, 1), unit="TFLOP/s", frac=round(mma / 1e12 / (full_ms * 1e-3) / tf, 4),
                                 peak_src=("TF32 dense = measured BF16 burst x 1.1 / 2.25 (nominal ratio)"
                                           if sprec == 2 else "BF16 dense, measured burst"))
        return out

    ranked = sorted(passes, key=lambda r: -r["ms"])
    kernels = [x for x in (roof(r) for r in ranked[:6]) if x]
    roofline = kernels[0] if kernels else None

    # every pass once more with the buckets one after another (no stream overlap): the
    # per-kernel roofline fractions of kernels[] (the timed step overlaps the buckets, so
    # there a kernel's pass time includes the SMs the other buckets hold)
    kernels_serial = []
    if len(buckets) > 1:
        for s in solvers:
            mhe.mhe_timing_read(s.ctx)
            mhe.mhe_timing_enable(s.ctx, True)
        step_serial(solvers)
        torch.cuda.synchronize()
        spasses = []
        for bk, s in zip(buckets, solvers):
            for (ph, lvl, calls, tms, tmax) in mhe.mhe_timing_read(s.ctx):
                spasses.append(dict(nx=bk["n"], phase=ph, level=lvl, calls=calls, ms=tms, ms_max=tmax))
            mhe.mhe_timing_enable(s.ctx, False)
        kernels_serial = [x for x in (roof(r) for r in sorted(spasses, key=lambda r: -r["ms"])[:8]) if x]
    else:
        kernels_serial = kernels

    # error against the FP64 oracle on sampled instances (the oracle solves each one on the
    # host) and the library's own per-instance estimate (the last correction's size) for all
    err_oracle = sample_errors(buckets, solvers, per_bucket=args.err_samples)
    est = np.asarray(infos["est_relerr"], dtype=np.float64)
    est_summary = dict(max=float(est.max()), p50=float(np.median(est)), p99=float(np.quantile(est, 0.99)),
                       instances=int(est.size),
                       note="mhe_info.est_relerr = ||dz_last||_inf / ||z||_inf of the last correction, per instance")

    # plain serial Riccati on the same GPU: one chunk per instance (top_len >= N)
    base = {}
    xl = args.workload in ("xl", "xl_profile")
    tree_plans = [dict(nx=b["n"], leaf_len=16, branching=4, top_len=4) for b in buckets]
    short_plans = [dict(nx=b["n"], leaf_len=8, branching=4, top_len=4) for b in buckets]
    # (name, precision, corrections, plans (None: serial), FP64 master levels)
    arms = [] if args.no_baseline else [("serial_same_precision", sprec, max_refine if prec == 1 else 0, None, 0)] + \
        ([("serial_fp64", 0, 2, None, 0)] if (prec == 1 and (args.serial_fp64 or xl)) else []) + \
        ([("tree_fp64", 0, 2, tree_plans, 0)] if (prec == 1 and xl) else []) + \
        ([("tree_short_leaves_fp64_masters", sprec, max_refine, short_plans, 1),
          ("tree_short_leaves_fp32_masters", sprec, max_refine, short_plans, 0)] if (prec == 1 and xl) else []) + \
        ([("fp32_simt_products_same_plan", 1, max_refine, plans, 0)] if sprec in (2, 3) else [])
    # the headline's own plans with each context's launch sequence replayed as a CUDA graph
    arms = [a + (False,) for a in arms] + \
        ([] if args.no_baseline else [("same_plans_cuda_graph", sprec, max_refine, plans, int(args.fp64_masters), True)])
    for name, bprec, mref, bplans, m64, graph in arms:
        ss = []
        for i, bk in enumerate(buckets):
            bpl = dict(top_len=int(np.max(bk["N"])) + 1) if bplans is None else \
                {k: v for k, v in bplans[i].items() if k != "nx"}
            s = mhe.Solver(bk["n"], bk["m"], bk["N"], prec=bprec, refine_tol=refine_tol, max_refine=mref,
                           stream=bstreams[i], fp64_masters=bool(m64), **bpl)
            mhe.mhe_set_double_float_residual(s.ctx, not args.fp64_residual)
            if graph:
                s.set_graph(True)
            s.out = s.outputs()
            ss.append(s)
        for _ in range(2 if graph else 1):   # graphs: one eager call, then the capture
            step(ss)
        torch.cuda.synchronize()
        k = max(1, min(args.steps, args.baseline_steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            step(ss)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / k
        binf = np.concatenate([s.infos() for s in ss])
        base[name] = dict(value=round(instances / (bms * 1e-3), 3), ms_per_step=round(bms, 3),
                          relres_max=float(np.max(binf["relres"])), steps=k,
                          all_ok=bool(np.all(binf["status"] == 0)),
                          refine_iters_max=int(np.max(binf["refine_iters"])),
                          precision={0: "FP64", 1: "FP32+IR", 2: "TF32+IR", 3: "BF16+IR"}[bprec] +
                          (" + FP64 master levels" if m64 else ""),
                          plan="serial" if bplans is None else {k: v for k, v in bplans[0].items() if k != "nx"},
                          cuda_graph=graph)
        for s in ss:
            s.close()

    # end to end: inputs from pinned host memory every step, the solution back to the host
    e2e = None
    if args.e2e:
        e2e = run_e2e(args, buckets, solvers, step, stream, instances)

    cpu = cpu_baseline(buckets, args) if not args.no_cpu else None
    serving = None
    if args.serve_duration > 0:
        # free the batch workload first: the serving run holds its own windows
        for s_ in solvers:
            s_.close()
        solvers = []
        for bk in buckets:
            bk.pop("dev", None)
        torch.cuda.empty_cache()
        sa = argparse.Namespace(**vars(args))
        sa.duration = args.serve_duration
        serving = run_serve(sa)
    value = instances / (ms * 1e-3)
    step_sorted = sorted(step_ms)
    p99 = step_sorted[min(len(step_sorted) - 1, int(np.ceil(0.99 * len(step_sorted))) - 1)]
    line = dict(metric=METRIC, value=round(value, 3), unit="KKT solves/s", n_gpus=1, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(ms, 4), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype={2: "tf32+f32+f64", 3: "bf16+f32+f64"}.get(sprec, "f32+f64") if prec == 1 else "f64",
                data="synthetic",
                config=dict(desc, refine_tol=refine_tol, relres_bar=RELRES_BAR, fp64_master_levels=bool(args.fp64_masters),
                            residual="FP64 instructions" if (args.fp64_residual or prec == 0) else
                            "double-float (float pairs on the FP32 pipes)",
                            generation_s=round(gen_s, 1),
                            plans=plans, autotune_s=round(tune_s, 1)),
                latency_ms=dict(p50=round(statistics.median(step_ms), 4), p99=round(p99, 4),
                                note="one step solves every instance; latency = step time"),
                relres_max=relres_max, all_ok=ok,
                refine_iters_max=int(np.max(infos["refine_iters"])),
                serial_gpu=base,
                speedup_vs_serial=dict({k: round(value / v["value"], 2) for k, v in base.items()},
                                       **({} if serving is None else dict(
                                           serving_solves_per_s=round(serving["tree_reuse"]["solves_per_s"] /
                                                                      max(serving["serial"]["solves_per_s"], 1e-9), 2),
                                           serving_p99=round(serving["serial"]["p99_ms"] /
                                                             max(serving["tree_reuse"]["p99_ms"], 1e-9), 2)))),
                serving=serving,
                err_vs_oracle=err_oracle, est_relerr=est_summary,
                roofline=roofline, kernels=kernels_serial, kernels_overlapped=kernels[1:],
                passes=sorted(passes, key=lambda r: -r["ms"])[:8],
                cpu_baseline=cpu, e2e=e2e, gpu_launches=int(launches), clocks=clk,
                wall_s=round(wall, 3))
    print(json.dumps(line))
    for s in solvers:
        s.close()


def sample_errors(buckets, solvers, per_bucket=2, seed=13):
    """max over sampled instances of ||z - z_oracle||_inf / ||z_oracle||_inf per block (x, w,
    lambda): the GPU solution of each sampled instance against the FP64 oracle (plain C)."""
    import oracle
    rng = np.random.default_rng(seed)
    rows = []
    for bk, s in zip(buckets, solvers):
        n, m, q = bk["n"], bk["m"], bk["q"]
        Nb = np.asarray(bk["N"])
        offs = np.concatenate([[0], np.cumsum(Nb - 1)])
        xo = np.concatenate([[0], np.cumsum(Nb + 1)])
        wo = np.concatenate([[0], np.cumsum(n + (Nb - 1) * m)])
        x, w, lam = s.out
        for j in rng.choice(len(Nb), size=min(per_bucket, len(Nb)), replace=False):
            p = synth.instance_from_pool(bk["pool"], bk["idx"][offs[j]:offs[j + 1]], bk["x0"][j], n, m, q)
            ref = oracle.riccati(oracle.mhe_to_uftoc(p))
            got = dict(x=x[xo[j]:xo[j + 1]].cpu().numpy(), lam=lam[xo[j]:xo[j + 1]].cpu().numpy(),
                       w=w[wo[j]:wo[j + 1]].cpu().numpy())
            e = 0.0
            for k in ("x", "w", "lam"):
                a, b = np.asarray(got[k]).ravel(), np.asarray(ref[k]).ravel()
                e = max(e, float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)))
            rows.append(dict(nx=n, instance=int(j), N=int(Nb[j]), rel_err=e))
    return dict(max=max(r["rel_err"] for r in rows) if rows else None, samples=rows,
                definition="max over x, w, lambda of ||z - z_oracle||_inf / ||z_oracle||_inf")


def run_long_sweep(args):
    """Depth scaling of the tree on one long horizon (nx = 20, nw = ny = 10, FP64): N in
    {1024, 16384, 131072} (prefixes of one seeded instance) x leaf_len in {8, 16, 32, 64} x
    branching in {2, 4, 8, 16} (top_len 4), and the serial recursion (top_len > N) at each N.
    Per plan: levels, ms per solve (CUDA events, best of the timed repetitions), relres, the
    level-0 reduction's FP64-pipe fraction; per N the error of the fastest plan against the
    FP64 oracle."""
    import torch

    import oracle
    from paper_1510_03110_gb300 import build, mhe
    build.build()
    torch.cuda.set_device(0)
    Ns = [int(v) for v in args.sweep_N.split(",")]
    leaves = [int(v) for v in args.sweep_leaf.split(",")]
    brs = [int(v) for v in args.sweep_branching.split(",")]
    n, m, q = 20, 10, 10
    t0 = time.time()
    full = synth.mhe_instance(1, n, m, q, max(Ns))
    gen_s = time.time() - t0
    pk = peaks()
    stream = torch.cuda.current_stream()
    rows = []
    for N in Ns:
        p = dict(full, N=N, **{k: full[k][:N - 1] for k in ("A", "B", "C", "R", "a", "yt", "wt")})
        bk = dict(n=n, m=m, q=q, N=np.array([N]), pool={k: p[k] for k in ("A", "B", "C", "R", "a", "yt", "wt")},
                  idx=np.arange(N - 1), x0=p["x0"][None, :])
        d = to_device(bk)
        S = N - 1
        Q = torch.empty(S, (n + m) ** 2, dtype=torch.float64, device="cuda")
        l = torch.empty(S, n + m, dtype=torch.float64, device="cuda")
        mhe.mhe_assemble(n, m, q, d["C"], d["R"], d["yt"], d["wt"], Q, l)
        plans = [(lf, br, 4) for lf in leaves for br in brs] + [(16, 4, N + 1)]
        best = None
        for (lf, br, top) in plans:
            s = mhe.Solver(n, m, [N], prec=mhe.MHE_FP64, leaf_len=lf, branching=br, top_len=top)
            out = s.outputs()
            reps = 1 if (top > N and N > 20000) else args.sweep_reps
            s.factor_solve(d["A"], d["B"], Q, d["P0inv"], l, d["a"], d["x0"], out=out)   # warm-up
            torch.cuda.synchronize()
            mhe.mhe_timing_read(s.ctx)
            mhe.mhe_timing_enable(s.ctx, True)
            times = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.factor_solve(d["A"], d["B"], Q, d["P0inv"], l, d["a"], d["x0"], out=out)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            tim = mhe.mhe_timing_read(s.ctx)
            red0 = [r for r in tim if r[0] == "reduce" and r[1] == 0]
            ms_red0 = red0[0][3] / max(red0[0][2], 1) if red0 else None
            f = (flops_serial_stage if top > N else flops_leaf_stage)(n, m) * N
            info = s.infos()
            levels = len(mhe.mhe_plan_info(s.ctx))
            row = dict(N=N, plan="serial" if top > N else dict(leaf_len=lf, branching=br, top_len=top),
                       levels=levels, ms=round(min(times), 4), relres=float(info["relres"][0]),
                       status=int(info["status"][0]),
                       level0_reduce_ms=round(ms_red0, 4) if ms_red0 else None,
                       level0_reduce_fp64_frac=round(f / (ms_red0 * 1e-3) / 1e12 / pk["fp64_tflops"], 4)
                       if ms_red0 else None)
            rows.append(row)
            if top <= N and (best is None or row["ms"] < best[0]["ms"]):
                best = (row, [v.clone() for v in out])
            s.close()
        # the fastest plan's solution against the FP64 oracle
        ref = oracle.riccati(oracle.mhe_to_uftoc(p))
        x, w, lam = best[1]
        e = 0.0
        for k, a in (("x", x), ("w", w), ("lam", lam)):
            a = a.cpu().numpy().ravel()
            b = np.asarray(ref[k]).ravel()
            e = max(e, float(np.abs(a - b).max() / np.abs(b).max()))
        best[0]["rel_err_vs_oracle"] = e
        del d, Q, l
        torch.cuda.empty_cache()
    # the Kalman filter + RTS smoother on the GPU (the comparison of Section VI) on an instance of the same
    # sizes with uncorrelated noises (S = 0, which the smoother needs), one warp walking the horizon
    rts_rows = []
    zs = synth.mhe_instance(2, n, m, q, max(Ns), s_zero=True)
    for N in Ns:
        p = dict(zs, N=N, **{k: zs[k][:N - 1] for k in ("A", "B", "C", "R", "a", "yt", "wt")})
        bk = dict(n=n, m=m, q=q, N=np.array([N]), pool={k: p[k] for k in ("A", "B", "C", "R", "a", "yt", "wt")},
                  idx=np.arange(N - 1), x0=p["x0"][None, :])
        d = to_device(bk)
        x = torch.empty((N + 1) * n, dtype=torch.float64, device="cuda")
        w = torch.empty(n + (N - 1) * m, dtype=torch.float64, device="cuda")
        work = torch.empty(int(mhe.lib().mhe_rts_workspace_bytes(n, m, q, 1, np.array([N], np.int32).ctypes.data_as(
            __import__("ctypes").POINTER(__import__("ctypes").c_int)))), dtype=torch.uint8, device="cuda")
        call = lambda: mhe.mhe_rts_smooth(n, m, q, [N], d["A"], d["B"], d["C"], d["R"], d["a"], d["yt"], d["wt"],  # noqa: E731
                                          d["x0"], d["P0inv"], x, w, work=work)
        call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        rts_rows.append(dict(N=N, rts_ms=round(e0.elapsed_time(e1), 4)))
        del d, x, w, work
    out = dict(workload="long-horizon depth sweep, nx=20, nw=ny=10, FP64", seed=1, generation_s=round(gen_s, 1),
               fp64_peak_tflops=pk["fp64_tflops"], rows=rows, rts=rts_rows)
    summary = []
    for N in Ns:
        r = [x for x in rows if x["N"] == N]
        tree = min((x for x in r if x["plan"] != "serial"), key=lambda x: x["ms"])
        ser = [x for x in r if x["plan"] == "serial"][0]
        rt = [x for x in rts_rows if x["N"] == N][0]["rts_ms"]
        summary.append(dict(N=N, best_tree_ms=tree["ms"], best_plan=tree["plan"], levels=tree["levels"],
                            serial_ms=ser["ms"], speedup=round(ser["ms"] / tree["ms"], 2), rts_ms=rt,
                            speedup_vs_rts=round(rt / tree["ms"], 2),
                            rel_err_vs_oracle=tree.get("rel_err_vs_oracle")))
    out["summary"] = summary
    return out


def run_small(args):
    """Config 1: one instance nx = 4, nw = ny = 2, N = 64, FP64, seed 0: the latency of one
    Newton step through the C-ABI (inputs resident on the device; each solve timed with CUDA
    events and synchronised), for the tree plan, the serial plan and the allocation-free
    single-kernel entry; error against the FP64 oracle."""
    import torch

    import oracle
    from paper_1510_03110_gb300 import build, mhe
    build.build()
    torch.cuda.set_device(0)
    n, m, q, N = 4, 2, 2, 64
    p = synth.mhe_instance(0, n, m, q, N)
    ref = oracle.riccati(oracle.mhe_to_uftoc(p))
    bk = dict(n=n, m=m, q=q, N=np.array([N]), pool={k: p[k] for k in ("A", "B", "C", "R", "a", "yt", "wt")},
              idx=np.arange(N - 1), x0=p["x0"][None, :])
    d = to_device(bk)
    Q = torch.empty(N - 1, (n + m) ** 2, dtype=torch.float64, device="cuda")
    l = torch.empty(N - 1, n + m, dtype=torch.float64, device="cuda")
    mhe.mhe_assemble(n, m, q, d["C"], d["R"], d["yt"], d["wt"], Q, l)
    stream = torch.cuda.current_stream()
    K = max(args.steps, 50)
    out = {}

    def lat(fn, st=None):
        st = st if st is not None else stream
        with torch.cuda.stream(st):
            for _ in range(max(args.warmup, 3)):
                fn()
            torch.cuda.synchronize()
            ts = []
            for _ in range(K):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                fn()
                e1.record(st)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
        ts = np.array(ts)
        return dict(p50_ms=round(float(np.median(ts)), 4), p99_ms=round(float(np.quantile(ts, 0.99)), 4),
                    mean_ms=round(float(ts.mean()), 4))

    def err(x, w, lam):
        e = 0.0
        for k, a in (("x", x), ("w", w), ("lam", lam)):
            a = a.cpu().numpy().ravel()
            b = np.asarray(ref[k]).ravel()
            e = max(e, float(np.abs(a - b).max() / np.abs(b).max()))
        return e

    tree_plan, serial_plan = dict(leaf_len=4, branching=2, top_len=2), dict(top_len=N + 1)
    # the "_graph" arms replay the launch sequence as a CUDA graph (mhe_set_graph) on a stream of their own
    for name, plan, graph in [("tree", tree_plan, False), ("serial", serial_plan, False),
                              ("tree_graph", tree_plan, True), ("serial_graph", serial_plan, True)]:
        gst = torch.cuda.Stream() if graph else None
        s = mhe.Solver(n, m, [N], prec=mhe.MHE_FP64, max_refine=0, stream=gst, **plan)
        if graph:
            s.set_graph(True)
        o = s.outputs()
        r = lat(lambda: s.factor_solve(d["A"], d["B"], Q, d["P0inv"], l, d["a"], d["x0"], out=o), gst)
        r["rel_err_vs_oracle"] = err(*o)
        r["relres"] = float(s.infos()["relres"][0])
        r["levels"] = len(mhe.mhe_plan_info(s.ctx))
        r["launches_per_solve"] = mhe.mhe_launch_count(s.ctx) // (K + max(args.warmup, 3))
        out[name] = r
        s.close()
    x = torch.empty((N + 1) * n, dtype=torch.float64, device="cuda")
    w = torch.empty(n + (N - 1) * m, dtype=torch.float64, device="cuda")
    lam = torch.empty((N + 1) * n, dtype=torch.float64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    r = lat(lambda: mhe.mhe_solve_serial_noalloc(n, m, N, d["A"], d["B"], Q.reshape(-1), d["P0inv"], l.reshape(-1),
                                                 d["a"], d["x0"], x, w, lam, st))
    r["rel_err_vs_oracle"] = err(x, w, lam)
    r["launches_per_solve"] = 1
    out["single_kernel_serial"] = r
    return out


def run_ip(args):
    """MHE with box-bounded process noise (the interior-point loop, mhe_ip_solve): 256 instances of nx = 12,
    nw = ny = 6, N ~ U[32,512] (seed 6), FP64; the box around zero at half the largest |w_t[j]| of the
    unconstrained solution (the library's own solve), shifted by 10%; the plan from the library's autotuner on
    the unconstrained problem.  Timed: whole mhe_ip_solve calls in both
    methods (predictor-corrector: a factor and two solves of the tree per iteration; path following: a factor +
    solve per iteration; one host synchronisation per iteration), against the unconstrained solve of the same
    problems; checked: every input strictly inside its box, every instance converged."""
    import torch
    from paper_1510_03110_gb300 import build, mhe
    build.build()
    torch.cuda.set_device(0)
    n, m, count = 12, 6, 256
    rng = np.random.default_rng(6)
    Ns = [int(v) for v in rng.integers(32, 513, size=count)]
    insts = [synth.mhe_instance(6000 + i, n, m, m, N) for i, N in enumerate(Ns)]
    cat = lambda key, cm: np.concatenate([(synth.colmajor(p[key]) if cm else p[key]).reshape(-1)  # noqa: E731
                                          for p in insts])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()  # noqa: E731
    S = int(sum(N - 1 for N in Ns))
    A, B, C, R = t(cat("A", True)), t(cat("B", True)), t(cat("C", True)), t(cat("R", True))
    a, yt, wt = t(cat("a", False)), t(cat("yt", False)), t(cat("wt", False))
    x0 = t(np.concatenate([p["x0"] for p in insts]))
    P0 = t(np.concatenate([synth.colmajor(p["P0inv"]).reshape(-1) for p in insts]))
    Q = torch.empty(S * (n + m) ** 2, dtype=torch.float64, device="cuda")
    l = torch.empty(S * (n + m), dtype=torch.float64, device="cuda")
    mhe.mhe_assemble(n, m, m, C.view(S, -1), R, yt, wt, Q, l)
    stream = torch.cuda.Stream()
    # the plan: the library's autotuner on the unconstrained problem (a Newton step has its sizes)
    dims, _keep = mhe.make_dims(n, m, Ns, mhe.MHE_FP64)
    tuned = mhe.mhe_autotune(dims, A, B, Q, P0, l, a, x0)
    plan = {k: tuned[k] for k in ("leaf_len", "branching", "top_len", "down_pass", "team")}
    s = mhe.Solver(n, m, Ns, prec=mhe.MHE_FP64, stream=stream, **plan)
    with torch.cuda.stream(stream):
        x, w, lam = s.factor_solve(A, B, Q, P0, l, a, x0)
    stream.synchronize()
    wh = w.cpu().numpy()
    lo, hi, off = [], [], 0
    for N in Ns:
        wb = wh[off + n:off + n + (N - 1) * m].reshape(N - 1, m)
        c = 0.5 * np.maximum(np.abs(wb).max(axis=0), 1e-3)
        sh = rng.uniform(-0.1, 0.1, m) * c
        lo.append(-c + sh)
        hi.append(c + sh)
        off += n + (N - 1) * m
    lo_t, hi_t = t(np.concatenate(lo)), t(np.concatenate(hi))

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), out

    with torch.cuda.stream(stream):
        s.factor_solve(A, B, Q, P0, l, a, x0)   # warm-up
        ms_unc, _ = timed(lambda: s.factor_solve(A, B, Q, P0, l, a, x0), 5)
    stream.synchronize()

    def arm(method):
        with torch.cuda.stream(stream):
            s.ip_solve(A, B, Q, P0, l, a, x0, lo_t, hi_t, method=method)   # warm-up
            ms, (xi, wi, li, steps) = timed(lambda: s.ip_solve(A, B, Q, P0, l, a, x0, lo_t, hi_t, method=method), 3)
        stream.synchronize()
        info = s.infos()
        wi = wi.cpu().numpy()
        inside, active, off = True, 0, 0
        for b, N in enumerate(Ns):
            wb = wi[off + n:off + n + (N - 1) * m].reshape(N - 1, m)
            inside = inside and bool(np.all(wb > lo[b]) and np.all(wb < hi[b]))
            active += int(np.sum((wb - lo[b] < 1e-6 * (hi[b] - lo[b])) | (hi[b] - wb < 1e-6 * (hi[b] - lo[b]))))
            off += n + (N - 1) * m
        return dict(ms_per_ip_solve=round(ms, 3), iterations=int(steps), ms_per_iteration=round(ms / max(int(steps), 1), 3),
                    ip_solves_per_s=round(count / (ms * 1e-3), 3), all_inside_the_box=inside,
                    bounds_within_1e6_of_the_box=active, all_ok=bool(np.all(info["status"] == 0))), wi

    pc, w_pc = arm(mhe.MHE_IP_PREDICTOR_CORRECTOR)
    pf, w_pf = arm(mhe.MHE_IP_PATH_FOLLOWING)
    # the same with the context's factor and solve launches replayed as CUDA graphs
    s.set_graph(True)
    pcg, w_pcg = arm(mhe.MHE_IP_PREDICTOR_CORRECTOR)
    s.set_graph(False)
    s.close()
    pc["graph_replay"] = dict(ms_per_ip_solve=pcg["ms_per_ip_solve"], iterations=pcg["iterations"],
                              all_ok=pcg["all_ok"], same_solution=bool(np.array_equal(w_pcg, w_pc)))
    pc.update(factorisations_per_iteration=1, solves_per_iteration=2)
    pf.update(factorisations_per_iteration=1, solves_per_iteration=1)
    return dict(workload="box-bounded MHE, interior-point loop: 256 instances nx=12, nw=ny=6, N ~ U[32,512], FP64",
                instances=count, stages=S, bounded_inputs=int(S * m), plan=plan, ms_unconstrained_solve=round(ms_unc, 3),
                predictor_corrector=pc, path_following=pf,
                max_abs_w_difference_between_methods=float(np.abs(w_pc - w_pf).max()),
                speedup_predictor_corrector=round(pf["ms_per_ip_solve"] / pc["ms_per_ip_solve"], 3),
                ip_solves_per_s=pc["ip_solves_per_s"], ms_per_ip_solve=pc["ms_per_ip_solve"])


def run_link(args):
    """The host link alone, for reading the end-to-end numbers: pinned host-to-device copies of 1 GiB spread
    over a 24 GiB pinned buffer, alone, beside a 256 MiB device-to-host copy, and beside an 8 GiB memory-bound
    kernel; then `--duration` seconds of back-to-back 1 GiB copies with nothing else on the GPU."""
    import torch
    GB = 1 << 30
    H = torch.empty(24 * GB, dtype=torch.uint8, pin_memory=True)
    H.fill_(1)
    O = torch.empty(GB // 4, dtype=torch.uint8, pin_memory=True)
    D = torch.empty(24 * GB, dtype=torch.uint8, device="cuda")
    src = torch.empty(GB // 4, dtype=torch.uint8, device="cuda")
    K1 = torch.ones(2 * GB, dtype=torch.float32, device="cuda")
    K2 = torch.empty_like(K1)
    s_in, s_out, s_k = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def summary(r):
        r = np.array(r)
        return dict(copies=int(r.size), min=round(float(r.min()), 1), p1=round(float(np.percentile(r, 1)), 1),
                    p10=round(float(np.percentile(r, 10)), 1), median=round(float(np.median(r)), 1),
                    max=round(float(r.max()), 1), below_150=round(float(np.mean(r < 150)), 4))

    def spread(other=None):
        rates = []
        for _ in range(2):
            for off in range(0, 24 * GB, GB):
                if other:
                    other()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(s_in):
                    e0.record(s_in)
                    D[off:off + GB].copy_(H[off:off + GB], non_blocking=True)
                    e1.record(s_in)
                e1.synchronize()
                rates.append(GB / e0.elapsed_time(e1) / 1e6)
        torch.cuda.synchronize()
        return summary(rates)

    def d2h():
        with torch.cuda.stream(s_out):
            O.copy_(src, non_blocking=True)

    def kern():
        with torch.cuda.stream(s_k):
            torch.add(K1, 1.0, out=K2)

    out = dict(alone=spread(), beside_d2h=spread(d2h), beside_kernel=spread(kern))
    rates, stamps = [], []
    t0 = time.perf_counter()
    i = 0
    with torch.cuda.stream(s_in):
        while time.perf_counter() - t0 < args.duration:
            evs = []
            for k in range(16):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                off = ((i + k) % 16) * GB
                e0.record(s_in)
                D[(k % 2) * GB:(k % 2 + 1) * GB].copy_(H[off:off + GB], non_blocking=True)
                e1.record(s_in)
                evs.append((e0, e1))
            evs[-1][1].synchronize()
            now = time.perf_counter() - t0
            for e0, e1 in evs:
                rates.append(GB / e0.elapsed_time(e1) / 1e6)
                stamps.append(now)
            i += 16
    r, st = np.array(rates), np.array(stamps)
    series = summary(rates)
    series["seconds"] = args.duration
    series["min_per_second"] = [round(float(r[(st >= k) & (st < k + 1)].min()), 1)
                                for k in range(int(args.duration)) if np.any((st >= k) & (st < k + 1))]
    out["series"] = series
    nodes = [d for d in os.listdir("/sys/devices/system/node") if d.startswith("node")] \
        if os.path.isdir("/sys/devices/system/node") else []
    out["numa_nodes"] = len(nodes)
    return out


def serve_setup(args, rates, T, seed=4):
    """The serving workload: a pool of estimators (nx ~ U{6,12,24}, nw = ny = nx/2, N ~ U{50,200,1000}),
    for each offered rate a seeded Poisson arrival sequence over T seconds (who and when), and every
    estimator's simulated plant stream long enough for the busiest sequence (y ~ N(C x, 0.01 I),
    R = blkdiag(W, 100 I))."""
    rng = np.random.default_rng(seed)
    E = args.estimators
    nxs = rng.choice(np.array([6, 12, 24]), size=E)
    Ns = rng.choice(np.array([50, 200, 1000]), size=E)
    seqs = {}
    per_max = np.zeros(E, dtype=np.int64)
    for rate in rates:
        r2 = np.random.default_rng([seed, int(rate)])
        count = int(rate * T * 1.05) + 16
        t_arr = np.cumsum(r2.exponential(1.0 / rate, size=count))
        count = int(np.searchsorted(t_arr, T))
        who = r2.integers(0, E, size=count)
        seqs[rate] = (t_arr[:count], who)
        per_max = np.maximum(per_max, np.bincount(who, minlength=E))
    t0 = time.time()
    streams = {}
    for n in (6, 12, 24):
        ids = np.nonzero(nxs == n)[0]
        if len(ids) == 0:
            continue
        L = int(np.max(Ns[ids] - 1 + per_max[ids])) + 2
        ps = synth.plant_streams([5, n], n, n // 2, n // 2, len(ids), L)
        for j, e in enumerate(ids):
            streams[int(e)] = synth.stream_of(ps, j)
    return dict(E=E, nxs=nxs, Ns=Ns, seqs=seqs, streams=streams, T=T, gen_s=round(time.time() - t0, 1))


def serve_once(args, ws, rate, plan, reuse=True):
    """One serving run: admit every estimator, warm up with one request each, then submit the
    rate's arrival sequence at its times from this thread and wait for every result; latency is
    submission to completion as the server records it."""
    from paper_1510_03110_gb300 import mhe
    E, nxs, Ns, streams = ws["E"], ws["nxs"], ws["Ns"], ws["streams"]
    t_arr, who = ws["seqs"][rate]
    count = len(t_arr)
    nxt = np.ones(E, dtype=np.int64)   # request 0 of each estimator is the warm-up
    packed = []
    for i in range(count):
        e = int(who[i])
        st = streams[e]
        k = int(Ns[e] - 1 + nxt[e])
        nxt[e] += 1
        packed.append(mhe.pack_stage(st["A"][k], st["B"][k], st["C"][k], st["R"][k], st["a"][k], st["yt"][k],
                                     st["wt"][k]))
    srv = mhe.Server(args.serve_bytes, prec=mhe.MHE_FP32_IR, refine_tol=args.serve_tol, max_refine=args.serve_refine)
    srv.set_plan(**plan)
    srv.set_reuse(reuse)
    ids = []
    for e in range(E):
        n = int(nxs[e])
        ids.append(srv.open(synth.window_of(streams[e], 0, int(Ns[e]), np.zeros(n), n, n // 2, n // 2)))
    warm = []
    for e in range(E):
        st = streams[e]
        k = int(Ns[e] - 1)
        warm.append(srv.submit(ids[e], mhe.pack_stage(*(np.asarray(st[f][k]) for f in
                                                       ("A", "B", "C", "R", "a", "yt", "wt")))))
    for e, tk in enumerate(warm):
        srv.wait(tk, int(nxs[e]), timeout=300)
    s0 = srv.stats()
    tickets = []
    tstart = time.perf_counter()
    for i in range(count):
        target = tstart + t_arr[i]
        while time.perf_counter() < target:
            pass
        tickets.append(srv.submit(ids[int(who[i])], packed[i]))
    t_sub_end = time.perf_counter()
    lat, statuses, relres, iters = [], {}, 0.0, 0
    for i, tk in enumerate(tickets):
        r = srv.wait(tk, int(nxs[int(who[i])]), timeout=600)
        lat.append(r["latency"])
        statuses[int(r["status"])] = statuses.get(int(r["status"]), 0) + 1
        relres = max(relres, r["relres"])
        iters = max(iters, r["iters"])
    s1 = srv.stats()
    srv.close()
    lat = np.array(lat)
    # the span from the first submission to the last completion (submission + the latency the server
    # measured), not to the end of this thread's polling of the results
    span = max(float(np.max(t_arr[:count] + lat)), 1e-9)
    req = max(s1["requests"] - s0["requests"], 1)
    return dict(offered_per_s=round(count / max(t_arr[-1], 1e-9), 1), submitted_per_s=round(count / (t_sub_end - tstart), 1),
                solves_per_s=round(count / span, 1), p50_ms=round(1e3 * float(np.median(lat)), 3),
                p99_ms=round(1e3 * float(np.quantile(lat, 0.99)), 3), mean_ms=round(1e3 * float(lat.mean()), 3),
                requests=count, failed=int(count - statuses.get(0, 0)), statuses=statuses, relres_max=relres,
                refine_iters_max=iters, submit_s=round(t_sub_end - tstart, 3),
                span_s=round(span, 3), rounds=s1["rounds"] - s0["rounds"],
                stages_reduced_per_request=round((s1["stages_reduced"] - s0["stages_reduced"]) / req, 1),
                stages_per_request=round((s1["stages_solved"] - s0["stages_solved"]) / req, 1))


SERVE_PLANS = [("tree_reuse", dict(leaf_len=0, branching=0, top_len=0), True),
               ("serial", dict(leaf_len=0, branching=0, top_len=1 << 20), True)]
# the tree without reuse (every chunk of every round reduced again), for the sweep
SERVE_FULL = ("tree_no_reuse", dict(leaf_len=0, branching=0, top_len=0), False)


def run_serve(args):
    """Receding-horizon serving at args.rate requests/s for args.duration s: the tree plan with
    factorisation reuse across shifts, and the plain serial recursion (top_len above every N,
    its one chunk re-reduced at every shift)."""
    import torch
    from paper_1510_03110_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    ws = serve_setup(args, [args.rate], args.duration)
    out = {}
    for name, plan, reuse in SERVE_PLANS:
        out[name] = serve_once(args, ws, args.rate, plan, reuse)
    return dict(estimators=ws["E"], rate=args.rate, duration_s=args.duration, generation_s=ws["gen_s"],
                nx="U{6,12,24}", N="U{50,200,1000}",
                precision="FP32 tree + FP64 refinement, relres<=%g" % args.serve_tol, **out)


def run_serve_sweep(args):
    """The offered rate raised until the server saturates, per plan: solves/s, p50/p99 at each
    rate; the highest rate whose throughput keeps up (>= 95% of the offered rate) with p99 below
    args.p99_bound_ms."""
    import torch
    from paper_1510_03110_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    rates = [float(v) for v in args.rates.split(",")]
    ws = serve_setup(args, rates, args.duration)
    plans = SERVE_PLANS + [SERVE_FULL]
    res = {name: [] for name, _, _ in plans}
    for rate in rates:
        for name, plan, reuse in plans:
            r = serve_once(args, ws, rate, plan, reuse)
            r["rate"] = rate
            res[name].append(r)
    sat = {}
    for name, rows in res.items():
        ok = [r for r in rows if r["solves_per_s"] >= 0.95 * r["offered_per_s"] and r["p99_ms"] <= args.p99_bound_ms]
        sat[name] = dict(max_sustained_rate=max((r["rate"] for r in ok), default=None),
                         max_solves_per_s=max(r["solves_per_s"] for r in rows))
    return dict(estimators=ws["E"], duration_s=args.duration, generation_s=ws["gen_s"], rates=rates,
                p99_bound_ms=args.p99_bound_ms, nx="U{6,12,24}", N="U{50,200,1000}",
                precision="FP32 tree + FP64 refinement, relres<=%g" % args.serve_tol, runs=res, saturation=sat)


def pinned_h2d_gbs(nbytes=1 << 31, reps=3):
    """Host-to-device bandwidth of one pinned 2 GiB copy on this machine (the floor of
    the end-to-end number: the host link is shared with the machine's other GPUs)."""
    import torch
    h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(reps):
        d.copy_(h, non_blocking=True)
    torch.cuda.synchronize()
    gbs = nbytes * reps / (time.perf_counter() - t) / 1e9
    del h, d
    return round(gbs, 1)


def run_e2e(args, buckets, solvers, step, stream, instances):
    """The same step through mhe_estimate_host: the FP64 problem in pinned host
    memory, the solution (x, w, lambda, info) back in pinned host memory, every
    copy inside the timed region (the library overlaps them with the solve)."""
    import torch
    from paper_1510_03110_gb300 import mhe
    host, outs = [], []
    h2d = d2h = 0
    for bk, s in zip(buckets, solvers):
        d = bk["dev"]
        hb = {}
        for k in ("A", "B", "C", "R", "a", "yt", "wt", "x0", "P0inv"):
            t = torch.empty(d[k].shape, dtype=d[k].dtype, pin_memory=True)
            t.copy_(d[k])
            hb[k] = t
            h2d += t.numel() * t.element_size()
        host.append(hb)
        x, w, lam = s.out
        hx = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in (x, w, lam)]
        info = torch.empty(s.info.numel(), dtype=torch.uint8, pin_memory=True)
        outs.append((hx, info))
        d2h += sum(t.numel() * t.element_size() for t in hx) + info.numel()
    k = max(1, min(args.steps, 5))

    import concurrent.futures as cf
    pool = cf.ThreadPoolExecutor(len(buckets))   # one caller thread per shape bucket (ctypes drops the GIL)

    for s in solvers:
        s.set_host_in_place(bool(args.e2e_in_place))

    calls = {}   # per bucket: host times (s) at which its call began and returned

    def one(i):
        bk, s, hb, (hx, info) = buckets[i], solvers[i], host[i], outs[i]
        t_in = time.perf_counter()
        mhe.mhe_estimate_host(s.ctx, bk["q"], hb["A"], hb["B"], hb["C"], hb["R"], hb["a"], hb["yt"], hb["wt"],
                              hb["x0"], hb["P0inv"], hx[0], hx[1], hx[2], info, pieces=args.e2e_pieces)
        calls[i] = (t_in, time.perf_counter())

    # one host thread: every bucket's pipeline issued (the largest first), then each waited on
    order = sorted(range(len(buckets)), key=lambda i: -int(np.sum(buckets[i]["N"])) * buckets[i]["n"] ** 2)

    def e2e_step_one_thread():
        t_in = time.perf_counter()
        for i in order:
            bk, s, hb, (hx, info) = buckets[i], solvers[i], host[i], outs[i]
            mhe.mhe_estimate_host_async(s.ctx, bk["q"], hb["A"], hb["B"], hb["C"], hb["R"], hb["a"], hb["yt"],
                                        hb["wt"], hb["x0"], hb["P0inv"], hx[0], hx[1], hx[2], info,
                                        pieces=args.e2e_pieces)
        for i in order:
            mhe.mhe_estimate_host_wait(solvers[i].ctx)
            calls[i] = (t_in, time.perf_counter())

    def e2e_step():
        if args.e2e_threads == "one":
            e2e_step_one_thread()
        else:
            list(pool.map(one, range(len(buckets))))

    for _ in range(2):   # warm-up: the pipeline's engines and device buffers, the pinned pages
        e2e_step()
    torch.cuda.synchronize()
    each = []
    t0 = time.perf_counter()
    for _ in range(k):
        t1 = time.perf_counter()
        e2e_step()
        each.append((time.perf_counter() - t1) * 1e3)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3 / k
    timeline = None
    if args.e2e_timeline:
        # more steps with the pipelines' timelines recorded (outside the timed steps): per step the
        # host window of each bucket's call and the device time its last output arrived; the
        # pieces of the slowest step
        for s in solvers:
            mhe.mhe_timing_enable(s.ctx, True)
        steps_tl, worst = [], None
        for _ in range(k):
            t1 = time.perf_counter()
            c1 = time.process_time()
            e2e_step()
            wall_tl = (time.perf_counter() - t1) * 1e3
            cpu_tl = (time.process_time() - c1) * 1e3
            host_calls = {buckets[i]["n"]: [round((a - t1) * 1e3, 2), round((b - t1) * 1e3, 2)]
                          for i, (a, b) in calls.items()}
            pieces = {bk["n"]: mhe.mhe_pipe_timeline(s.ctx) for bk, s in zip(buckets, solvers)}
            steps_tl.append(dict(step_ms=round(wall_tl, 2), host_cpu_ms=round(cpu_tl, 2), host_calls_ms=host_calls,
                                 device_last_out_ms={n: round(max(r[7] for r in p), 2) for n, p in pieces.items() if p}))
            if worst is None or wall_tl > worst[0]:
                worst = (wall_tl, pieces)
        timeline = dict(steps=steps_tl, columns=["engine", "b0", "b1", "host_issue_ms", "h2d_issued_ms",
                                                 "inputs_arrived_ms", "solved_ms", "outputs_back_ms"],
                        slowest=dict(step_ms=round(worst[0], 2),
                                     buckets=[dict(nx=n, pieces=[[round(v, 3) for v in row] for row in p])
                                              for n, p in worst[1].items()]))
        for s in solvers:
            mhe.mhe_timing_enable(s.ctx, False)
            mhe.mhe_timing_read(s.ctx)
    pool.shutdown()
    gbs = pinned_h2d_gbs()
    infos = np.concatenate([info.numpy().view(mhe.INFO_DTYPE) for _, info in outs])
    del mhe
    return dict(value=round(instances / (ms * 1e-3), 3), unit="KKT solves/s", h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(d2h), ms_per_step=round(ms, 3),
                ms_median=round(float(np.median(each)), 3), steps=k, pieces=args.e2e_pieces,
                ms_each=[round(v, 2) for v in each], h2d_gbs_pinned=gbs,
                h2d_floor_ms=round(h2d / (gbs * 1e6), 1),
                relres_max=float(np.max(infos["relres"])), all_ok=bool(np.all(infos["status"] == 0)),
                api=("mhe_estimate_host (pinned host buffers), one caller thread per shape bucket"
                     if args.e2e_threads == "bucket" else
                     "mhe_estimate_host_async for every shape bucket, then mhe_estimate_host_wait (pinned host "
                     "buffers), one caller thread") +
                    (", inputs read in place (mhe_set_host_in_place)" if args.e2e_in_place else ""),
                timer="host wall clock around the synchronous calls", timeline=timeline)


# ---------------------------------------------------------------- CPU oracle

def _sample(buckets, count):
    """A bounded, seeded sample of instances across the buckets (MHE-form dicts)."""
    rng = np.random.default_rng(11)
    out = []
    per = max(1, count // len(buckets))
    for bk in buckets:
        offs = np.concatenate([[0], np.cumsum(bk["N"] - 1)])
        for j in rng.choice(len(bk["N"]), size=min(per, len(bk["N"])), replace=False):
            idx = bk["idx"][offs[j]:offs[j + 1]]
            out.append(synth.instance_from_pool(bk["pool"], idx, bk["x0"][j], bk["n"], bk["m"], bk["q"]))
    return out


def _oracle_solve(p):
    import oracle
    r = oracle.riccati(oracle.mhe_to_uftoc(p))
    return r["status"]


def cpu_baseline(buckets, args, seconds=15.0):
    """The FP64 oracle (serial Riccati, plain C) on host cores, on a bounded sample."""
    import concurrent.futures as cf
    cores = os.cpu_count() or 1
    sample = _sample(buckets, max(cores, 6) if len(buckets) > 1 else 1)
    cores = min(cores, len(sample))
    t0 = time.time()
    done = 0
    with cf.ThreadPoolExecutor(cores) as ex:
        while time.time() - t0 < seconds and done < 4 * len(sample):
            list(ex.map(_oracle_solve, sample))
            done += len(sample)
            if len(buckets) == 1:
                break
    dt = time.time() - t0
    stages = sum(p["N"] for p in sample) * (done // len(sample))
    return dict(value=round(done / dt, 4), unit="KKT solves/s", cores=cores, kind="oracle",
                sample=f"{len(sample)} instances of the workload ({stages} stages solved), {done} solves "
                       f"in {dt:.1f} s on a thread pool (ctypes releases the GIL)")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    desc, buckets, prec = make_workload(args.workload)
    import concurrent.futures as cf
    cores = os.cpu_count() or 1
    sample = _sample(buckets, max(cores, 6) if len(buckets) > 1 else 1)
    cores = min(cores, len(sample))
    with cf.ThreadPoolExecutor(cores) as ex:
        for _ in range(args.warmup if len(buckets) > 1 else 0):
            list(ex.map(_oracle_solve, sample))
        times = []
        for _ in range(args.steps):
            t0 = time.time()
            list(ex.map(_oracle_solve, sample))
            times.append(time.time() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = len(sample) / (ms * 1e-3)
    cpu = dict(kind="oracle", cores=cores, value=round(value, 4),
               sample=f"{len(sample)} instances of the workload per step, serial FP64 Riccati in plain C")
    print(json.dumps(dict(metric=METRIC, impl="reference", value=round(value, 4), unit="KKT solves/s",
                          n_gpus=int(os.environ.get("WORLD_SIZE", "1")), steps=args.steps, warmup=args.warmup,
                          ms_per_step=round(ms, 3), higher_is_better=True, scaling="weak", vs_baseline=None,
                          dtype="f64", data="synthetic", config=desc, cpu_baseline=cpu,
                          e2e=dict(value=round(value, 4), unit="KKT solves/s", h2d_bytes_per_step=0,
                                   d2h_bytes_per_step=0))))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="batch",
                    choices=["batch", "long", "profile", "serve", "xl", "xl_profile", "alu_peaks", "small", "ip", "link"])
    ap.add_argument("--N", type=int, default=131072, help="long workload: the horizon")
    ap.add_argument("--sweep", action="store_true", help="long workload: the depth sweep over N, leaf, branching")
    ap.add_argument("--sweep-N", default="1024,16384,131072")
    ap.add_argument("--sweep-leaf", default="8,16,32,64")
    ap.add_argument("--sweep-branching", default="2,4,8,16")
    ap.add_argument("--sweep-reps", type=int, default=3)
    ap.add_argument("--err-samples", type=int, default=2, help="instances per bucket checked against the oracle")
    ap.add_argument("--refine-tol", type=float, default=1e-12,
                    help="relative KKT residual the refinement reaches (1e-12: the forward error of the "
                         "worst-conditioned instances then meets 1e-8 against the oracle; relres 1e-9, the "
                         "metric's bar alone, leaves up to ~5e-7)")
    ap.add_argument("--fp64-masters", action="store_true", help="master levels k >= 1 in FP64 (mixed precisions)")
    ap.add_argument("--fp64-residual", action="store_true",
                    help="mixed precisions: the MHE-form residual with FP64 instructions (default: double-float)")
    ap.add_argument("--plan", default=None, help="leaf_len,branching,top_len used instead of the autotuner")
    ap.add_argument("--rate", type=float, default=20000.0, help="serving: Poisson arrival rate (requests/s)")
    ap.add_argument("--duration", type=float, default=5.0, help="serving: seconds of arrivals")
    ap.add_argument("--estimators", type=int, default=1024, help="serving: estimator pool")
    ap.add_argument("--rates", default="", help="serving: comma-separated offered rates for a saturation sweep")
    ap.add_argument("--p99-bound-ms", type=float, default=50.0, help="serving sweep: p99 a sustained rate keeps")
    ap.add_argument("--serve-tol", type=float, default=1e-9, help="serving: relres the refinement reaches")
    ap.add_argument("--serve-refine", type=int, default=16, help="serving: corrections allowed per request")
    ap.add_argument("--serve-bytes", type=int, default=96 << 30, help="serving: device-memory budget")
    ap.add_argument("--serve-duration", type=float, default=10.0,
                    help="batch workload: seconds of a serving run appended to the line (0: none)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the serial-plan GPU baseline")
    ap.add_argument("--baseline-steps", type=int, default=2)
    ap.add_argument("--serial-fp64", action="store_true", help="also time the serial plan in FP64")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--e2e-pieces", type=int, default=8, help="pieces of the host-buffer pipeline per bucket")
    ap.add_argument("--e2e-threads", choices=["one", "bucket"], default="one",
                    help="end to end: one host thread issuing every bucket's pipeline, or a thread per bucket")
    ap.add_argument("--e2e-in-place", action="store_true", help="end to end: the kernels read the pinned inputs in place")
    ap.add_argument("--e2e-timeline", action="store_true", help="end to end: record one step's pipeline timeline")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--tune-instances", type=int, default=256)
    ap.add_argument("--serial-nx", type=lambda v: [int(x) for x in v.split(",") if x], default=[],
                    help="shape buckets (nx list) that take the serial plan instead of the autotuner's")
    ap.add_argument("--prec", default="auto", choices=["auto", "fp32", "tf32", "bf16"],
                    help="tree precision of the FP32 workloads: tf32 / bf16 = stage products on the tensor "
                         "cores (MHE_TF32_IR / MHE_BF16_IR; auto: tf32 for the nx = 64 workloads, fp32 otherwise)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if int(os.environ.get("RANK", "0")) != 0:
        # one GPU does the work: rank 0 runs the workload, the other ranks exit without work
        return
    if args.workload == "alu_peaks":
        raise SystemExit(run_alu_peaks())
    global LONG_N
    LONG_N = args.N
    if args.workload == "long" and args.sweep:
        res = run_long_sweep(args)
        big = res["summary"][-1]
        print(json.dumps(dict(metric=METRIC, value=round(1e3 / big["best_tree_ms"], 3), unit="KKT solves/s",
                              n_gpus=1, steps=args.sweep_reps, warmup=1, ms_per_step=big["best_tree_ms"],
                              higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                              data="synthetic", config=dict(workload=res["workload"], N=big["N"]),
                              sweep=res)))
        return
    if args.workload == "small":
        res = run_small(args)
        t = res["tree"]
        print(json.dumps(dict(metric=METRIC, value=round(1e3 / t["mean_ms"], 3), unit="KKT solves/s", n_gpus=1,
                              steps=max(args.steps, 50), warmup=max(args.warmup, 3), ms_per_step=t["mean_ms"],
                              higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                              data="synthetic",
                              config=dict(workload="single MHE instance nx=4, nw=ny=2, N=64, FP64, seed 0",
                                          l2="inputs smaller than L2 (latency case; not flushed)"),
                              latency_ms=dict(p50=t["p50_ms"], p99=t["p99_ms"]), arms=res)))
        return
    if args.workload == "link":
        res = run_link(args)
        print(json.dumps(dict(metric="pinned host-to-device copy rate", value=res["series"]["median"], unit="GB/s",
                              n_gpus=1, higher_is_better=True, data="synthetic", dtype="u8",
                              config=dict(workload="host link: 1 GiB pinned copies"), link=res)))
        return
    if args.workload == "ip":
        res = run_ip(args)
        print(json.dumps(dict(metric=METRIC, value=res["ip_solves_per_s"], unit="box-bounded MHE solves/s", n_gpus=1,
                              steps=3, warmup=1, ms_per_step=res["ms_per_ip_solve"], higher_is_better=True,
                              scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                              config=dict(workload=res["workload"]), ip=res)))
        return
    if args.workload == "serve" and args.rates:
        res = run_serve_sweep(args)
        print(json.dumps(dict(metric=METRIC, value=res["saturation"]["tree_reuse"]["max_solves_per_s"],
                              unit="KKT solves/s", n_gpus=1, steps=len(res["rates"]), warmup=1,
                              ms_per_step=None, higher_is_better=True, scaling="weak", vs_baseline=None,
                              dtype="f32+f64", data="synthetic",
                              config=dict(workload="receding-horizon serving, Poisson arrivals, rate sweep",
                                          estimators=res["estimators"], duration_s=res["duration_s"]),
                              serve_sweep=res)))
        return
    if args.workload == "serve":
        res = run_serve(args)
        tree, ser = res["tree_reuse"], res["serial"]
        print(json.dumps(dict(metric=METRIC, value=tree["solves_per_s"], unit="KKT solves/s", n_gpus=1,
                              steps=tree["requests"], warmup=1, ms_per_step=tree["mean_ms"], higher_is_better=True,
                              scaling="weak", vs_baseline=None, dtype="f32+f64", data="synthetic",
                              config=dict(workload="receding-horizon serving, Poisson arrivals", **{
                                  k: v for k, v in res.items() if k not in ("tree", "serial")}),
                              latency_ms=dict(p50=tree["p50_ms"], p99=tree["p99_ms"]),
                              serving=res, speedup_vs_serial=dict(
                                  solves_per_s=round(tree["solves_per_s"] / max(ser["solves_per_s"], 1e-9), 3),
                                  p99=round(ser["p99_ms"] / max(tree["p99_ms"], 1e-9), 3)))))
        return
    run_gpu(args)


if __name__ == "__main__":
    main()
