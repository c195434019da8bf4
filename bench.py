"""Throughput benchmark of the data-annealed SMC sampler on GB300.

A step is one SMC iteration through the C ABI: smc_anneal_next, smc_resample
and smc_step (S leapfrog steps, each a forward + adjoint pass of all J
particle networks over the annealed subset D_k, then the reweight,
normalisation and ESS).  Workload: the MNIST-shaped stand-in (60000 synthetic
28x28 10-class images), MLP 784-100-10 ReLU, J = 256 particles, mini-batch
1000, Linear data annealing taken at its full-subset phase (|D_k| = 60000),
HMC with S = 3, h = 0.002, BF16 tcgen05 contractions with FP32 accumulation.

Metric: particle-sample gradient evaluations per second = J * |D_k| * (gradient
evaluations) / time.  `value` is device-timed with inputs resident in HBM;
`e2e` streams the annealed subset from pinned host memory every step
(smc_upload_rows_async: step k+1's rows copy on the library's copy stream
while step k computes) and reads the step statistics back.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload instead (the reference arm: there is no reference implementation of
the paper to run).
"""
from __future__ import annotations

import argparse
import json
import datetime
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle*sample grad-evals/s"
UNIT = "grad-evals/s"
N_TRAIN, DIN, H, NCLS = 60000, 784, 100, 10
J_DEFAULT, MB, K_SCHED, K_START, STEP_H, S_LF = 256, 1000, 200, 100, 0.002, 3


def workload_config(args):
    return {
        "workload": (f"MLP {DIN}-{H}-{NCLS} ReLU, J={args.J} particles, synthetic {args.n}x{DIN} 10-class images, "
                     f"Linear DA (C=kappa={MB}, K={K_SCHED}) at its full-subset phase |D_k|={args.n}, "
                     f"HMC S={S_LF}, h={STEP_H}"),
        "particles": args.J, "rows": args.n,
        "schedule": "linear", "leapfrog_steps": S_LF,
        "l2": "no flush: per-step working set (activations 2x3 GB) far above the 129 MB L2",
    }


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), d.get("bf16_tflops_sustained", 1700.0), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


# DRAM bytes (read + write) of one launch at the default workload (J = 256,
# 60000 rows), from a one-pass ncu capture of that launch
# (dram__bytes_read.sum + dram__bytes_write.sum).  Reported only while the
# kernel's sources hash to the value recorded with the capture, so a changed
# kernel reports null until it is captured again.
KERNEL_SOURCES = {
    "fused_fwd_head": ["k_fused.cu", "tc_ptx.cuh", "mma_ptx.cuh", "tmap.cuh"],
    "wgrad_gemm": ["k_tc.cu", "tc_ptx.cuh", "tmap.cuh"],
}
TRAFFIC = {
    "fused_fwd_head": {"J": 256, "n": 60000, "bytes": 1.2929e9 + 3.0351e9,
                       "sha256": "ea5589df86fe9eb99ce03940560241ee6481d52725c6ec897459a55eb80d9bc6"},
    "wgrad_gemm": {"J": 256, "n": 60000, "bytes": 3.8466e9 + 0.2161e9,
                   "sha256": "db78c31838ff81c850427fa41081cb8ed376cd27b43217dce04adbd63ae518f3"},
}


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2601_21983_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def measured_traffic(kernel, J, n):
    t = TRAFFIC.get(kernel)
    if t is None or (J, n) != (t["J"], t["n"]) or source_hash(kernel) != t["sha256"]:
        return None
    return t["bytes"]


class Clocks:
    """nvidia-smi samples (every 100 ms, host-timestamped) kept for the timed
    region only: start() before the warm-up, mark(t0, t1) with the host times
    around the timed loop, stop() after it."""

    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, idx):
        self.proc = None
        self.window = None
        out_dir = os.environ.get("SMC_CLOCKS_DIR", tempfile.gettempdir())
        self.path = os.path.join(out_dir, f"smc_clocks_{os.getpid()}.csv")
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(idx), "--query-gpu=timestamp,clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)          # let the sampler write the sample that closes the window
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        t0, t1 = self.window if self.window else (rows[0][0], rows[-1][0])
        inside = [r for r in rows if t0 <= r[0] <= t1]
        note = "samples inside the timed region"
        if not inside:       # a region shorter than the sampling period: the sample closest to it
            inside = [min(rows, key=lambda r: abs(r[0] - 0.5 * (t0 + t1)))]
            note = "timed region shorter than the 100 ms sampling period: nearest sample"
        reasons = sorted({nm for r in inside for nm, v in zip(self.NAMES, r[4]) if v.lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[1] for r in inside])), "sm_max_mhz": float(max(r[2] for r in inside)),
                "reasons": reasons, "samples": len(inside), "power_w": float(np.median([r[3] for r in inside])),
                "note": note}


def make_data(n, seed=0):
    import synthetic
    return synthetic.template_images(n, seed=seed)


def host_threads():
    """Threads the oracle's numpy BLAS may use: an explicit thread-count
    variable when set, else the cores this process may run on."""
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        try:
            n = int(os.environ.get(var, ""))
        except ValueError:
            continue
        if n > 0:
            return n
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def _oracle_eval_rate(seconds, J_s, M_s, seed, scale=False):
    """Particle-sample gradient evaluations per second of the FP64 oracle on
    J_s particles x M_s rows of the workload's model and data (this process);
    scale: the 784-400-400-10 network instead of 784-100-10."""
    import synthetic
    from oracle import nn
    if scale == "cnn":
        spec = nn.Spec(CNN_LAYERS, (3, 32, 32), nn.TANH)
        X, y = synthetic.smooth_field_images(M_s, seed=3)
    else:
        layers = [("dense", DIN, 400), ("dense", 400, 400), ("dense", 400, NCLS)] if scale else \
            [("dense", DIN, H), ("dense", H, NCLS)]
        spec = nn.Spec(layers, (DIN,), nn.RELU)
        X, y = synthetic.template_images(M_s, seed=3)
    X = X.astype(np.float64)
    th = synthetic.particles(J_s, spec.n_params, seed, std=0.05).astype(np.float64)
    coef = np.full(M_s, N_TRAIN / M_s)
    n_eval = 0
    t0 = time.perf_counter()
    while True:
        for j in range(J_s):
            nn.loglik_grad(spec, th[j], X, y, coef)
        n_eval += J_s
        el = time.perf_counter() - t0
        if el >= seconds:
            break
    return n_eval, el


def _oracle_workers(n, seconds, J_s, M_s):
    """n concurrent single-threaded oracle processes (particles split across
    them, as the oracle's particles are independent); returns their total
    evaluations and the longest elapsed time."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", str(seconds), str(J_s), str(M_s)]
    procs = [subprocess.Popen(cmd + [str(10 + w)], env=env, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                              text=True) for w in range(n)]
    total, longest = 0, 0.0
    for p in procs:
        out, _ = p.communicate(timeout=300)
        ev, el = json.loads(out.strip().splitlines()[-1])
        total += ev
        longest = max(longest, el)
    return total, longest


def cpu_baseline(seconds=8.0, J_s=2, M_s=2000):
    """The FP64 oracle's gradient evaluation on a bounded sample of the
    workload (J_s particles x M_s rows of the same model and data per
    process), single-threaded and on every host core (one single-threaded
    process per core, particles split across them)."""
    cores = host_threads()
    ev1, el1 = _oracle_workers(1, seconds, J_s, M_s)
    evn, eln = _oracle_workers(cores, seconds, J_s, M_s)
    single = ev1 * M_s / el1
    allc = evn * M_s / eln
    return {"value": allc, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle gradient evaluations of single particles over {M_s} rows of the workload, "
                      f"{seconds:.0f} s per run: {cores} single-threaded processes ({evn} evaluations) and "
                      f"one single-threaded process ({ev1} evaluations)",
            "single_thread": {"value": single, "unit": UNIT, "cores": 1},
            "all_cores": {"value": allc, "unit": UNIT, "cores": cores}}


# ---------------------------------------------------------------- scale configuration
SCALE_H, SCALE_J, SCALE_LAYERS = 400, 1024, [("dense", DIN, 400), ("dense", 400, 400), ("dense", 400, NCLS)]
SCALE_FLOP = 2.238e6       # per particle-sample gradient evaluation (955,200 forward + 1,283,200 backward)


def scale_workload(J, n):
    return {"workload": (f"MLP {DIN}-400-400-{NCLS} ReLU (D = 478,410), J={J} particles, synthetic {n}x{DIN} "
                         f"10-class images, full batch |D_k|={n} (FB), HMC S={S_LF}, h={STEP_H}, BF16 tcgen05 "
                         f"contractions with FP32 accumulation"),
            "particles": J, "rows": n, "schedule": "fb", "leapfrog_steps": S_LF,
            "l2": "no flush: per-step working set (activations 3 x 6.7 GB per chunk) far above the 129 MB L2"}


def scale_cpu_baseline(seconds=6.0, M_s=500):
    """The FP64 oracle on a bounded sample of the scale configuration: single
    particles of the 784-400-400-10 network over M_s rows, one
    single-threaded process and one per host core."""
    cores = host_threads()
    cmd_extra = ["--scale"]
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")

    def workers(n):
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", str(seconds), "1", str(M_s)]
        procs = [subprocess.Popen(cmd + [str(20 + w)] + cmd_extra, env=env, stdout=subprocess.PIPE,
                                  stderr=subprocess.DEVNULL, text=True) for w in range(n)]
        total, longest = 0, 0.0
        for p in procs:
            out, _ = p.communicate(timeout=300)
            ev, el = json.loads(out.strip().splitlines()[-1])
            total, longest = total + ev, max(longest, el)
        return total, longest

    ev1, el1 = workers(1)
    evn, eln = workers(cores)
    return {"value": evn * M_s / eln, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle gradient evaluations of single particles of the 784-400-400-10 network over "
                      f"{M_s} rows, {seconds:.0f} s per run: {cores} single-threaded processes ({evn} evaluations) "
                      f"and one ({ev1} evaluations)",
            "single_thread": {"value": ev1 * M_s / el1, "unit": UNIT, "cores": 1},
            "all_cores": {"value": evn * M_s / eln, "unit": UNIT, "cores": cores}}


CNN_LAYERS = [("conv", 3, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 800, NCLS)]
CNN_J, CNN_N = 128, 50000
CNN_FLOP = 11.49e6         # per particle-sample gradient evaluation (4,457,600 forward + 7,033,600 backward)


def cnn_workload(J, n):
    return {"workload": (f"CNN conv5x5 3->16, tanh, pool, conv5x5 16->32, tanh, pool, fc 800->{NCLS} (D = 22,058), "
                         f"J={J} particles, synthetic {n} 3x32x32 10-class smooth-field images, full data |D_k|={n} "
                         f"(the end of SDA's annealing), HMC S={S_LF}, h={STEP_H}, BF16 tcgen05 convolutions with "
                         f"FP32 accumulation"),
            "particles": J, "rows": n, "schedule": "fb", "leapfrog_steps": S_LF,
            "l2": "no flush: per-step working set (pooled maps, conv-2 outputs, dZ2 and dZ1 of ~15 GB per chunk of 2048 images) far above the L2"}


def _section(kind, steps, warmup, J, n, e2e=True, roofline=True, cpu=True):
    """One SMC iteration (anneal, resample, HMC move with S = 3 gradient
    evaluations over all n rows, reweight) of another configuration through
    the C ABI, device-timed with CUDA events on the library's stream; then the
    same end to end with the rows streamed from pinned host memory each step;
    then per-kernel-family times for the roofline.  kind: "scale" (MLP
    784-400-400-10, the engine for two or more hidden layers) or "cnn" (the
    CIFAR-shaped CNN)."""
    import torch
    import synthetic
    from paper_2601_21983_gb300 import smc as S
    S.load()
    stream = torch.cuda.current_stream()
    if kind == "scale":
        X, y = make_data(n, seed=0)
        model = S.make_model(SCALE_LAYERS, (DIN,), S.ACT_RELU)
        flop_unit, workload = SCALE_FLOP, scale_workload(J, n)
    else:
        X, y = synthetic.smooth_field_images(n, seed=0)
        model = S.make_model(CNN_LAYERS, (3, 32, 32), S.ACT_TANH)
        flop_unit, workload = CNN_FLOP, cnn_workload(J, n)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    sched = S.make_schedule("fb", n, n, K_SCHED)

    def new_ctx(timing=0):
        ctx = S.smc_init(model, Xd, y_class=yd, cfg=S.make_config(J, 4321, S.PREC_BF16, stream=stream, timing=timing))
        D = S.smc_num_params(ctx)
        std = 0.05 if kind == "scale" else 0.1
        S.smc_set_state_device(ctx, std * torch.randn(J, D, device="cuda",
                                                        generator=torch.Generator(device="cuda").manual_seed(5)))
        S.smc_set_schedule(ctx, sched)
        return ctx

    evals = [0]

    def one_step(ctx):
        S.smc_anneal_next(ctx)
        S.smc_resample(ctx)
        st = S.smc_step(ctx, STEP_H, S_LF)
        evals[0] += st["grad_evals"] * st["rows"] * J
        return st

    ctx = new_ctx()
    for _ in range(warmup):
        one_step(ctx)
    torch.cuda.synchronize()
    n0, _, _ = S.smc_get_counters(ctx)
    evals[0] = 0
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        st = one_step(ctx)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    n1, _, _ = S.smc_get_counters(ctx)
    out = {"metric": METRIC, "value": evals[0] / (ms / 1e3), "unit": UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps, "dtype": "bf16", "data": "synthetic", "config": workload,
           "gpu_launches": n1 - n0, "last_ess": st["ess"]}
    if e2e:
        perm = S.smc_get_permutation(ctx, n)
        hx = torch.from_numpy(np.ascontiguousarray(X[perm])).pin_memory()
        hy = torch.from_numpy(np.ascontiguousarray(y[perm])).pin_memory()
        hxn, hyn = hx.numpy(), hy.numpy()
        torch.cuda.synchronize()
        evals[0] = 0
        t0 = time.perf_counter()
        S.smc_upload_rows_async(ctx, 0, hxn, hyn)
        for i in range(steps):
            S.smc_anneal_next(ctx)
            S.smc_resample(ctx)
            if i + 1 < steps:
                S.smc_upload_rows_async(ctx, 0, hxn, hyn)
            st = S.smc_step(ctx, STEP_H, S_LF)
            evals[0] += st["grad_evals"] * st["rows"] * J
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        out["e2e"] = {"value": evals[0] / el, "unit": UNIT, "h2d_bytes_per_step": int(hxn.nbytes + hyn.nbytes),
                      "d2h_bytes_per_step": 16 * 8 + 2 * 4}
    S.smc_destroy(ctx)
    if roofline:
        ctx = new_ctx(timing=1)
        one_step(ctx)
        S.smc_reset_counters(ctx)
        n_evals = one_step(ctx)["grad_evals"]
        _, times, calls = S.smc_get_counters(ctx)
        S.smc_destroy(ctx)
        hbm, tf_burst, tf_sus, src = peaks()
        units = float(n) * J                           # particle-sample pairs per evaluation
        if kind == "scale":
            H = SCALE_H
            work = {"fwd_gemm": ("tensor", 2.0 * units * H * DIN),
                    "hidden_gemm": ("tensor", 2.0 * units * H * H),
                    "adjoint_gemm": ("tensor", 2.0 * units * H * H),
                    "hidden_wgrad_gemm": ("tensor", 2.0 * units * H * (H + 1)),
                    "wgrad_gemm": ("tensor", 2.0 * units * H * (DIN + 1)),
                    # the head reads the last hidden activations and writes dZ over them (BF16)
                    "head": ("hbm", 2.0 * units * H * 2.0)}
        else:
            # conv 1 (784 positions x 16 x 75, pool 1 in its epilogue), conv 2 (100 x 32
            # x 400), their weight gradients (with the bias column) and the conv-2 data
            # gradient: the valid convolutions' multiply-adds
            work = {"fwd_gemm": ("tensor", 2.0 * units * 784 * 16 * 75),
                    "hidden_gemm": ("tensor", 2.0 * units * 100 * 32 * 400),
                    "hidden_wgrad_gemm": ("tensor", 2.0 * units * 100 * 32 * 401),
                    "adjoint_gemm": ("tensor", 2.0 * units * 100 * 32 * 400),
                    "wgrad_gemm": ("tensor", 2.0 * units * 784 * 16 * 76),
                    # im2col of the images (written once per image, shared by the particles)
                    # and pool 2 forward / backward: Z2 read, P2 + idx2 written, dP2 + idx2
                    # read, Z2 at each argmax read, dZ2 written (BF16, per particle-image)
                    "simt_net": ("hbm", float(n) * (784 * 80 * 2.0 + 3 * 32 * 32 * 2.0) +
                                 units * (6400.0 + 2400.0 + 2400.0 + 1600.0 + 6400.0)),
                    # the head reads P2 and writes dP2 over it
                    "head": ("hbm", units * 800 * 2 * 2.0)}
        kern = {}
        gemm_flop, gemm_ms = 0.0, 0.0
        for k, (bound, amount) in work.items():
            if not calls.get(k):
                continue
            per_eval = times[k] / n_evals                  # ms per gradient evaluation over all rows
            if bound == "tensor":
                ach = amount / (per_eval / 1e3) / 1e12
                kern[k] = {"bound": "tensor", "achieved": ach, "peak": tf_burst, "unit": "TFLOP/s",
                           "frac": ach / tf_burst, "ms_per_eval": per_eval, "work_per_eval": amount,
                           "launches_per_eval": calls[k] / n_evals}
                gemm_flop += amount
                gemm_ms += per_eval
            else:
                ach = amount / (per_eval / 1e3) / 1e9
                kern[k] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                           "ms_per_eval": per_eval, "work_per_eval": amount,
                           "launches_per_eval": calls[k] / n_evals}
        dom = max(kern, key=lambda k: kern[k]["ms_per_eval"])
        roof = dict(kern[dom])
        roof["kernel"] = dom
        roof["traffic"] = None
        roof["peak_kind"] = f"{src} " + ("bf16_tflops (burst)" if roof["bound"] == "tensor" else "hbm_gbs")
        roof["all_gemms"] = {"achieved": gemm_flop / (gemm_ms / 1e3) / 1e12, "unit": "TFLOP/s",
                             "frac": gemm_flop / (gemm_ms / 1e3) / 1e12 / tf_burst, "ms_per_eval": gemm_ms}
        roof["whole_step"] = {"achieved": units * flop_unit * S_LF / (out["ms_per_step"] / 1e3) / 1e12,
                              "unit": "TFLOP/s",
                              "frac": units * flop_unit * S_LF / (out["ms_per_step"] / 1e3) / 1e12 / tf_burst}
        roof["others"] = {k: {"frac": round(v["frac"], 4), "achieved": round(v["achieved"], 1), "unit": v["unit"],
                              "ms_per_eval": round(v["ms_per_eval"], 3)} for k, v in kern.items() if k != dom}
        out["roofline"] = roof
        out["families_ms"] = {k: {"ms": times[k], "calls": calls[k]} for k in times if calls[k]}
    if cpu:
        out["cpu_baseline"] = scale_cpu_baseline() if kind == "scale" else cnn_cpu_baseline()
    return out


def run_scale_config(steps, warmup, J=SCALE_J, n=N_TRAIN, e2e=True, roofline=True, cpu=True):
    return _section("scale", steps, warmup, J, n, e2e, roofline, cpu)


def run_cnn_config(steps, warmup, J=CNN_J, n=CNN_N, e2e=True, roofline=True, cpu=True):
    return _section("cnn", steps, warmup, J, n, e2e, roofline, cpu)


def cnn_cpu_baseline(seconds=6.0, M_s=20):
    """The FP64 oracle on a bounded sample of the CNN configuration: single
    particles over M_s images, one single-threaded process and one per core."""
    cores = host_threads()
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")

    def workers(nw):
        cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", str(seconds), "1", str(M_s)]
        procs = [subprocess.Popen(cmd + [str(30 + w), "--cnn"], env=env, stdout=subprocess.PIPE,
                                  stderr=subprocess.DEVNULL, text=True) for w in range(nw)]
        total, longest = 0, 0.0
        for p in procs:
            o, _ = p.communicate(timeout=300)
            ev, el = json.loads(o.strip().splitlines()[-1])
            total, longest = total + ev, max(longest, el)
        return total, longest

    ev1, el1 = workers(1)
    evn, eln = workers(cores)
    return {"value": evn * M_s / eln, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle gradient evaluations of single particles of the CNN over {M_s} images, "
                      f"{seconds:.0f} s per run: {cores} single-threaded processes ({evn} evaluations) and one "
                      f"({ev1} evaluations)",
            "single_thread": {"value": ev1 * M_s / el1, "unit": UNIT, "cores": 1},
            "all_cores": {"value": evn * M_s / eln, "unit": UNIT, "cores": cores}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synthetic
    from oracle import nn, rng, smc as osmc
    J_s, M_s = 2, 2000
    spec = nn.Spec([("dense", DIN, H), ("dense", H, NCLS)], (DIN,), nn.RELU)
    X, y = synthetic.template_images(M_s, seed=3)
    orc = osmc.Sampler(spec, X, y, J_s, rng.fisher_yates_permutation(M_s, 1))
    orc.set_schedule("fb", M_s, M_s, K_SCHED, synthetic.particles(J_s, spec.n_params, 1, std=0.05))
    z = synthetic.normals((J_s, spec.n_params), 2)
    for _ in range(args.warmup):
        orc.step(STEP_H, S_LF, z)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        orc.step(STEP_H, S_LF, z)
    el = time.perf_counter() - t0
    value = J_s * M_s * S_LF * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": host_threads(), "kind": "oracle",
                             "sample": f"each step: one FP64 oracle SMC move (S={S_LF}) of {J_s} particles over "
                                       f"{M_s} rows (bounded sample of the workload)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


EVAL_CONFIGS = {
    # name: (layers, input shape, activation, J, rows, chunk rows, FLOP per particle-sample evaluation, data)
    "cnn": ([("conv", 3, 16, 5), ("pool2",), ("conv", 16, 32, 5), ("pool2",), ("dense", 800, 10)], (3, 32, 32),
            "tanh", 128, 4096, 1024, 11.49e6, "smooth_field_images"),
    "mlp4": ([("dense", 784, 400), ("dense", 400, 400), ("dense", 400, 10)], (784,), "relu", 1024, 2048, 512,
             2.238e6, "template_images"),
    # Sec. 4's FashionMNIST network with its batchnorm layers (D = 96,658): contractions
    # 566,368 FLOP forward + 1,035,392 backward (the first layer has no data gradient)
    "fashion_bn": ([("conv", 1, 8, 3), ("bnorm", 8), ("pool2",), ("conv", 8, 16, 3), ("bnorm", 16), ("pool2",),
                    ("dense", 400, 232), ("dense", 232, 10)], (1, 28, 28), "tanh", 128, 4096, 1024, 1.60176e6,
                   "template_images"),
}


def run_eval_config(args):
    """Gradient-evaluation throughput of the FP32 engine's other configurations:
    the 3x32x32 CNN (conv5x5 3-16, pool, conv5x5 16-32, pool, fc 10; J = 128),
    the MLP 784-400-400-10 (J = 1024) and Sec. 4's FashionMNIST network with
    batchnorm (J = 128).  Each evaluation is log pi and its
    full gradient for every particle over the rows (smc_eval_device), timed
    with CUDA events after one warm-up evaluation."""
    import torch
    import synthetic
    from paper_2601_21983_gb300 import smc as S
    S.load()
    layers, shape, act, J, rows, chunk, flop, data = EVAL_CONFIGS[args.eval_config]
    X, y = getattr(synthetic, data)(rows, seed=0)
    model = S.make_model(layers, shape, S.ACT_TANH if act == "tanh" else S.ACT_RELU)
    stream = torch.cuda.current_stream()
    cfg = S.make_config(J, 5, S.PREC_FP32, stream=stream, chunk_rows=chunk)
    ctx = S.smc_init(model, torch.from_numpy(np.ascontiguousarray(X, np.float32)).cuda(),
                     y_class=torch.from_numpy(y.astype(np.int32)).cuda(), cfg=cfg)
    S.smc_set_schedule(ctx, S.make_schedule("fb", rows, rows, 5))
    D = S.smc_num_params(ctx)
    theta = torch.from_numpy(synthetic.particles(J, D, 5, std=0.05)).cuda()
    lp = torch.empty(J, dtype=torch.float64, device="cuda")
    g = torch.empty((J, D), dtype=torch.float32, device="cuda")
    S.smc_set_state_device(ctx, theta)
    S.smc_eval_device(ctx, lp, g)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        S.smc_eval_device(ctx, lp, g)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    S.smc_destroy(ctx)
    units = J * rows
    print(json.dumps({"metric": "particle*sample grad-evals/s (FP32 engine)", "value": units / (ms / 1e3),
                      "unit": UNIT, "ms_per_eval": ms, "tflops": units * flop / (ms / 1e3) / 1e12,
                      "config": {"workload": args.eval_config, "layers": [list(l) for l in layers], "J": J,
                                 "rows": rows, "chunk_rows": chunk, "params_per_particle": D,
                                 "flop_per_unit": flop, "precision": "fp32"}}), flush=True)


def tta_compare(J, n, K, seeds, every=4, explore_iters=15, explore_rounds=2):
    """Time to test accuracy, learned vs plain proposal (configuration c3).

    The proposal network is trained on exploratory trajectories of the same
    setup with other seeds (100, 101, ...: `explore_rounds` runs of
    `explore_iters` iterations each, the network trained after each run on
    everything collected so far); then, for each seed, both proposals run
    the same Linear-DA schedule (C = kappa = 1000, K iterations, HMC S = 3)
    from that seed.  The clock runs over the sampler iterations
    (GPU-synchronous; the test-set evaluations every `every` iterations are
    excluded) until the test accuracy first reaches the plain run's final
    accuracy minus 0.5 pt.  Reported per seed and as medians, without and with
    the training time charged to the learned proposal."""
    import torch
    import synthetic
    from paper_2601_21983_gb300 import smc as S
    S.load()
    stream = torch.cuda.current_stream()
    X, y = make_data(n, seed=0)
    Xt, yt = synthetic.template_images(10000, seed=0, test=True)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    Xtd = torch.from_numpy(Xt).cuda()
    probs = torch.empty((10000, NCLS), device="cuda", dtype=torch.float32)
    model = S.make_model([("dense", DIN, H), ("dense", H, NCLS)], (DIN,), S.ACT_RELU)

    def new_ctx(seed):
        ctx = S.smc_init(model, Xd, y_class=yd, cfg=S.make_config(J, seed, S.PREC_BF16, stream=stream))
        S.smc_set_schedule(ctx, S.make_schedule("linear", MB, MB, K))
        return ctx

    # ---- training data from the sampler's own exploratory iterations (other seeds)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    trainer = new_ctx(100)
    for rnd, seed in enumerate(range(100, 100 + explore_rounds)):
        ctx = trainer if rnd == 0 else new_ctx(seed)
        if rnd > 0:
            S.smc_learned_params(ctx, S.smc_learned_params(trainer))
            F0, T0 = S.smc_learned_data(trainer)
            S.smc_learned_load_data(ctx, F0, T0)
        for k in range(1, explore_iters):
            S.smc_anneal_next(ctx)
            S.smc_resample(ctx)
            S.smc_step(ctx, STEP_H, S_LF, S.PROPOSAL_EXPLORE, groups=8, explore_sigma=0.5)
        S.smc_learned_train(ctx, 300, 0.01)
        if rnd > 0:
            S.smc_learned_params(trainer, S.smc_learned_params(ctx))
            F1, T1 = S.smc_learned_data(ctx)
            S.smc_learned_load_data(trainer, F1, T1)
            S.smc_destroy(ctx)
    trained = S.smc_learned_params(trainer)
    train_rows = len(S.smc_learned_data(trainer)[0])
    S.smc_destroy(trainer)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0

    def run(prop, seed):
        ctx = new_ctx(seed)
        if prop == S.PROPOSAL_LEARNED:
            S.smc_learned_params(ctx, trained)
        curve, clock = [], 0.0
        for k in range(1, K):
            torch.cuda.synchronize()
            a = time.perf_counter()
            S.smc_anneal_next(ctx)
            S.smc_resample(ctx)
            S.smc_step(ctx, STEP_H, S_LF, prop)
            torch.cuda.synchronize()
            clock += time.perf_counter() - a
            if k % every == 0 or k == K - 1:
                S.smc_posterior_predict(ctx, Xtd, probs)
                curve.append((k, clock, float((probs.argmax(dim=1).cpu().numpy() == yt).mean())))
        S.smc_destroy(ctx)
        return curve

    def first_reach(curve, target):
        for k, t, acc in curve:
            if acc >= target:
                return t, k
        return None, None

    per_seed = []
    for seed in seeds:
        plain, learned = run(S.PROPOSAL_PLAIN, seed), run(S.PROPOSAL_LEARNED, seed)
        target = plain[-1][2] - 0.005
        tp, kp = first_reach(plain, target)
        tl, kl = first_reach(learned, target)
        per_seed.append({"seed": seed, "target_acc": target, "plain_final_acc": plain[-1][2],
                         "learned_final_acc": learned[-1][2], "plain_s": tp, "learned_s": tl,
                         "plain_iters": kp, "learned_iters": kl,
                         "plain_run_s": plain[-1][1], "learned_run_s": learned[-1][1],
                         "speedup": (tp / tl) if (tp and tl) else None,
                         "speedup_with_training": (tp / (tl + train_s)) if (tp and tl) else None})

    def med(key):
        v = [r[key] for r in per_seed if r[key] is not None]
        return float(np.median(v)) if v else None

    return {"metric": "time-to-test-acc, learned vs plain proposal", "unit": "s", "higher_is_better": False,
            "value": med("learned_s"), "plain_value": med("plain_s"), "speedup": med("speedup"),
            "speedup_with_training": med("speedup_with_training"), "train_seconds": train_s,
            "train_rows": train_rows, "train_budget": {"rounds": explore_rounds, "explore_iters": explore_iters,
                                                        "adam_epochs_per_round": 300},
            "seeds": per_seed,
            "config": {"workload": f"c3: MLP {DIN}-{H}-{NCLS} ReLU, J={J}, {n} synthetic images, Linear DA "
                                   f"(C=kappa={MB}, K={K}), HMC S={S_LF}, h={STEP_H}, BF16, seeds {list(seeds)}",
                       "test_rows": 10000, "eval_every": every,
                       "target": "plain proposal's final test accuracy minus 0.5 pt, per seed"}}


def run_tta(args):
    print(json.dumps(tta_compare(args.J, args.n, args.tta_iters, list(range(args.tta_seeds)), args.tta_every,
                                 args.tta_explore, args.tta_rounds)), flush=True)


def run_grid(args):
    """The scheme grid of Sec. 4 (Table 1) on a synthetic stand-in: every
    data-annealing scheme (Sec. 3.1: Constant, FB, CTR, Linear, Automated, SDA,
    and Constant / CTR with a fresh mini-batch per iteration) x {LD (S = 1),
    HMC (S = 3)} from the same seed for K iterations, C = kappa = the
    mini-batch size.  Runtime = GPU-synchronous wall time over the
    iterations (test evaluation excluded); then the posterior-predictive
    accuracy and NLL on a separate test draw.  --grid-model mlp: the
    MNIST-shaped images with MLP 784-100-10; cnn: the CIFAR-shaped images with
    the CNN (BF16 CNN engine)."""
    import torch
    from paper_2601_21983_gb300 import smc as S
    S.load()
    stream = torch.cuda.current_stream()
    import synthetic
    if args.grid_model == "cnn":
        n = args.grid_n or 10000
        X, y = synthetic.smooth_field_images(n, seed=0)
        Xt, yt = synthetic.smooth_field_images(2000, seed=0, test=True)
        model = S.make_model(CNN_LAYERS, (3, 32, 32), S.ACT_TANH)
        desc = (f"CNN conv5x5 3->16, pool, conv5x5 16->32, pool, fc 800->{NCLS} (tanh), J={args.J}, {n} synthetic "
                f"3x32x32 smooth-field images")
    else:
        n = args.grid_n or args.n
        X, y = make_data(n, seed=0)
        Xt, yt = synthetic.template_images(10000, seed=0, test=True)
        model = S.make_model([("dense", DIN, H), ("dense", H, NCLS)], (DIN,), S.ACT_RELU)
        desc = f"MLP {DIN}-{H}-{NCLS} ReLU, J={args.J}, {n} synthetic images"
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    Xtd = torch.from_numpy(Xt).cuda()
    probs = torch.empty((len(yt), NCLS), device="cuda", dtype=torch.float32)
    K, mb = args.grid_iters, args.grid_mb
    rows = []
    for kernel, steps in [("LD", 1), ("HMC", S_LF)]:
        for scheme in ["constant", "fb", "ctr", "linear", "automated", "sda", "constant_fresh", "ctr_fresh"]:
            ctx = S.smc_init(model, Xd, y_class=yd, cfg=S.make_config(args.J, 7, S.PREC_BF16, stream=stream))
            S.smc_set_schedule(ctx, S.make_schedule(scheme, mb, mb, K, delta_s=1.0))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rows_seen = 0
            for _ in range(1, K):
                info = S.smc_anneal_next(ctx)
                S.smc_resample(ctx)
                S.smc_step(ctx, STEP_H, steps)
                rows_seen += info["rows"]
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            S.smc_posterior_predict(ctx, Xtd, probs)
            p = probs.double().cpu().numpy()
            acc = float((p.argmax(axis=1) == yt).mean())
            nll = float(-np.mean(np.log(np.maximum(p[np.arange(len(yt)), yt], 1e-300))))
            S.smc_destroy(ctx)
            rows.append({"kernel": kernel, "scheme": scheme, "seconds": secs, "test_acc": acc, "test_nll": nll,
                         "mean_subset_rows": rows_seen / (K - 1)})
    for r in rows:
        fb = next(q for q in rows if q["kernel"] == r["kernel"] and q["scheme"] == "fb")
        r["speedup_vs_fb"] = fb["seconds"] / r["seconds"]
    print(json.dumps({"metric": "scheme grid (Sec. 4 Table 1 on synthetic stand-ins)", "rows": rows,
                      "config": {"workload": f"{desc}, C=kappa={mb}, K={K}, h={STEP_H}, BF16, seed 7",
                                 "test_rows": len(yt)}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--J", type=int, default=J_DEFAULT)
    ap.add_argument("--rows", "--n", dest="n", type=int, default=N_TRAIN, help="training rows (images)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-roofline", action="store_true")
    ap.add_argument("--tta", action="store_true", help="time-to-test-accuracy, learned vs plain proposal")
    ap.add_argument("--eval-config", choices=sorted(EVAL_CONFIGS),
                    help="gradient-evaluation throughput of another configuration (FP32 engine)")
    ap.add_argument("--grid", action="store_true", help="every DA scheme x {LD, HMC}: runtime and test accuracy")
    ap.add_argument("--grid-iters", type=int, default=200)
    ap.add_argument("--grid-model", choices=["mlp", "cnn"], default="mlp")
    ap.add_argument("--grid-n", type=int, default=0, help="training rows of the grid (0: 60000 mlp, 10000 cnn)")
    ap.add_argument("--grid-mb", type=int, default=500)
    ap.add_argument("--dist-backend", default="nccl", help="collective backend of multi-rank runs (gloo: tests)")
    ap.add_argument("--trace", action="store_true", help="add each timed step's global ESS and ancestors")
    ap.add_argument("--tta-iters", type=int, default=200)
    ap.add_argument("--tta-seeds", type=int, default=5)
    ap.add_argument("--no-tta", action="store_true", help="leave the time-to-accuracy comparison out of the line")
    ap.add_argument("--no-scale", action="store_true", help="leave the 784-400-400-10 J = 1024 section out")
    ap.add_argument("--scale-only", action="store_true", help="only the 784-400-400-10 J = 1024 section")
    ap.add_argument("--scale-steps", type=int, default=5)
    ap.add_argument("--scale-J", type=int, default=SCALE_J, help="particles of the scale section (profiling runs)")
    ap.add_argument("--scale-n", type=int, default=N_TRAIN, help="rows of the scale section (profiling runs)")
    ap.add_argument("--no-cnn", action="store_true", help="leave the CNN section out")
    ap.add_argument("--cnn-only", action="store_true", help="only the CNN section")
    ap.add_argument("--cnn-steps", type=int, default=3)
    ap.add_argument("--cnn-J", type=int, default=CNN_J, help="particles of the CNN section (profiling runs)")
    ap.add_argument("--cnn-n", type=int, default=CNN_N, help="images of the CNN section (profiling runs)")
    ap.add_argument("--tta-explore", type=int, default=15, help="exploratory iterations per training run")
    ap.add_argument("--tta-rounds", type=int, default=2, help="exploratory training runs (seeds 100, 101, ...)")
    ap.add_argument("--tta-every", type=int, default=4)
    if len(sys.argv) >= 6 and sys.argv[1] == "--oracle-worker":
        sec, j_s, m_s, seed = float(sys.argv[2]), int(sys.argv[3]), int(sys.argv[4]), int(sys.argv[5])
        which = "cnn" if "--cnn" in sys.argv[6:] else ("--scale" in sys.argv[6:])
        print(json.dumps(list(_oracle_eval_rate(sec, j_s, m_s, seed, scale=which))), flush=True)
        return
    args = ap.parse_args()
    args.steps = max(1, args.steps)
    if args.impl == "reference":
        return run_reference(args)
    if args.eval_config:
        return run_eval_config(args)
    if args.tta:
        return run_tta(args)
    if args.grid:
        return run_grid(args)
    if args.cnn_only:
        line = run_cnn_config(args.cnn_steps, max(3, args.warmup), J=args.cnn_J, n=args.cnn_n,
                              cpu=not args.no_cpu_baseline, e2e=not args.no_e2e, roofline=not args.no_roofline)
        line["n_gpus"] = 1
        print(json.dumps(line), flush=True)
        return
    if args.scale_only:
        line = run_scale_config(args.scale_steps, max(3, args.warmup), J=args.scale_J, n=args.scale_n,
                                cpu=not args.no_cpu_baseline, e2e=not args.no_e2e, roofline=not args.no_roofline)
        line["n_gpus"] = 1
        print(json.dumps(line), flush=True)
        return

    import torch
    from paper_2601_21983_gb300 import smc as S

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local % max(1, torch.cuda.device_count()))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(args.dist_backend)
    S.load()
    stream = torch.cuda.current_stream()

    # One sampler of J particles per rank (weak scaling): on N ranks the J N
    # particles are sharded J per rank over replicated data; the ranks gather
    # the log-weights for the global normalisation and ESS after every move,
    # add the SDA moments, and exchange particle rows when the global ESS falls
    # below J N / 2 (shard.py).
    X, y = make_data(args.n, seed=0)
    Xd = torch.from_numpy(X).cuda()
    yd = torch.from_numpy(y).cuda()
    model = S.make_model([("dense", DIN, H), ("dense", H, NCLS)], (DIN,), S.ACT_RELU)
    cfg = S.make_config(args.J, 1234, S.PREC_BF16, stream=stream)
    sched = S.make_schedule("linear", MB, MB, K_SCHED, k_start=K_START)
    sharded = None
    if world > 1:
        from paper_2601_21983_gb300.shard import ShardedSampler
        sharded = ShardedSampler(model, Xd, args.J * world, cfg, y_class=yd)
        ctx = sharded.ctx
        sharded.set_schedule(sched)
    else:
        ctx = S.smc_init(model, Xd, y_class=yd, cfg=cfg)
        S.smc_set_schedule(ctx, sched)
    evals = [0]
    trace = []          # (global ESS, resampled?, ancestors) per step when --trace

    def iteration(upload_next=None):
        """anneal -> resample -> move, on one context or on the sharded sampler;
        upload_next: pinned rows to stream in for the following iteration."""
        if sharded is not None:
            sharded.anneal_next()
            did, anc = sharded.resample()
        else:
            S.smc_anneal_next(ctx)
            did = S.smc_resample(ctx)
            anc = S.smc_get_ancestors(ctx, args.J) if (did and args.trace) else None
        if upload_next is not None:
            S.smc_upload_rows_async(ctx, 0, upload_next[0], upload_next[1])
        st = sharded.step(STEP_H, S_LF) if sharded is not None else S.smc_step(ctx, STEP_H, S_LF)
        evals[0] += st["grad_evals"] * st["rows"] * args.J
        if args.trace:
            trace.append([float(st["ess"]), bool(did), None if anc is None else [int(a) for a in anc]])
        return st

    def one_step(upload=None):
        if upload is not None:
            S.smc_upload_rows(ctx, 0, upload[0], upload[1])
        return iteration()

    clocks = Clocks(local) if rank == 0 else None
    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    n0, _, _ = S.smc_get_counters(ctx)
    evals[0] = 0
    trace.clear()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    h0 = time.time()
    ev0.record(stream)
    for _ in range(args.steps):
        one_step()
    ev1.record(stream)
    torch.cuda.synchronize()
    h1 = time.time()
    ms = ev0.elapsed_time(ev1)
    n1, _, _ = S.smc_get_counters(ctx)
    if clocks:
        clocks.mark(h0, h1)
    clk = clocks.stop() if clocks else None
    my_evals = evals[0]
    timed_trace = list(trace)
    red_dev = "cpu" if args.dist_backend == "gloo" else "cuda"     # gloo reduces host tensors
    t = torch.tensor([ms], dtype=torch.float64, device=red_dev)
    e = torch.tensor([float(my_evals)], dtype=torch.float64, device=red_dev)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(e, op=dist.ReduceOp.SUM)
    ms_max, total_evals = t.item(), e.item()
    value = total_evals / (ms_max / 1e3)

    # ---- end to end: subset streamed from pinned host memory every step
    e2e = None
    if not args.no_e2e:
        perm = S.smc_get_permutation(ctx, args.n)
        hx = torch.from_numpy(np.ascontiguousarray(X[perm])).pin_memory()
        hy = torch.from_numpy(np.ascontiguousarray(y[perm])).pin_memory()
        hxn, hyn = hx.numpy(), hy.numpy()
        one_step((hxn, hyn))
        torch.cuda.synchronize()
        evals[0] = 0
        t0 = time.perf_counter()
        # every step's rows cross from pinned host memory inside the timed
        # region; step i+1's copy runs on the library's copy stream while step
        # i computes and takes effect at step i+1's smc_anneal_next
        S.smc_upload_rows_async(ctx, 0, hxn, hyn)
        for i in range(args.steps):
            iteration((hxn, hyn) if i + 1 < args.steps else None)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e_evals = evals[0]
        if dist:   # whole job: every rank's evaluations over the slowest rank's time
            te = torch.tensor([el], dtype=torch.float64, device=red_dev)
            ee = torch.tensor([float(e2e_evals)], dtype=torch.float64, device=red_dev)
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            dist.all_reduce(ee, op=dist.ReduceOp.SUM)
            el, e2e_evals = te.item(), ee.item()
        e2e = {"value": e2e_evals / el, "unit": UNIT, "h2d_bytes_per_step": int(hxn.nbytes + hyn.nbytes) * world,
               "d2h_bytes_per_step": (16 * 8 + 2 * 4) * world}

    # ---- per-kernel-family times for the roofline (separate pass, events per launch)
    roof = None
    fam = None
    if not args.no_roofline:
        S.smc_destroy(ctx)
        sharded = None          # per-rank kernel times come from a plain context of J particles
        cfg_t = S.make_config(args.J, 1234 + rank, S.PREC_BF16, stream=stream, timing=1)
        ctx = S.smc_init(model, Xd, y_class=yd, cfg=cfg_t)
        S.smc_set_schedule(ctx, sched)
        one_step()
        S.smc_reset_counters(ctx)
        nsteps = 2
        for _ in range(nsteps):
            one_step()
        _, times, calls = S.smc_get_counters(ctx)
        fam = {k: {"ms": times[k], "calls": calls[k]} for k in times if calls[k]}
        hbm, tf_burst, tf_sus, src = peaks()
        M = args.n
        act_bytes = 2.0 * M * args.J * H          # one BF16 activation matrix [M][J*H]
        # algorithmic work per launch: GEMM FLOPs; the unfused head reads H1 and writes
        # dZ1^T; the fused kernel does the first-layer GEMM plus the head's three
        # contractions (logits, W2^T dlogits, dlogits h^T)
        work = {"fwd_gemm": ("tensor", 2.0 * M * args.J * H * DIN),
                "head": ("hbm", 2.0 * act_bytes + 4.0 * M),
                "fused_fwd_head": ("tensor", 2.0 * M * args.J * H * DIN + 6.0 * M * args.J * H * NCLS)}
        if calls.get("fused_fwd_head"):
            work.pop("head")      # only the particle-image kernel is counted there
            work["wgrad_gemm"] = ("tensor", 2.0 * M * args.J * H * (DIN + 1))
        else:
            work["wgrad_gemm"] = ("tensor", 2.0 * M * args.J * H * DIN)
        kern = {}
        for k, (bound, amount) in work.items():
            if calls.get(k):
                avg = times[k] / calls[k]
                if bound == "tensor":
                    # the timed step is sub-second at full clock: the burst peak applies
                    ach = amount / (avg / 1e3) / 1e12
                    kern[k] = {"bound": "tensor", "achieved": ach, "peak": tf_burst, "unit": "TFLOP/s",
                               "frac": ach / tf_burst, "frac_of_sustained": ach / tf_sus,
                               "avg_launch_ms": avg, "work_per_launch": amount}
                else:
                    ach = amount / (avg / 1e3) / 1e9
                    kern[k] = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                               "avg_launch_ms": avg, "work_per_launch": amount}
        dom = max(kern, key=lambda k: kern[k]["avg_launch_ms"])
        roof = dict(kern[dom])
        roof["kernel"] = dom
        roof["traffic"] = measured_traffic(dom, args.J, args.n)
        roof["peak_kind"] = f"{src} " + ("bf16_tflops (burst)" if roof["bound"] == "tensor" else "hbm_gbs")
        roof["others"] = {k: {"frac": round(v["frac"], 4), "achieved": round(v["achieved"], 1), "unit": v["unit"],
                              "avg_launch_ms": round(v["avg_launch_ms"], 4)} for k, v in kern.items() if k != dom}
    S.smc_destroy(ctx)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
                "config": workload_config(args), "e2e": e2e, "gpu_launches": n1 - n0,
                "clocks": clk, "roofline": roof, "families_ms": fam}
        line["config"]["parallelism"] = (f"particles sharded {args.J} per rank over {world} ranks ({args.dist_backend}):"
                                         f" global log-weight normalisation, SDA moments and resampling exchange"
                                         if world > 1 else "one GPU")
        if args.trace:
            line["trace"] = timed_trace
        if world == 1 and not args.no_scale:
            line["scale_config"] = run_scale_config(args.scale_steps, max(3, args.warmup),
                                                    cpu=not args.no_cpu_baseline)
        if world == 1 and not args.no_cnn:
            line["cnn_config"] = run_cnn_config(args.cnn_steps, max(3, args.warmup), cpu=not args.no_cpu_baseline)
        if world == 1 and not args.no_tta:
            line["tta"] = tta_compare(args.J, args.n, args.tta_iters, list(range(args.tta_seeds)), args.tta_every,
                                      args.tta_explore, args.tta_rounds)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
