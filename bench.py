"""Benchmark of the probed FWI gradient (Gpts/s fwd+adj) on GB300.

One step = one probed gradient (forward sweep with windowed probe GEMMs,
residual/misfit, adjoint sweep with probe GEMMs, combine, gradient norm)
over the 3-D workload: 256^3 grid at 10 m, nt = 2000, 8th order, one shot,
256 x 256 surface receivers, r = 32 Rademacher probes, window T = 32.
The full-storage gradient (N x nt history) of the same problem is timed
beside it.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank runs an independent replica (shots are
independent; no data-path collective): `value` = all ranks' grid-point
updates / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gpts/s fwd+adj, probed vs full-storage gradient; err vs FP64; p50/p99 latency"
STENCIL_BYTES_PER_POINT = 16  # read u[t], u[t-1], c; write u[t+1] (fp32)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="config3", choices=["config1", "config2", "config3", "config4"],
                    help="config3 (3-D 256^3) is the headline; the 2-D configs are L2-resident")
    ap.add_argument("--n", type=int, default=256, help="grid points per axis")
    ap.add_argument("--nt", type=int, default=2000)
    ap.add_argument("--r", type=int, default=32)
    ap.add_argument("--T", type=int, default=32)
    ap.add_argument("--form", default="auto", choices=["auto", "levels", "increment", "compensated"],
                    help="fp32 time-stepping form (auto: compensated forward for 2-D grids that fit one cluster)")
    ap.add_argument("--acc", default="f32", choices=["f32", "bf16", "bf16_kahan", "f32_fold"],
                    help="probe accumulator storage of the headline gradient")
    ap.add_argument("--no-fold", action="store_true", help="skip the single-accumulator comparison")
    ap.add_argument("--no-full", action="store_true", help="skip the full-storage comparison")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-nt", type=int, default=48, help="time levels of the bounded CPU sample")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving (p50/p99) leg")
    ap.add_argument("--serve-requests", type=int, default=100)
    ap.add_argument("--no-2d", action="store_true",
                    help="skip the 2-D configurations (1, 2, 4) and config 4's precision leg (N = 1 only)")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("bf16_tflops", 1903.7)), "measured"
    return 6800.0, 1900.0, "fallback"


def profile_traffic(kernel_file: str, src_file: str, key: str):
    """dram bytes per launch recorded by an ncu capture in profiles/, if the
    kernel source has not changed since (hash match) and the capture is of
    this workload (`applies_to` = key); else None."""
    path = os.path.join(ROOT, "profiles", kernel_file)
    if not os.path.exists(path):
        return None
    with open(path) as f:
        text = f.read()
    m = re.search(r"dram_bytes_per_launch_full_size\s*=\s*([0-9.eE+]+)", text)
    h = re.search(r"source_sha256\s*=\s*([0-9a-f]+)", text)
    a = re.search(r"applies_to\s*=\s*(.+)", text)
    if not m or not h or not a or a.group(1).strip() != key:
        return None
    with open(os.path.join(ROOT, src_file), "rb") as f:
        cur = hashlib.sha256(f.read()).hexdigest()[:16]
    return float(m.group(1)) if cur == h.group(1)[:16] else None


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ workloads
def make_workload(args, nt=None, seed_offset=0):
    from paper_2104_00794_gb300 import workloads as wl
    seed = wl.DEFAULT_SEED + seed_offset
    if args.workload == "config3":
        return wl.config3(n=args.n, nt=nt or args.nt, T=args.T, r=args.r, seed=seed)
    w = {"config1": wl.config1, "config2": wl.config2, "config4": wl.config4}[args.workload](seed=seed)
    if nt:
        w = truncate(w, nt)
    return w


def truncate(w, nt):
    import dataclasses
    return dataclasses.replace(w, nt=nt, wavelet=np.ascontiguousarray(w.wavelet[:, :nt]), name=w.name + f"_nt{nt}")


def cpu_sample(args):
    """A bounded sample of the workload for the FP64 oracle (10-30 s of CPU)."""
    w = make_workload(args)
    if args.workload == "config3":
        return make_workload(args, nt=args.cpu_nt), f"256^3 grid, nt={args.cpu_nt} of {w.nt} levels, r={w.r}"
    import dataclasses
    shots = 1 if args.workload != "config1" else w.nshots
    ws = dataclasses.replace(w, nshots=shots, src=w.src[:shots], rec=w.rec[:shots], wavelet=w.wavelet[:shots])
    if args.workload != "config1":
        ws = truncate(ws, min(w.nt, 1500))
    return ws, f"{shots} of {w.nshots} shots, nt={ws.nt} of {w.nt}, r={w.r}"


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank: int):
    """The FP64 CPU oracle on a bounded sample of the same workload."""
    if rank != 0:
        return
    import oracle
    from paper_2104_00794_gb300 import workloads as wl
    w, sample = cpu_sample(args)
    dobs = wl.synthetic_data(w.nshots, w.nt, w.nrec, seed=7)
    oracle.build()
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.batch_gradient_probed(w, w.vel0, dobs)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    t = statistics.median(times)
    v = 2.0 * w.N * w.nt * w.nshots / t / 1e9
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "Gpts/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": make_workload(args).name, "sample": f"probed gradient, {sample}",
                   "grid": [w.nz, w.ny, w.nx], "r": w.r},
        "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving leg
# Request shapes of the serving mix (config 5): 2-D grids 201^2 .. 1001x401 and
# 3-D 128^3 .. 320^3, nt 1000-4000, r in {8, 16, 32}, order 8.  Requests of one
# shape differ in their source position, their model and their data.
SERVE_SHAPES = [("2d", (201, 201), 1000, 8), ("2d", (601, 301), 2000, 16), ("2d", (1001, 401), 3000, 16),
                ("2d", (401, 401), 4000, 32), ("3d", 128, 1000, 8), ("3d", 192, 2000, 16), ("3d", 256, 2000, 32),
                ("3d", 320, 1000, 16)]


def serving_mix(n: int, seed: int):
    """n probed-gradient requests (one shot each) drawn from SERVE_SHAPES.
    Per shape one base model (seeded, on the host); per request a source
    position, a model scaled by a factor in [0.97, 1] of the base and
    synthetic observed data, made on the device."""
    import torch
    from paper_2104_00794_gb300 import api, serve
    from paper_2104_00794_gb300 import workloads as wl
    rng = np.random.default_rng(seed)
    bases = []
    for i, (dim, size, nt, r) in enumerate(SERVE_SHAPES):
        if dim == "2d":
            w = wl.small_2d(nx=size[0], nz=size[1], nt=nt, order=8, r=r, probe_kind="rademacher", h=10.0, dt=1e-3,
                            f0=10.0, seed=seed + i)
        else:
            w = wl.config3(n=size, nt=nt, r=r, seed=seed + i, rec_stride=2)
        bases.append((w, torch.tensor(np.ascontiguousarray(w.vel0), device="cuda"),
                      torch.tensor(np.ascontiguousarray(w.wavelet), device="cuda")))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    reqs = []
    for i in range(n):
        w, vel, wav = bases[int(rng.integers(len(bases)))]
        src = int(w.src[0, 0])
        if w.ndim == 2:
            src = src - (src % w.nx) + int(rng.integers(w.nx // 8, w.nx - w.nx // 8))
        else:
            plane = w.nx * w.ny
            src = (src // plane) * plane + int(rng.integers(w.ny // 4, 3 * w.ny // 4)) * w.nx + \
                int(rng.integers(w.nx // 4, 3 * w.nx // 4))
        vmax = float(w.vel0.max())
        p = api.Problem(w.ndim, w.nx, w.ny, w.nz, w.h, w.dt, w.nt, w.order, [[src]], w.rec[:1], vmax=vmax)
        v = vel * (1.0 - 0.03 * float(rng.uniform()))
        d_obs = 1e-3 * torch.randn((1, w.nt, w.rec.shape[1]), device="cuda", generator=gen)
        probe = api.ProbeSpec(kind="rademacher", r=w.r, T=32, seed=w.seed)
        reqs.append((serve.GradientJob(p, v, wav, d_obs, probe), 2.0 * w.N * w.nt))
    return reqs


def run_serving(args, rank):
    import torch
    from paper_2104_00794_gb300 import serve
    jobs = serving_mix(args.serve_requests, seed=wl_seed() + 17 * rank)
    torch.cuda.synchronize()
    work = [wk for _, wk in jobs]
    # service-time estimate from the 3-D rate, arrival rate for ~75 % busy
    est = float(np.mean(work)) / 150e9
    rng = np.random.default_rng(99 + rank)
    arrivals = np.cumsum(rng.exponential(est / 0.75, size=len(jobs)))
    arrivals -= arrivals[0]
    reqs = [serve.Request(i, float(arrivals[i]), j.footprint(), work[i], j) for i, (j, _) in enumerate(jobs)]
    budget = int(80e9)
    sched = serve.Scheduler(budget, max_slots=8)
    ex = serve.GpuExecutor(cache_bytes=int(60e9))
    t0 = time.perf_counter()
    serve.run(reqs, sched, ex.start, ex.poll)
    torch.cuda.synchronize()
    makespan = time.perf_counter() - t0
    s = serve.summarize(reqs, makespan, captured=ex.captured)
    s.update({"slots_max": sched.max_slots, "peak_concurrent": sched.peak_active, "budget_bytes": budget,
              "peak_bytes": sched.peak_used, "shapes": len(SERVE_SHAPES),
              "mix": "2-D 201^2..1001x401 and 3-D 128^3..320^3, nt 1000-4000, r 8/16/32 (8 shapes)",
              "arrivals": "Poisson, rate for ~75 % busy"})
    s.update(ex.stats())
    return s


def graph_time(fn, steps, warmup):
    """ms per call of fn captured once as a CUDA graph and replayed (CUDA
    events on the current stream, W warm-up replays)."""
    import torch
    fn()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        g = torch.cuda.CUDAGraph()
        g.capture_begin()
        fn()
        g.capture_end()
    torch.cuda.synchronize()
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def run_2d(args):
    """The 2-D configurations (L2-resident batches on the persistent cluster
    path): probed-gradient Gpts/s in the default form and in the levels form,
    and config 4's errors against FP64 on two of its shots (the default
    compensated form, the levels form, bf16 and bf16 + compensation storage,
    and the autograd backward)."""
    import torch
    import oracle
    from paper_2104_00794_gb300 import api
    from paper_2104_00794_gb300 import workloads as wl
    from paper_2104_00794_gb300.autograd import modeling
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    out = {}
    for name in ("config1", "config2", "config4"):
        w = getattr(wl, name)()
        vel_true, vel0, wav = dev(w.vel_true), dev(w.vel0), dev(w.wavelet)
        rec = {"workload": w.name, "shots": w.nshots}
        for form in ("auto", "levels"):
            p = api.Problem.from_workload(w, form=form)
            d_obs = p.forward(vel_true, wav).clone()
            spec = api.ProbeSpec(kind=w.probe_kind, r=w.r, T=w.T, seed=w.seed)
            grad = torch.empty(p.shape, dtype=torch.float32, device="cuda")
            scal = torch.empty(2, dtype=torch.float64, device="cuda")
            ms = graph_time(lambda: p.gradient_probed(vel0, wav, d_obs, spec, grad=grad, scalars=scal),
                            args.steps, args.warmup)
            key = "default" if form == "auto" else "levels"
            rec[key] = {"form": p.form, "ms_per_step": ms, "value": 2.0 * w.N * w.nt * w.nshots / (ms * 1e-3) / 1e9,
                        "unit": "Gpts/s"}
            p.release()
            del p
        out[name] = rec
    # config 4's precision on two of its shots (the oracle takes about a minute per pair)
    w = wl.config4()
    k = [0, w.nshots - 1]
    w = dataclasses.replace(w, nshots=2, src=w.src[k], rec=w.rec[k], wavelet=np.ascontiguousarray(w.wavelet[k]))
    dobs = oracle.batch_forward(w, w.vel_true).astype(np.float32)
    t0 = time.perf_counter()
    ref, J = oracle.batch_gradient_probed(w, w.vel0, dobs)
    t_or = time.perf_counter() - t0
    vel0, wav, d_obs = dev(w.vel0), dev(w.wavelet), dev(dobs)
    rel = lambda g: float(np.linalg.norm(g.double().cpu().numpy().ravel() - ref) / np.linalg.norm(ref))
    errs = {}
    for form in ("auto", "levels"):
        p = api.Problem.from_workload(w, form=form)
        for acc in (("f32", "bf16", "bf16_kahan") if form == "auto" else ("f32",)):
            g, _ = p.gradient_probed(vel0, wav, d_obs, api.ProbeSpec(kind="gaussian", r=16, T=w.T, seed=w.seed, acc=acc))
            errs[f"{p.form}_{acc}"] = rel(g)
            p.release()
    p = api.Problem.from_workload(w)
    v = vel0.clone().requires_grad_(True)
    loss = 0.5 * ((modeling(v, p, wav, api.ProbeSpec(kind="gaussian", r=16, T=w.T, seed=w.seed)) - d_obs).double() ** 2).sum()
    loss.backward()
    gv_ref = ref * (-2.0 / w.vel0.astype(np.float64).ravel() ** 3)
    ag = float(np.linalg.norm(v.grad.double().cpu().numpy().ravel() - gv_ref) / np.linalg.norm(gv_ref))
    out["config4_precision"] = {
        "case": (f"2 of the 8 shots (first and last), 801x301, nt=2500, r=16 Gaussian, T={w.T}, "
                 "same probes as the FP64 oracle"),
        "probed_gradient_rel_l2": errs, "autograd_backward_rel_l2": ag,
        "misfit_rel": abs(float(loss.detach()) - J) / J, "oracle_seconds": t_or}
    return out


def wl_seed():
    from paper_2104_00794_gb300 import workloads as wl
    return wl.DEFAULT_SEED


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    from paper_2104_00794_gb300.replicas import Replicas
    reps = Replicas()
    world, rank, local = reps.world, reps.rank, reps.local
    if args.impl == "reference":
        return run_reference(args, rank)

    import torch
    from paper_2104_00794_gb300 import api, native
    from paper_2104_00794_gb300 import workloads as wl

    torch.cuda.set_device(local)
    reps.init("nccl", torch.device("cuda", local))

    def barrier():
        reps.barrier()
        torch.cuda.synchronize()

    max_over_ranks = reps.max_over_ranks

    w = make_workload(args, seed_offset=reps.seed_offset())
    p = api.Problem.from_workload(w, form=args.form)
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")  # copies (inputs may be read-only)
    vel_true, vel0, wav = dev(w.vel_true), dev(w.vel0), dev(w.wavelet)
    d_obs = p.forward(vel_true, wav).clone()  # observed data of the true model (setup, untimed)
    probe = api.ProbeSpec(kind=w.probe_kind, r=w.r, T=w.T, seed=w.seed, acc=args.acc)
    grad = torch.empty(p.shape, dtype=torch.float32, device="cuda")
    scal = torch.empty(2, dtype=torch.float64, device="cuda")
    pts = 2.0 * w.N * w.nt * w.nshots  # grid-point updates per gradient (fwd + adj)
    stream = torch.cuda.current_stream()

    def timed(fn, steps, warmup, prof=False):
        for _ in range(warmup):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if prof:
            native.tp_profile_begin(60000)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        barrier()
        kern = native.tp_profile_end() if prof else None
        return e0.elapsed_time(e1) / steps, kern

    def graph_timed(fn, clocks=None):
        """The whole call captured once as a CUDA graph (every kernel of the
        library, no host work per launch) and replayed K times after W warm-up
        replays; a second graph with CUDA-event pairs around every kernel gives
        the per-kernel durations (of its last replay, scaled to K gradients)."""
        fn()
        torch.cuda.synchronize()
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            g_clean = torch.cuda.CUDAGraph()
            g_clean.capture_begin()
            fn()
            g_clean.capture_end()
            native.tp_profile_begin(60000)
            g_prof = torch.cuda.CUDAGraph()
            g_prof.capture_begin()
            fn()
            g_prof.capture_end()
        torch.cuda.synchronize()
        if clocks is not None:
            with clocks:
                ms_, _ = timed(g_clean.replay, args.steps, args.warmup)
        else:
            ms_, _ = timed(g_clean.replay, args.steps, args.warmup)
        timed(g_prof.replay, 1, 1)
        k1 = native.tp_profile_end()
        del g_clean, g_prof
        return ms_, {k: {"ms": v["ms"] * args.steps, "launches": v["launches"] * args.steps} for k, v in k1.items()}

    # ---- probed gradient (headline)
    run_probed = lambda: p.gradient_probed(vel0, wav, d_obs, probe, grad=grad, scalars=scal)
    clk = Clocks(local)
    ms, kern = graph_timed(run_probed, clocks=clk)
    clocks = clk.summary()
    p.status(native.OP_GRADIENT_PROBED)
    ms_max = max_over_ranks(ms)
    value = reps.whole_job_rate(pts, ms_max) / 1e9
    grad_probed = grad.clone()
    mem = api.memory_model(p, probe)
    p.release()

    # ---- end to end through the public API with pinned host buffers (right after the
    # headline, on the same problem, before the larger legs)
    e2e = None
    if not args.no_e2e:
        h_vel = torch.from_numpy(np.array(w.vel0, dtype=np.float32, copy=True)).pin_memory()
        h_wav = torch.from_numpy(np.array(w.wavelet, dtype=np.float32, copy=True)).pin_memory()
        h_dobs = d_obs.cpu().pin_memory()
        h_grad = torch.empty(p.shape, dtype=torch.float32).pin_memory()
        h_scal = torch.empty(2, dtype=torch.float64).pin_memory()
        # the public graphed call: host inputs in, the two halves replayed as graphs, gradient and scalars out
        gg = api.GraphedGradient(p, probe)

        def run_e2e():
            gg(h_vel, h_wav, h_dobs, grad_out=h_grad, scalars_out=h_scal)

        clk_e = Clocks(local)
        with clk_e:
            ems, _ = timed(run_e2e, args.steps, args.warmup)
        ems = max_over_ranks(ems)
        h2d = h_vel.numel() * 4 + h_wav.numel() * 4 + h_dobs.numel() * 4
        e2e = {"value": pts * world / (ems * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_step": ems,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h_grad.numel() * 4 + 16),
               "api": "api.GraphedGradient (captured once, replayed per call; d_obs uploaded beside the forward half)",
               "clocks": clk_e.summary()}
        del gg
        p.release()

    # ---- roofline of the dominant kernel (leapfrog stencil step)
    hbm_peak, _, peak_kind = measured_peaks()
    st = kern["stencil_step"]
    # time per time step (a 2-D launch on the cluster path runs many steps)
    steps_per_grad = 2 * (w.nt - 2)
    avg_stencil_ms = st["ms"] / (args.steps * steps_per_grad)
    stencil_bytes = STENCIL_BYTES_PER_POINT * w.N * w.nshots
    achieved = stencil_bytes / (avg_stencil_ms * 1e-3) / 1e9
    key = f"{w.ndim}d {w.nx}^3 r{w.r} T{w.T}" if (w.ndim == 3 and w.nx == w.ny == w.nz) else w.name
    traffic = profile_traffic("stencil_step_3d_256cubed.md", "paper_2104_00794_gb300/csrc/tp_sweep3d_tma.cu", key)
    gemm_traffic = profile_traffic("probe_gemm_3d_256cubed.md", "paper_2104_00794_gb300/csrc/tp_gemm.cu", key)
    if getattr(w, "sponge", 0):  # the captures are of the undamped kernels
        traffic = None
    gm = kern["probe_gemm_tcgen05"]
    avg_gemm_ms = gm["ms"] / max(gm["launches"], 1)
    # algorithmic bytes of one window GEMM: T snapshots read + r accumulators read and written
    from paper_2104_00794_gb300.native import tp_probe  # noqa: F401
    # the GEMM walks interior row segments of 128 points: T snapshots read,
    # r accumulators read and written per point
    gemm_pts = w.nz * w.ny * ((w.nx + 127) // 128 * 128) * w.nshots
    gemm_bytes = gemm_pts * 4 * (w.T + 2 * w.r)
    gemm_flops = 2.0 * gemm_pts * w.T * w.r * 2  # hi and lo products (Rademacher probes exact in tf32)
    launches = sum(v["launches"] for v in kern.values())

    # ---- single-accumulator form (one N r set, vbar folded into the gradient)
    fold = None
    if not args.no_fold and args.acc == "f32" and w.r <= 32:
        fprobe = dataclasses.replace(probe, acc="f32_fold")
        run_fold = lambda: p.gradient_probed(vel0, wav, d_obs, fprobe, grad=grad, scalars=scal)
        fdms, fdkern = graph_timed(run_fold)
        fdms = max_over_ranks(fdms)
        p.status(native.OP_GRADIENT_PROBED)
        rel = float((grad.double() - grad_probed.double()).norm() / grad_probed.double().norm())
        fg = fdkern.get("probe_gemm_tcgen05", {"ms": 0.0, "launches": 0})
        fold = {"value": pts * world / (fdms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_step": fdms,
                "workspace_bytes": p.workspace_bytes(native.OP_GRADIENT_PROBED, fprobe),
                "accumulator_values": mem["probed_accumulator_values"] // 2,
                "rel_l2_vs_two_sets": rel,
                "gemm_ms_per_launch": fg["ms"] / max(fg["launches"], 1),
                "kernels": {k: v for k, v in fdkern.items() if v["launches"]}}
        p.release()

    # ---- full-storage gradient of the same problem
    full = None
    if not args.no_full:
        run_full = lambda: p.gradient_full(vel0, wav, d_obs, grad=grad, scalars=scal)
        fms, fkern = graph_timed(run_full)
        fms = max_over_ranks(fms)
        g_full = grad.clone()
        cos = float(torch.nn.functional.cosine_similarity(grad_probed.double().ravel(), g_full.double().ravel(), dim=0))
        full = {"value": pts * world / (fms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_step": fms,
                "probed_over_full_runtime": ms_max / fms,
                "workspace_bytes": mem["workspace_full_bytes"],
                "history_bytes_algorithmic": 4 * mem["full_history_values"],
                "cosine_probed_vs_full_gradient": cos,
                "kernels": {k: v for k, v in fkern.items() if v["launches"]}}
        p.release()

    # ---- CPU baseline (the FP64 oracle, bounded sample), rank 0 at N = 1 only
    cpu = None
    err = None
    if not args.no_cpu and rank == 0 and world == 1:
        import oracle
        wc, sample = cpu_sample(args)
        pc = api.Problem.from_workload(wc)
        dobs_c = wl.synthetic_data(wc.nshots, wc.nt, wc.nrec, seed=7)
        oracle.build()
        t0 = time.perf_counter()
        gref, Jref = oracle.batch_gradient_probed(wc, wc.vel0, dobs_c)
        tc = time.perf_counter() - t0
        gcpu, sc = pc.gradient_probed(dev(wc.vel0), dev(wc.wavelet), dev(dobs_c),
                                      api.ProbeSpec(kind=wc.probe_kind, r=wc.r, T=wc.T, seed=wc.seed))
        gg = gcpu.double().cpu().numpy().ravel()
        err = {"probed_gradient_rel_l2": float(np.linalg.norm(gg - gref) / np.linalg.norm(gref)),
               "misfit_rel": abs(float(sc[0].item()) - Jref) / Jref,
               "case": f"{sample}, same probes"}
        cpu = {"value": 2.0 * wc.N * wc.nt * wc.nshots / tc / 1e9, "unit": "Gpts/s", "cores": os.cpu_count(),
               "kind": "oracle", "sample": f"probed gradient, {sample}", "seconds": tc}
        pc.release()

    # ---- the 2-D configurations and config 4's precision (N = 1)
    configs_2d = None
    if not args.no_2d and args.workload == "config3" and world == 1:
        configs_2d = run_2d(args)

    # ---- serving: Poisson stream of mixed-size shot-gradient requests
    serving = None
    if not args.no_serve and args.workload == "config3":
        serving = run_serving(args, rank)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "execution": "CUDA graph replay of the whole gradient",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "grid": [w.nz, w.ny, w.nx], "h_m": w.h, "nt": w.nt, "dt_s": w.dt,
                       "order": w.order, "shots_per_gpu": w.nshots, "nrec": w.nrec, "r": w.r, "T": w.T,
                       "probes": w.probe_kind,
                       "l2": ("inputs larger than L2 (fields 67 MB, >100 GB streamed per step)" if w.ndim == 3 else
                              "2-D batch is L2-resident (no flush): reported for completeness, not an HBM roofline"),
                       "parallelism": f"replicas x{world}"},
            "roofline": {"kernel": "stencil_step", "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                         "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": peak_kind,
                         "traffic": traffic, "bytes_per_step_algorithmic": stencil_bytes,
                         "avg_step_ms": avg_stencil_ms, "launches": st["launches"],
                         "steps": args.steps * steps_per_grad, "form": p.form},
            "probe_gemm": {"avg_launch_ms": avg_gemm_ms, "launches": gm["launches"],
                           "bytes_per_launch_algorithmic": gemm_bytes,
                           "achieved_gbs": gemm_bytes / (avg_gemm_ms * 1e-3) / 1e9 if gm["launches"] else None,
                           "frac_of_hbm": (gemm_bytes / (avg_gemm_ms * 1e-3) / 1e9 / hbm_peak
                                           if gm["launches"] and hbm_peak else None),
                           "traffic": gemm_traffic,
                           "tensor_tflops": gemm_flops / (avg_gemm_ms * 1e-3) / 1e12 if gm["launches"] else None},
            "kernels": {k: v for k, v in kern.items() if v["launches"]},
            "gpu_launches": launches,
            "clocks": clocks,
            "memory": mem,
            "single_accumulator": fold,
            "full_storage": full,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "err_vs_fp64": err,
            "serving": serving,
            "configs_2d": configs_2d,
        }
        print(json.dumps(line), flush=True)
    reps.close()


if __name__ == "__main__":
    main()
