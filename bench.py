#!/usr/bin/env python
"""Benchmark of the DZS TreePM step on GB300 (one JSON line on rank 0).

Workload (default): a single 128^3-particle lightcone mock, L = 256 Mpc/h,
PM mesh 256^3, FP32 forces, DZS on (merge level 3), Zel'dovich ICs at z = 49
(seed 2, sigma8 = 0.8), 96 global KDK steps uniform in ln a to z = 0, observer
at the box centre, R_lc sweeping the box once.  A "step" is one full KDK step
(kick + drift + crossing + records, Morton sort, DZS merge, tree, PM, walk +
closing kick).  W warm-up steps start from the ICs; the K timed steps continue
the run (when the run reaches a = 1 it restarts from fresh ICs outside the
timed region).  value = N_init x K / device time ("effective" particle-steps/s).

--impl reference times the FP64 CPU oracle (there is no other reference
implementation) on the same metric and workload name, each step on a 32^3
sub-box with the same particle and mesh spacing.
"""
import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s DZS FP32 vs plain FP64 at stated force error; mocks/h, p99 lat"
UNIT = "particle-steps/s"
# nominal FP32 pipe: 152 SMs x 128 lanes x 2 flop (FMA) x 2.07 GHz max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP32 arithmetic of one pair evaluation of the walk (FMA = 2; rsqrt, exp2 = 1):
# r^2 6, rsqrt 1, r 1, r^-3 2, t 2, split polynomial 22, exp 3 (r^2 scale, exp2,
# times Q), force 2, accumulate 6
FLOP_PER_PAIR = 45

# algorithmic HBM bytes per step of the streaming stages, FP32 state
# (u 12 B, p 12 B, g 12 B, k 4 B, id 4 B, flags 1 B per particle; mesh M^3)
STAGE_BYTES = {
    "kick_drift": lambda n, m3: 90 * n,
    "sort": lambda n, m3: 326 * n,
    "merge": lambda n, m3: 194 * n,
    "tree": lambda n, m3: 95 * n,
    # CIC deposit (cell bounds 8 B, delta 4 B per cell; u, k 16 B per particle)
    # and gradient + interpolation (phi 4 B per cell; u 12 B in, g 12 B out)
    "pm": lambda n, m3: 16.0 * m3 + 40 * n,
    # five passes over the mesh: Z r2c, Y, X with the Green multiply, Y^-1, Z c2r
    "fft": lambda n, m3: 40.3 * m3,
}

# DRAM bytes (read + write) of one k_walk launch from an ncu capture (step 41 of
# the bench run, z ~ 4) and the walk source it was taken on: reported as
# roofline traffic only while the source is unchanged
WALK_TRAFFIC_BYTES = 172.605e6 + 35.825e6
WALK_TRAFFIC_SRC = "86812881f7ef2e16"

# serving sample (Poisson stream of mock requests, sizes 32^3 .. 256^3)
SERVE_RATE = 4.0
SERVE_SIZES = (32, 64, 128, 256)
SERVE_BUDGET = 150e9


def splitmix64(state):
    """SplitMix64 (Steele, Lea & Flood 2014): returns (next state, output)"""
    state = (state + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return state, z ^ (z >> 31)


def serve_requests(n, seed=5, rate=SERVE_RATE):
    """Poisson arrivals (exponential gaps), N1 uniform over SERVE_SIZES,
    L = 2 N1 Mpc/h, mesh 2 N1, sigma8 uniform in [0.7, 0.9], random seeds."""
    st, t, out = seed, 0.0, []
    for i in range(n):
        st, a = splitmix64(st)
        st, b = splitmix64(st)
        st, c = splitmix64(st)
        st, d = splitmix64(st)
        t += -np.log1p(-(a >> 11) / 2.0 ** 53) / rate
        n1 = SERVE_SIZES[b % len(SERVE_SIZES)]
        out.append(dict(arrival_s=t, n1d=n1, mesh=2 * n1, box=2.0 * n1, sigma8=0.7 + 0.2 * (c >> 11) / 2.0 ** 53,
                        seed=int(d % (2 ** 31 - 1)) + 1))
    return out


def serving_sample(dzs, nreq, warm):
    """C ABI serving loop over a bounded Poisson stream; latency statistics
    over the requests after the first `warm` ones."""
    reqs = serve_requests(nreq + warm)
    st, wall, res = dzs.dzs_serve(reqs, hbm_budget_bytes=SERVE_BUDGET, steps_per_slice=8, precision=dzs.FP32)
    lat = sorted(r["latency_s"] for r in res[warm:])
    work = sum(q["n1d"] ** 3 * 96 for q in reqs)
    offered = SERVE_RATE * float(np.mean([n ** 3 for n in SERVE_SIZES])) * 96
    return {"requests": nreq, "warmup_requests": warm, "status": st, "rate_per_s": SERVE_RATE,
            "hbm_budget_GB": SERVE_BUDGET / 1e9, "wall_s": wall,
            "mocks_per_h": 3600.0 * len(res) / wall,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "effective_particle_steps_per_s": work / wall,
            "offered_particle_steps_per_s": offered,
            "note": "offered load of the stream vs what the GPU sustained; when offered > sustained the queue "
                    "grows and p99 grows with the number of requests (no steady state)"}


def batched_sample(dzs):
    """The batched configuration: 64 mocks (16 each of N1 = 32, 48, 64, 96; L =
    2 N1 Mpc/h, mesh 2 N1; seeds 1000 + i; sigma8 = 0.7 + 0.2 U, U from
    SplitMix64(4242)), all admitted at once by the serving loop, FP32."""
    st, reqs = 4242, []
    for i in range(64):
        st, z = splitmix64(st)
        n1 = (32, 48, 64, 96)[i % 4]
        reqs.append(dict(arrival_s=0.0, n1d=n1, mesh=2 * n1, box=2.0 * n1, sigma8=0.7 + 0.2 * (z >> 11) / 2.0 ** 53,
                         seed=1000 + i))
    status, wall, res = dzs.dzs_serve(reqs, hbm_budget_bytes=SERVE_BUDGET, steps_per_slice=8, precision=dzs.FP32)
    work = sum(q["n1d"] ** 3 * 96 for q in reqs)
    return {"mocks": 64, "status": status, "wall_s": wall, "particle_steps_per_s": work / wall,
            "mocks_per_h": 64 * 3600.0 / wall, "sum_N": sum(q["n1d"] ** 3 for q in reqs)}


def c3_sample(dzs, stream, steps=4):
    """512^3 particles in 1024 Mpc/h, mesh 512^3, 128 steps, merge level 4: the
    ICs, then `steps` steps at z ~ 49 timed (CUDA events on the stream)"""
    import torch
    P = dzs.params(n1d=512, mesh=512, box=1024.0, merge_level=4, nsteps=128, seed=3, precision=dzs.FP32)
    ctx = dzs.Context(P, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        ctx.ics()
        ctx.step(1)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.step(steps)
        b.record(stream)
        b.synchronize()
    ms = a.elapsed_time(b)
    ctx.close()
    return {"workload": "512^3, L = 1024 Mpc/h, mesh 512^3, FP32, steps 1..%d (z ~ 49)" % steps,
            "ms_per_step": ms / steps, "particle_steps_per_s": 512 ** 3 * steps / (ms / 1e3)}


def cufft_compare(stream, M, iters=20):
    """cuFFT (through torch.fft) r2c + Green-like multiply + c2r of an M^3 FP32
    mesh, the library comparison for the hand-written FFT stage"""
    import torch
    with torch.cuda.stream(stream):
        x = torch.randn(M, M, M, device="cuda", dtype=torch.float32)
        g = torch.rand(M, M, M // 2 + 1, device="cuda", dtype=torch.float32)
        for _ in range(3):
            y = torch.fft.irfftn(torch.fft.rfftn(x) * g, s=(M, M, M))
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(iters):
            y = torch.fft.irfftn(torch.fft.rfftn(x) * g, s=(M, M, M))
        b.record(stream)
        b.synchronize()
    del y
    return a.elapsed_time(b) / iters


def active_counts(dzs, P, stream, warmup, steps):
    """Particle count before each timed step, from an untimed replay of the
    same deterministic run (the timed loop itself never synchronises)."""
    import torch
    ctx = dzs.Context(P, stream=stream.cuda_stream)
    counts = []
    with torch.cuda.stream(stream):
        ctx.ics()
        step = 0
        for _ in range(warmup):
            ctx.step(1)
            step += 1
        for _ in range(steps):
            if step == P.nsteps:
                ctx.ics()
                step = 0
                for _ in range(warmup):
                    ctx.step(1)
                    step += 1
            counts.append(ctx.count()[0])
            ctx.step(1)
            step += 1
    ctx.close()
    return counts

C2 = dict(n1d=128, mesh=256, box=256.0, merge_level=3, seed=2, sigma8=0.8)


def workload_params(dzs, precision):
    return dzs.params(**C2, precision=precision)


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        smi = shutil.which("nvidia-smi")
        if not smi:
            return
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        self.proc = subprocess.Popen([smi, "-i", str(self.index), "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                      "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def cpu_baseline(steps_cap=96):
    """The FP64 oracle, as it stands, on a 32^3 sub-box with the bench's particle
    spacing (2 Mpc/h), mesh spacing (1 Mpc/h) and DZS parameters: a full run of
    96 steps (about 10-30 s of host CPU work)."""
    import oracle as O
    P = O.params(n1d=32, mesh=64, box=64.0, merge_level=3, seed=2, sigma8=0.8)
    st = O.initial_state(P)
    t0 = time.perf_counter()
    n = min(steps_cap, P.nsteps)
    for s in range(n):
        st, _ = O.step(P, s, st)
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 32 ** 3 * n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "full %d-step run of a 32^3-particle, 64 Mpc/h sub-box (mesh 64^3) with the bench's "
                      "spacing and DZS parameters, FP64 oracle, %.1f s" % (n, dt)}


def workload_name(warmup, steps):
    """the bench workload, as both arms name it in `config`"""
    return ("single lightcone mock: N=128^3, L=256 Mpc/h, mesh 256^3, FP32 forces (u32 lattice positions), "
            "DZS merge level 3, 96 KDK steps z=49->0, steps %d..%d timed" % (warmup, warmup + steps - 1))


def run_reference(args, rank, world):
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
    import oracle as O
    P = O.params(n1d=32, mesh=64, box=64.0, merge_level=3, seed=2, sigma8=0.8)
    st = O.initial_state(P)
    step = 0
    for _ in range(args.warmup):
        if step == P.nsteps:
            st, step = O.initial_state(P), 0
        st, _ = O.step(P, step, st)
        step += 1
    total = 0.0
    for _ in range(args.steps):
        if step == P.nsteps:
            st, step = O.initial_state(P), 0
        t0 = time.perf_counter()
        st, _ = O.step(P, step, st)
        total += time.perf_counter() - t0
        step += 1
    v = 32 ** 3 * args.steps / total
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.warmup, args.steps), "global_batch": 128 ** 3,
                       "parallelism": "host cores (%d threads)" % cores},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "each step: one FP64 oracle step of a 32^3-particle, 64 Mpc/h sub-box (mesh "
                                       "64^3) with the mock's particle and mesh spacing and DZS parameters; "
                                       "particle-steps/s of the sample"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_variant(dzs, P, stream, warmup, steps, budget_s=120.0):
    """Device time of `steps` KDK steps after `warmup` steps from the ICs, on a
    fresh context (CUDA events on the context stream).  Stops early once the
    timed steps exceed budget_s seconds; returns (steps timed, seconds)."""
    import torch
    ctx = dzs.Context(P, stream=stream.cuda_stream)
    done, total = 0, 0.0
    with torch.cuda.stream(stream):
        ctx.ics()
        ctx.step(warmup)
        torch.cuda.synchronize()
        while done < steps and ctx.count()[1] < P.nsteps:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            chunk = min(8, steps - done)
            a.record(stream)
            got = ctx.step(chunk)
            b.record(stream)
            b.synchronize()
            total += a.elapsed_time(b) / 1e3
            done += got
            if got == 0 or total > budget_s:
                break
    ctx.close()
    return done, total


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=93)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP64 and no-DZS runs")
    ap.add_argument("--serve-requests", type=int, default=24, help="serving sample size (0: skip)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import paper_2005_05328_gb300 as dzs
    from paper_2005_05328_gb300 import build as libbuild
    from paper_2005_05328_gb300 import replicas as R

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()
    dzs.load()
    stream = torch.cuda.Stream()
    P = workload_params(dzs, dzs.FP32)
    P.device = local
    P.seed = R.replica_seed(C2["seed"], rank)  # each replica runs its own mock
    ctx = dzs.Context(P, stream=stream.cuda_stream)
    n0 = P.n1d ** 3
    nst = P.nsteps
    with torch.cuda.stream(stream):
        ctx.ics()
        step = 0
        for _ in range(args.warmup):
            if step == nst:
                ctx.ics()
                step = 0
            ctx.step(1)
            step += 1
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        ctx.set_profiling(True)
        l0 = int(ctx.counters()[4])
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        segs = []
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_a.record(stream)
        done = 0
        relaunch = 0
        while done < args.steps:
            if step == nst:
                ev_b = torch.cuda.Event(enable_timing=True)
                ev_b.record(stream)
                segs.append((ev_a, ev_b))
                prof_keep = ctx.profile()
                ctx.ics()
                step = 0
                for _ in range(args.warmup):
                    ctx.step(1)
                    step += 1
                relaunch += 1
                ev_a = torch.cuda.Event(enable_timing=True)
                ev_a.record(stream)
            ctx.step(1)
            step += 1
            done += 1
        ev_b = torch.cuda.Event(enable_timing=True)
        ev_b.record(stream)
        segs.append((ev_a, ev_b))
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        clocks = sampler.stop()
        ms = sum(a.elapsed_time(b) for a, b in segs)
        prof = ctx.profile()
        cnt = ctx.counters()
        launches = int(cnt[4]) - l0
        pairs = int(cnt[2])
        n_final, _ = ctx.count()
    t_local = ms / 1e3
    units_total, t_max = R.aggregate(n0 * args.steps, t_local,
                                     device=torch.device("cuda", local) if world > 1 else None)
    value = R.throughput(units_total, t_max)

    # e2e through the public API with host buffers (rank 0 measures, others replicate)
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(dzs, P, stream, min(args.steps, nst))

    if rank != 0:
        return
    # HBM rooflines of the streaming stages (algorithmic bytes / stage time)
    counts = active_counts(dzs, P, stream, args.warmup, args.steps)
    m3 = P.mesh ** 3
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))  # measured copy bandwidth, else the 6.8 TB/s fallback
    stage_roof = {}
    for name, fn in STAGE_BYTES.items():
        ms_s = prof[name][0]
        if ms_s <= 0:
            continue
        gb = sum(fn(n, m3) for n in counts) / 1e9
        stage_roof[name] = {"bound": "hbm", "algorithmic_GB": gb, "achieved_GBs": gb / (ms_s / 1e3),
                            "frac": gb / (ms_s / 1e3) / hbm}
    # roofline of the dominant stage
    dom = max(prof, key=lambda k: prof[k][0])
    walk_ms, walk_calls = prof["walk"]
    walk_avg_s = walk_ms / 1e3 / max(1, walk_calls)
    achieved_tf = pairs / max(1, walk_calls) * FLOP_PER_PAIR / walk_avg_s / 1e12
    import hashlib
    wsrc = hashlib.sha256(open(os.path.join(ROOT, "paper_2005_05328_gb300", "csrc", "walk.cu"), "rb").read())
    traffic = WALK_TRAFFIC_BYTES if wsrc.hexdigest()[:16] == WALK_TRAFFIC_SRC else None
    roof = {"bound": "alu", "kernel": "k_walk<float> (tree walk + closing kick)", "achieved": achieved_tf,
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tf / FP32_PEAK_TFLOPS, "traffic": traffic,
            "traffic_note": "bytes of the step-41 launch (ncu, one capture); the timed launches average "
                            "over z = 49 -> 0",
            "peak_source": "nominal FP32 FMA rate 152 SM x 128 lanes x 2 x 2.07 GHz (no measured FP32 peak in "
                           "MEASURED_PEAKS.json)",
            "pairs_per_launch": pairs / max(1, walk_calls), "flop_per_pair": FLOP_PER_PAIR,
            "avg_launch_ms": walk_avg_s * 1e3, "dominant_stage": dom}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(args.warmup, args.steps),
                   "global_batch": n0 * world, "parallelism": "replicas x%d" % world,
                   "l2": "inputs larger than L2 (state + 256^3 mesh > 129 MB)", "restarts_in_timed_region": relaunch,
                   "n_active_end": int(n_final)},
        "roofline": roof,
        "stage_ms": {k: v[0] for k, v in prof.items()},
        "stage_roofline": stage_roof,
        "gpu_launches": launches,
        "clocks": clocks,
        "e2e": e2e,
    }
    if world == 1 and not args.no_compare:
        # the metric compares DZS FP32 with the plain FP64 path (no DZS, FP64
        # forces) and, for the DZS speed-up itself, FP32 without DZS
        comp = {}
        for name, kw in (("plain_fp64_no_dzs", dict(precision=dzs.FP64, dzs_on=0)),
                         ("fp32_no_dzs", dict(precision=dzs.FP32, dzs_on=0))):
            Pv = workload_params(dzs, kw["precision"])
            Pv.dzs_on = kw["dzs_on"]
            Pv.device = local
            k, sec = time_variant(dzs, Pv, stream, args.warmup, args.steps)
            comp[name] = {"value": n0 * k / sec if sec > 0 else None, "unit": UNIT, "steps_timed": k,
                          "ms_per_step": 1e3 * sec / max(1, k),
                          "ratio_dzs_fp32_over_this": (value / (n0 * k / sec)) if sec > 0 else None}
        fft_ms = prof["fft"][0] / max(1, prof["fft"][1])
        cu = cufft_compare(stream, P.mesh)
        comp["cufft_256cubed_r2c_green_c2r"] = {"ms": cu, "ours_ms": fft_ms, "ours_over_cufft_time": fft_ms / cu,
                                                "note": "torch.fft (cuFFT) rfftn * G + irfftn, FP32, same mesh"}
        line["comparisons"] = comp
    line["config"]["mocks_per_h_single_stream"] = 3600.0 / (P.nsteps * ms / args.steps / 1e3)
    line["config"]["actual_particle_steps_per_s"] = sum(counts) / (ms / 1e3)  # sum of N_active per step
    if world == 1 and args.serve_requests > 0:
        line["serving"] = serving_sample(dzs, args.serve_requests, 4)
    if world == 1 and not args.no_compare:
        line["batched"] = batched_sample(dzs)
        line["large_instance"] = c3_sample(dzs, stream)
    if world == 1 and not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as ex:  # the oracle needs gcc; report why it is missing
            line["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                    "sample": "unavailable: %s" % ex}
    print(json.dumps(line), flush=True)


def measure_e2e(dzs, P, stream, k):
    """Same metric through the C ABI with host buffers: the IC state is copied
    in from pinned host memory, then every step runs and its lightcone records
    and diagnostics are copied back to the host."""
    import torch
    ctx = dzs.Context(P, stream=stream.cuda_stream)
    with torch.cuda.stream(stream):
        ctx.ics()
        st = ctx.state()
        n = st["u"].shape[1]
        pinned = {}
        for key, arr in st.items():
            t = torch.empty(arr.shape, dtype={np.uint32: torch.int32, np.float64: torch.float64,
                                              np.uint8: torch.uint8}[arr.dtype.type], pin_memory=True)
            t.numpy().view(arr.dtype)[...] = arr
            pinned[key] = t.numpy().view(arr.dtype)
        h2d = sum(a.nbytes for a in pinned.values())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_state(pinned, 0)
        d2h = 0
        for _ in range(k):
            ctx.step(1)
            rec = ctx.drain(cap=n)
            d = ctx.diagnostics()
            d2h += rec.nbytes + d.nbytes
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ctx.close()
    return {"value": P.n1d ** 3 * k / wall, "unit": UNIT, "h2d_bytes_per_step": h2d / k,
            "d2h_bytes_per_step": d2h / k, "steps": k}


if __name__ == "__main__":
    main()
