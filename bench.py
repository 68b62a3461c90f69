#!/usr/bin/env python3
"""Throughput of the batched per-wavenumber inversion on the 2D production workload.

Workload: 512 shots x 512 receivers (dx 12.5 m, periodic line), 128 frequencies 3-60 Hz,
256 depths of 8 m, a 20-layer reference (seeded), a Gaussian-correlated 3 % random
velocity field, complex64 Born data from the library's own forward model plus complex
Gaussian noise at 20 dB SNR per frequency, damping alpha = 1e-2 (lam = alpha trace G).
One step = one full inversion (all 257 split systems standing for the 512 midpoint
wavenumbers): depth march, data transform, right-hand sides, tensor-core Gram, double-float
(FP64-class) Cholesky, one refinement step, inverse transform.  Subproblems counted = nx (512)
per inversion, one per midpoint wavenumber.  Independent lines are inverted two at a time
(--lines-in-flight), each with its own context and CUDA stream, consecutive steps alternating
between them, so that one line's tensor-core Gram overlaps another's Cholesky and refinement.

Multi-GPU: each rank inverts its own independent survey line (weak scaling, no
data-path collective); time = max over ranks.

--impl reference times the FP64 CPU oracle (the only reference this project has) on a
bounded sample of the same workload on the host cores.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "production_2d"
CPU_SAMPLE_M = (1, 64, 128, 192)      # midpoint indices solved by the CPU baseline sample


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--passes", type=int, default=3)
    ap.add_argument("--refine", type=int, default=1)
    ap.add_argument("--chol-df", type=int, default=0,
                    help="Cholesky of the mixed path: 0/1 double-float on the FP32 pipes (default), "
                         "2 native FP64")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lines-in-flight", type=int, default=2,
                    help="production line: independent lines inverted concurrently, one context "
                         "and CUDA stream each (the timed steps alternate between them)")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--freq-stride", type=int, default=1,
                    help="profiling aid: keep every k-th frequency of the 2D line (a smaller case of "
                         "the same kernels for profiler captures; not a bench line)")
    ap.add_argument("--cpu-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-autotune", action="store_true",
                    help="time the default launch shapes instead of the autotuned ones")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batched_3d", "differentiation_2d", "streaming", "paper_2d_tsvd",
                             "fma_peak"],
                    help="batched_3d: the finite-aperture 3D workload; differentiation_2d: misfit "
                         "gradients on the production geometry; streaming: 4096 independent 1D "
                         "subproblems in Poisson bursts (separate lines, not the headline)")
    return ap.parse_args()


def workload_summary(wl):
    return (f"{WORKLOAD}: {wl.nx}x{wl.nx} sources/receivers dx {wl.dx} m, {len(wl.freq_hz)} freqs "
            f"{wl.freq_hz.min():g}-{wl.freq_hz.max():g} Hz, nz {wl.nz} dz {wl.dz} m, "
            f"{len(wl.layer_top)} layers, 3% random field, c64 Born data + 20 dB noise")


# ------------------------------------------------------------------ multi-rank host logic
def line_salt(rank: int) -> int:
    """Seed salt of the survey line a rank inverts: every rank gets its own line."""
    return 1 + int(rank)


def max_over_ranks(value: float, world: int) -> float:
    """The largest of the ranks' values (the job's time); identity on one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_step: int, steps: int, ms_total: float) -> float:
    """Units processed by all ranks per second of the slowest rank's time."""
    return world * units_per_step * steps / (ms_total / 1e3)


# ------------------------------------------------------------------ CPU oracle timing
def cpu_child_window(spec):
    """Oracle sample of the batched 3D workload: kernel rows of a few (frequency, pair)
    combinations by the wavenumber-sum route and one damped QR solve, extrapolated to the
    cost of one pair (all frequencies) per two subproblems."""
    import numpy as np
    import synth
    from oracle import edt3d
    wl = synth.preset3d("batched_3d")
    reps = edt3d.pair_representatives(wl)
    nf = len(wl.freq_hz)
    m = reps[spec["pair"]]
    t_rows = []
    for f in spec["freqs"]:
        a = time.perf_counter()
        edt3d.window_dft(edt3d.kernel_offsets_spectral(wl, f, m), axes=(0, 1))
        t_rows.append(time.perf_counter() - a)
    rng = synth.rng_for(2, salt=77)
    keep = edt3d.kept_mask(wl, m)
    R = int(keep.sum())
    A = rng.standard_normal((R, wl.nz)) + 1j * rng.standard_normal((R, wl.nz))
    d = rng.standard_normal(R) + 1j * rng.standard_normal(R)
    a = time.perf_counter()
    Ahat = np.vstack([A.real, A.imag])
    from oracle.edt2d import damped_lstsq
    damped_lstsq(Ahat, np.stack([np.concatenate([d.real, d.imag])] * 2, axis=1),
                 wl.alpha * float(np.sum(Ahat ** 2)))
    t_qr = time.perf_counter() - a
    t_pair = nf * statistics.mean(t_rows) + t_qr
    rate = 2.0 / t_pair
    out = dict(value=rate, unit="subproblems/s", cores=1, kind="oracle",
               sample=(f"FP64 numpy oracle, 1 thread: kernel rows of pair {m} at frequency indices "
                       f"{spec['freqs']} by the wavenumber sum (mean {statistics.mean(t_rows):.2f} s "
                       f"per frequency, x {nf} frequencies) plus one damped QR of its {R} rows "
                       f"({t_qr:.2f} s); one pair = two subproblems; the data transform is not "
                       f"counted"))
    print("CPUJSON " + json.dumps(out))


def cpu_child_grad(spec):
    """Oracle sample of the misfit gradients: J, dJ/dV and dJ/dc of one frequency of the
    production geometry (the gradients are sums over frequencies), scaled to one full
    evaluation (all frequencies)."""
    import synth
    from oracle import edt2d, grad2d
    wl = synth.preset(WORKLOAD)
    wl.cutoff = 0.0
    nf = len(wl.freq_hz)
    wl.freq_hz = wl.freq_hz[[spec["freq"]]]
    rng = synth.rng_for(3, 11)
    Vt = synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                         wl.layer_vel)
    D = edt2d.forward(wl, Vt)
    a = time.perf_counter()
    grad2d.misfit(wl, 0.5 * Vt, D)
    grad2d.grad_V(wl, 0.5 * Vt, D)
    grad2d.grad_c(wl, 0.5 * Vt, D)
    t = time.perf_counter() - a
    out = dict(value=1.0 / (t * nf), unit="gradients/s", cores=1, kind="oracle",
               sample=(f"FP64 numpy oracle, 1 thread: J, dJ/dV and dJ/dc (forward-mode depth march, "
                       f"{len(wl.layer_vel)} layers) of frequency index {spec['freq']} "
                       f"({t:.1f} s), x {nf} frequencies"))
    print("CPUJSON " + json.dumps(out))


def cpu_child_stream(spec):
    """Oracle sample of the streaming workload: QR solves of every 512th request of the stream."""
    from synth import stream
    from oracle import stream1d
    subs = stream.stream_requests(spec["n"], salt=0)
    idx = list(range(0, spec["n"], spec["every"]))
    a = time.perf_counter()
    for i in idx:
        stream1d.solve(subs[i])
    t = time.perf_counter() - a
    out = dict(value=len(idx) / t, unit="subproblems/s", cores=1, kind="oracle",
               sample=(f"FP64 numpy oracle, 1 thread: Green's rows and Householder QR of requests "
                       f"{idx} of the {spec['n']}-request stream ({t:.1f} s)"))
    print("CPUJSON " + json.dumps(out))


PAPER_TSVD = dict(tsvd_tol=-1e-2, kz_disk=2.2)   # relative sigma, disk |k| <= 2.2 omega_max / c0


def cpu_child_paper(spec):
    """Oracle sample of the paper-shaped workload with the paper's solver: truncated-SVD solves
    (vertical-wavenumber disk) of sampled midpoint indices, transform and table amortised."""
    import numpy as np
    import synth
    from oracle import edt2d
    wl = synth.preset("paper_2d")
    rng = synth.rng_for(1, salt=78)
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx))
    t0 = time.perf_counter()
    D2 = edt2d.data_transform(D)
    g = edt2d.green_table(wl)
    t1 = time.perf_counter()
    per = []
    for m in spec["ms"]:
        a = time.perf_counter()
        edt2d.solve_wavenumber(wl, D2, m, g, solver="tsvd", tsvd_tol=PAPER_TSVD["tsvd_tol"],
                               kz_disk=PAPER_TSVD["kz_disk"])
        per.append(time.perf_counter() - a)
    nsolve = wl.nx // 2 + 1
    t_sys = statistics.mean(per) + (t1 - t0) / nsolve
    out = dict(value=(wl.nx / nsolve) / t_sys, unit="subproblems/s", cores=1, kind="oracle",
               sample=(f"FP64 numpy oracle, 1 thread: truncated-SVD solves with the k_z disk of midpoint "
                       f"indices {list(spec['ms'])} (mean {statistics.mean(per) * 1e3:.1f} ms), data transform "
                       f"and Green's table ({t1 - t0:.2f} s) amortised over {nsolve} systems"))
    print("CPUJSON " + json.dumps(out))


def cpu_child(spec_path):
    """Runs in a subprocess with single-threaded BLAS: time the oracle on a sample."""
    import numpy as np
    import synth
    from oracle import edt2d
    spec = json.load(open(spec_path))
    if spec.get("workload") == "batched_3d":
        cpu_child_window(spec)
        return
    if spec.get("workload") == "differentiation_2d":
        cpu_child_grad(spec)
        return
    if spec.get("workload") == "streaming":
        cpu_child_stream(spec)
        return
    if spec.get("workload") == "paper_2d_tsvd":
        cpu_child_paper(spec)
        return
    wl = synth.preset(spec["workload"])
    rng = synth.rng_for(1, salt=77)
    D = synth.random_data(rng, (len(wl.freq_hz), wl.nx, wl.nx), np.complex64).astype(np.complex128)
    t0 = time.perf_counter()
    D2 = edt2d.data_transform(D)
    t1 = time.perf_counter()
    g = edt2d.green_table(wl)
    t2 = time.perf_counter()
    ms = spec["ms"]
    per = []
    for m in ms:
        a = time.perf_counter()
        edt2d.solve_wavenumber(wl, D2, m, g)
        per.append(time.perf_counter() - a)
    nsolve = wl.nx // 2 + 1
    # per-subproblem cost: one split system solves the pair +-k_m, i.e. nx/nsolve subproblems;
    # the transform and the Green's table are amortised over the nsolve systems
    t_sys = statistics.mean(per) + ((t1 - t0) + (t2 - t1)) / nsolve
    rate = (wl.nx / nsolve) / t_sys
    out = dict(value=rate, unit="subproblems/s", cores=1, kind="oracle",
               sample=(f"FP64 numpy oracle, 1 thread: full data transform ({t1 - t0:.1f} s) and "
                       f"Green's table ({t2 - t1:.1f} s) amortised over {nsolve} split systems, "
                       f"plus QR solves of midpoint indices {list(ms)} "
                       f"(mean {statistics.mean(per):.2f} s each); random c64 data of the "
                       f"workload's shape"),
               per_solve_s=per, transform_s=t1 - t0, green_s=t2 - t1)
    print("CPUJSON " + json.dumps(out))


def run_cpu_baseline(ms, spec=None):
    spec = spec or dict(workload=WORKLOAD, ms=list(ms))
    with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as f:
        json.dump(spec, f)
        path = f.name
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-child", path],
                       capture_output=True, text=True, env=env, cwd=ROOT)
    os.unlink(path)
    for line in r.stdout.splitlines():
        if line.startswith("CPUJSON "):
            return json.loads(line[8:])
    raise RuntimeError("cpu baseline failed:\n" + r.stdout[-2000:] + r.stderr[-2000:])


def run_cpu_baseline_all_cores(max_cores=16):
    """The oracle on every host core at once: one single-threaded child per core, each with its
    own data transform, Green's table and one QR solve of a different midpoint index, started
    together; the job's rate is the sum of the children's rates (each measured while all
    children compete for the memory system)."""
    try:
        ncores = len(os.sched_getaffinity(0))
    except AttributeError:
        ncores = os.cpu_count() or 1
    ncores = max(1, min(int(max_cores), ncores))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs, paths = [], []
    t0 = time.perf_counter()
    for c in range(ncores):
        spec = dict(workload=WORKLOAD, ms=[(1 + 17 * c) % 257])
        with tempfile.NamedTemporaryFile("w", suffix=".json", delete=False) as f:
            json.dump(spec, f)
            paths.append(f.name)
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-child", paths[-1]],
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                                      env=env, cwd=ROOT))
    rates = []
    for pr in procs:
        out, err = pr.communicate()
        for line in out.splitlines():
            if line.startswith("CPUJSON "):
                rates.append(json.loads(line[8:])["value"])
    wall = time.perf_counter() - t0
    for pth in paths:
        os.unlink(pth)
    if len(rates) != ncores:
        raise RuntimeError(f"{ncores - len(rates)} of {ncores} oracle children failed")
    return dict(value=sum(rates), unit="subproblems/s", cores=ncores, kind="oracle",
                sample=(f"{ncores} single-threaded FP64 numpy oracle processes at once (wall {wall:.1f} s), "
                        f"each: the full data transform and Green's table amortised over the 257 split "
                        f"systems plus one QR solve of its own midpoint index; the sum of their rates"))


# ------------------------------------------------------------------ clocks
class Clocks:
    def __init__(self, gpu_index):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    ms_per_step = 1
    nsolve = 257
    sample = []
    # step i solves one midpoint index; K + W steps stay within a few minutes at 1 core
    for i in range(args.warmup + args.steps):
        sample.append((1 + 37 * i) % nsolve)
    base = run_cpu_baseline(sample)
    per = base["per_solve_s"][args.warmup:]
    amort = (base["transform_s"] + base["green_s"]) / nsolve
    step_t = [p + amort for p in per]
    total = sum(step_t)
    import synth
    wl = synth.preset(WORKLOAD)
    value = (wl.nx / nsolve) * len(step_t) / total
    line = dict(impl="reference", metric="subproblems_per_sec", value=value, unit="subproblems/s",
                n_gpus=args.gpus, steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * total / len(step_t), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=workload_summary(wl), per_step=f"{ms_per_step} split system"),
                cpu_baseline=dict(kind="oracle", cores=1, value=value, unit="subproblems/s",
                                  sample=base["sample"]),
                e2e=dict(value=value, unit="subproblems/s", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0))
    print(json.dumps(line))


# ------------------------------------------------------------------ our arm
def main():
    args = parse()
    if args.cpu_child:
        cpu_child(args.cpu_child)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batched_3d":
        main_window(args, world, rank, local)
        return
    if args.workload == "streaming":
        main_stream(args, world, rank, local)
        return
    if args.workload == "paper_2d_tsvd":
        main_paper(args, world, rank, local)
        return
    if args.workload == "differentiation_2d":
        main_grad(args, world, rank, local)
        return
    if args.workload == "fma_peak":
        main_fma_peak(args, world, rank, local)
        return

    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED, EDT_FP64

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.preset(WORKLOAD)
    if args.freq_stride > 1:
        wl.freq_hz = wl.freq_hz[::args.freq_stride]
    rng = synth.rng_for(1, salt=line_salt(rank))     # each rank: its own survey line
    V = synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0,
                                        wl.layer_top, wl.layer_vel, corr=40.0, rms=0.03)
    fp64 = Solver(Config.from_workload(wl, precision=EDT_FP64), device=dev)
    D = fp64.forward(torch.from_numpy(V).to(dev), out_dtype=torch.complex64)
    # complex Gaussian noise at 20 dB SNR per frequency (seeded, generated on the device)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_BASE + 1 + 1000 * rank)
    p_sig = (D.abs() ** 2).mean(dim=(1, 2), keepdim=True)
    sd = torch.sqrt(p_sig / 10 ** (wl.snr_db / 10) / 2)
    D = D + torch.complex(torch.randn(D.shape, device=dev, generator=gen),
                          torch.randn(D.shape, device=dev, generator=gen)) * sd
    D = D.contiguous()
    torch.cuda.synchronize()

    mixed = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=args.passes,
                                        refine=args.refine, chol_df=args.chol_df), device=dev)
    Vout = torch.empty((wl.nx, wl.nz), device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream(dev)
    tuning = None
    if not args.no_autotune:
        tuning = mixed.autotune(D, out=Vout, reps=3)     # launch shapes (same arithmetic)
    # independent lines in flight: one context (workspace, streams, tuned shapes) and one CUDA
    # stream each; consecutive steps alternate between them, so one line's tensor-core Gram
    # overlaps another's FP32-bound Cholesky and L1-bound refinement
    lines = max(1, args.lines_in_flight)
    ctxs, outs = [mixed], [Vout]
    for _ in range(lines - 1):
        c2 = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=args.passes,
                                         refine=args.refine, chol_df=args.chol_df), device=dev)
        c2.set_tuning(**{k: v for k, v in mixed.tuning().items() if k != "invert_ms"})
        ctxs.append(c2)
        outs.append(torch.empty_like(Vout))
    lstreams = [torch.cuda.Stream(device=dev) for _ in range(lines)]

    def run_lines(k_steps):
        for k in range(k_steps):
            i = k % lines
            with torch.cuda.stream(lstreams[i]):
                ctxs[i].invert(D, out=outs[i])

    for _ in range(max(3, args.warmup)):
        run_lines(lines)
    torch.cuda.synchronize()
    for c in ctxs:
        st = c.stats()
        if st.n_notpd or st.n_nonfinite:
            raise RuntimeError(f"mixed path: {st.n_notpd} not PD, {st.n_nonfinite} non-finite")

    # ---- device-resident timed region ----------------------------------------------
    clocks = Clocks(local)
    time.sleep(0.3)                      # let the sampler start before the timed region
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(lstreams[0])
    for ls in lstreams[1:]:
        ls.wait_event(e0)
    run_lines(args.steps)
    for ls in lstreams[1:]:
        ej = torch.cuda.Event()
        ej.record(ls)
        lstreams[0].wait_event(ej)
    e1.record(lstreams[0])
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    # stage breakdown: the same calls with per-stage CUDA events (begin and end of each stage
    # on the stream it runs on), right after the timed region
    mixed.set_profiling(True)
    for _ in range(min(args.steps, 50)):
        mixed.invert(D, out=Vout)
    stages, ncalls = mixed.read_profile()
    mixed.set_profiling(False)
    ms_total = max_over_ranks(ms_total, world)
    ms_step = ms_total / args.steps
    sub_per_step = wl.nx                             # one subproblem per midpoint wavenumber
    value = job_throughput(world, sub_per_step, args.steps, ms_total)

    # ---- end to end through the host-buffer entry point ----------------------------
    # every step copies its 268 MB of data in and V out inside the timed region; with the
    # host pipeline on, a context's next input copy overlaps its current stages (the serial
    # figure, one context with every copy in line with the stages, is reported beside it).
    # The same lines in flight as the device-resident region, each context on its own stream.
    Dh = D.cpu().pin_memory()
    Vhs = [torch.empty((wl.nx, wl.nz), dtype=torch.float32).pin_memory() for _ in range(lines)]

    def e2e_ms(pipe, nl):
        for c in ctxs[:nl]:
            c.set_host_pipeline(pipe)
        for i in range(nl):
            with torch.cuda.stream(lstreams[i]):
                for _ in range(2):
                    ctxs[i].invert_host(Dh, Vhs[i])
        torch.cuda.synchronize()
        barrier()
        h0 = torch.cuda.Event(enable_timing=True)
        h1 = torch.cuda.Event(enable_timing=True)
        h0.record(lstreams[0])
        for ls in lstreams[1:nl]:
            ls.wait_event(h0)
        for k in range(args.steps):
            i = k % nl
            with torch.cuda.stream(lstreams[i]):
                ctxs[i].invert_host(Dh, Vhs[i])
        for ls in lstreams[1:nl]:
            ej = torch.cuda.Event()
            ej.record(ls)
            lstreams[0].wait_event(ej)
        h1.record(lstreams[0])
        torch.cuda.synchronize()
        barrier()
        for c in ctxs[:nl]:
            c.set_host_pipeline(False)
        return max_over_ranks(h0.elapsed_time(h1), world)

    ms_e2e_serial = e2e_ms(False, 1)
    ms_e2e = e2e_ms(True, lines)
    e2e_value = job_throughput(world, sub_per_step, args.steps, ms_e2e)
    del ctxs[1:], outs[1:]

    # ---- accuracy vs the FP64 GPU path, and the FP64 path's own throughput --------------
    acc = {}
    if not args.no_fp64:
        V64 = torch.empty((wl.nx, wl.nz), device=dev, dtype=torch.float64)
        fp64.invert(D, out=V64)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        nf64 = 3
        f0.record(stream)
        for _ in range(nf64):
            fp64.invert(D, out=V64)
        f1.record(stream)
        torch.cuda.synchronize()
        ms64 = f0.elapsed_time(f1) / nf64
        Vm = Vout.double()
        rel = float(torch.linalg.norm(Vm - V64) / torch.linalg.norm(V64))
        vh_m = mixed.vhat(); vh_d = fp64.vhat()
        relh = float(torch.linalg.norm(vh_m - vh_d) / torch.linalg.norm(vh_d))
        acc = dict(rel_l2_V_vs_fp64_gpu=rel, rel_l2_vhat_vs_fp64_gpu=relh,
                   fp64_gpu_ms_per_step=ms64,
                   fp64_gpu_subproblems_per_sec=sub_per_step / (ms64 / 1e3),
                   speedup_vs_fp64_gpu=(ms64 / ms_step))

    # ---- variants: the native FP64 Cholesky and the double-float one with its trailing updates
    # on the tensor cores (library options) beside the default double-float one ----
    variants = {}
    if args.chol_df not in (2, 3):
        for vname, vcd, vdesc in (
                ("chol_fp64", 2, "native FP64 Cholesky factorisation and solves (chol_df = 2)"),
                ("chol_tensor_slices", 3, "double-float Cholesky with the trailing updates on the tensor "
                                          "cores, eight 7-bit BF16 slices per panel value (chol_df = 3)")):
            dfs = Solver(Config.from_workload(wl, precision=EDT_MIXED, passes=args.passes,
                                              refine=args.refine, chol_df=vcd), device=dev)
            # the same launch shapes, so that only the factorisation differs (the shapes set FP32
            # summation orders in the transform and the residual)
            dfs.set_tuning(**{k: v for k, v in mixed.tuning().items() if k != "invert_ms"})
            Vdf = torch.empty_like(Vout)
            for _ in range(3):
                dfs.invert(D, out=Vdf)
            torch.cuda.synchronize()
            barrier()
            v0 = torch.cuda.Event(enable_timing=True)
            v1 = torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            for _ in range(args.steps):
                dfs.invert(D, out=Vdf)
            v1.record(stream)
            torch.cuda.synchronize()
            ms_df = max_over_ranks(v0.elapsed_time(v1), world)
            Ldf = torch.tril(mixed.factor())
            L64 = torch.tril(dfs.factor())
            fac_err = float(torch.max(torch.linalg.norm(Ldf - L64, dim=(1, 2))
                                      / torch.clamp(torch.linalg.norm(L64, dim=(1, 2)), min=1e-300)))
            variants[vname] = dict(
                description=vdesc,
                factor_rel_diff_max=fac_err,
                value=job_throughput(world, sub_per_step, args.steps, ms_df), unit="subproblems/s",
                ms_per_step=ms_df / args.steps,
                rel_l2_V_vs_default=float(torch.linalg.norm(Vdf.double() - Vout.double())
                                          / torch.linalg.norm(Vout.double())),
                rel_l2_vhat_vs_default=float(torch.linalg.norm(dfs.vhat() - mixed.vhat())
                                             / torch.linalg.norm(mixed.vhat())))
            del dfs

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (tensor-core Gram) --------------------------
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    nzp = (wl.nz + 31) // 32 * 32
    ncols = (nzp + 16) + (nzp - 128 + 16 if nzp > 128 else 0)
    padded_rows = st.gram_rows_padded
    issued = args.passes * 2.0 * (2 * padded_rows) * 128 * ncols          # MMA flops / launch
    useful = 2.0 * (2 * st.rows_solved) * wl.nz * (wl.nz + 2)             # full-square G + b
    gram_ms = stages.get("gram", 0.0) / max(ncalls, 1)
    # The Gram runs about 1 ms inside a 4-5 ms step at full clock, so the burst peak
    # applies; FP16 and BF16 share the dense tensor rate (nominal ratio 1).
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = issued / (gram_ms / 1e3) / 1e12 if gram_ms > 0 else None
    useful_tf = useful / (gram_ms / 1e3) / 1e12 if gram_ms > 0 else None
    roof = dict(bound="tensor", kernel="gram_tc_kernel", achieved=achieved, peak=peak,
                unit="TFLOP/s", frac=(achieved / peak) if achieved else None,
                traffic=_traffic_from_profile(),
                peak_source=("MEASURED_PEAKS.json bf16_tflops (burst, of measured; FP16 operands run "
                             "at the BF16 rate)" if "bf16_tflops" in peaks else "fallback 1.9 PFLOP/s burst"),
                flops_per_launch=issued, useful_flops_per_launch=useful,
                useful_tflops=useful_tf, useful_frac=(useful_tf / peak) if useful_tf else None,
                gram_ms=gram_ms)
    stage_ms = {k: v / max(ncalls, 1) for k, v in stages.items()}
    chol_roof = cholesky_roofline(wl.nz, wl.nx // 2 + 1, stage_ms.get("cholesky", 0.0),  # split systems
                                  chol_fp64=args.chol_df == 2)

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_cpu_baseline(CPU_SAMPLE_M)
            cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}
        except Exception as ex:  # the GPU number stands; report why the baseline is missing
            cpu = dict(value=None, unit="subproblems/s", cores=0, kind="oracle", sample=str(ex)[:300])
        try:
            cpu["all_cores"] = run_cpu_baseline_all_cores()
        except Exception as ex:
            cpu["all_cores"] = dict(value=None, unit="subproblems/s", cores=0, kind="oracle",
                                    sample=str(ex)[:300])

    line = dict(
        metric="subproblems_per_sec", value=value, unit="subproblems/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms_step, higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f16x3+f32acc+f64", data="synthetic",
        config=dict(workload=workload_summary(wl), l2=f"inputs larger than L2 ({D.numel() * D.element_size() / 1e6:.0f} MB data per step)",
                    passes=args.passes, refine=args.refine, chol_df=args.chol_df, alpha=wl.alpha,
                    rows_total=int(st.rows_total), rows_solved=int(st.rows_solved),
                    parallelism=f"replicas x{world} (independent lines)", lines_in_flight=lines,
                    launch_shapes=(tuning or mixed.tuning()), autotuned=tuning is not None),
        model_pts_per_sec=world * wl.nx * wl.nz * args.steps / (ms_total / 1e3),
        e2e=dict(value=e2e_value, unit="subproblems/s",
                 h2d_bytes_per_step=int(Dh.numel() * Dh.element_size()),
                 d2h_bytes_per_step=int(Vhs[0].numel() * Vhs[0].element_size()),
                 pipelined=True, lines_in_flight=lines, ms_per_step=ms_e2e / args.steps,
                 serial_value=job_throughput(world, sub_per_step, args.steps, ms_e2e_serial),
                 serial_ms_per_step=ms_e2e_serial / args.steps),
        gpu_launches=int(st.launches_per_invert) * args.steps,
        roofline=roof, cholesky_roofline=chol_roof, stage_ms=stage_ms, accuracy=acc,
        variants=variants, clocks=clk, cpu_baseline=cpu)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main_window(args, world, rank, local):
    """The finite-aperture 3D workload: 128 x 128 midpoints (12.5 m), 16 x 16 half-offsets,
    64 frequencies 4-50 Hz, 200 depths of 10 m, 20 random layers, alpha = 1e-2, seeded
    complex64 random data of the workload's shape (any data define a valid least-squares
    problem); 16 384 subproblems (midpoint wavenumbers) per inversion, 8 194 pair systems."""
    import torch
    import torch.distributed as dist
    import synth
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import Config, Solver
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.preset3d("batched_3d")
    nf = len(wl.freq_hz)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_BASE + 2 + 1000 * line_salt(rank))
    shape = (nf, wl.ny, wl.nx, wl.wy, wl.wx)
    D = torch.complex(torch.randn(shape, device=dev, generator=gen),
                      torch.randn(shape, device=dev, generator=gen)).contiguous()
    s = Solver(Config.from_workload(wl, passes=args.passes, refine=args.refine,
                                    chol_df=args.chol_df), device=dev)
    Vout = torch.empty((wl.ny, wl.nx, wl.nz), device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream(dev)
    tuning = None
    if not args.no_autotune:
        tuning = s.autotune(D, out=Vout, reps=1)
    for _ in range(max(3, args.warmup)):
        s.invert(D, out=Vout)
    torch.cuda.synchronize()
    st = s.stats()
    if st.n_notpd or st.n_nonfinite:
        raise RuntimeError(f"window path: {st.n_notpd} not PD, {st.n_nonfinite} non-finite")
    clocks = Clocks(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.invert(D, out=Vout)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    s.set_profiling(True)
    for _ in range(min(args.steps, 3)):
        s.invert(D, out=Vout)
    stages, ncalls = s.read_profile()
    s.set_profiling(False)
    ms_total = max_over_ranks(e0.elapsed_time(e1), world)
    sub_per_step = wl.nx * wl.ny
    value = job_throughput(world, sub_per_step, args.steps, ms_total)
    # end to end through the host-buffer entry point
    Dh = D.cpu().pin_memory()
    Vh = torch.empty((wl.ny, wl.nx, wl.nz), dtype=torch.float32).pin_memory()
    s.set_host_pipeline(True)            # step k+1's input copy overlaps step k
    s.invert_host(Dh, Vh)
    torch.cuda.synchronize()
    barrier()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        s.invert_host(Dh, Vh)
    h1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(h0.elapsed_time(h1), world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    stage_ms = {k: v / max(ncalls, 1) for k, v in stages.items()}
    nzp = (wl.nz + 31) // 32 * 32
    ncols = (nzp + 16) + (nzp - 128 + 16 if nzp > 128 else 0)
    issued = args.passes * 2.0 * (2 * st.gram_rows_padded) * 128 * ncols
    gram_ms = stage_ms.get("gram", 0.0)
    peak = peaks.get("bf16_tflops_sustained", 1700.0)
    achieved = issued / (gram_ms / 1e3) / 1e12 if gram_ms > 0 else None
    roof = dict(bound="tensor", kernel="gram_tc_kernel", achieved=achieved, peak=peak,
                unit="TFLOP/s", frac=(achieved / peak) if achieved else None, traffic=None,
                peak_source="MEASURED_PEAKS.json bf16_tflops_sustained (of measured)",
                flops_per_launch=issued, gram_ms=gram_ms,
                useful_flops_per_launch=2.0 * (2 * st.rows_solved) * wl.nz * (wl.nz + 2))
    # kernel-row assembly: its irreducible output is the row table (every kept row's nz FP32
    # complex values, written once); the window products are an on-device intermediate whose
    # measured traffic the launch list reports.  The stage is bound by its FFTs (issue and
    # latency), not by HBM, so the table rate below is a lower bound of its memory use.
    k3_bytes = st.rows_solved * wl.nz * 8
    k3_ms = stage_ms.get("kernel_rows", 0.0)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_cpu_baseline(None, dict(workload="batched_3d", pair=4100, freqs=[10, 40]))
        except Exception as ex:
            cpu = dict(value=None, unit="subproblems/s", cores=0, kind="oracle", sample=str(ex)[:300])
    line = dict(
        metric="subproblems_per_sec", value=value, unit="subproblems/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms_total / args.steps,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="bf16x3+f32acc+f64",
        data="synthetic (seeded complex64 random data)",
        config=dict(workload=("batched_3d: 128x128 midpoints dx=dy 12.5 m, 16x16 half-offsets "
                              "(offsets every 25 m), 64 freqs 4-50 Hz, nz 200 dz 10 m, 20 layers"),
                    l2="inputs larger than L2 (2.1 GB data per step)", passes=args.passes,
                    refine=args.refine, alpha=wl.alpha, pairs=int(st.n_sub),
                    rows_total=int(st.rows_total), parallelism=f"replicas x{world}",
                    launch_shapes=(tuning or s.tuning()), autotuned=tuning is not None),
        model_pts_per_sec=world * wl.nx * wl.ny * wl.nz * args.steps / (ms_total / 1e3),
        e2e=dict(value=job_throughput(world, sub_per_step, args.steps, ms_e2e), unit="subproblems/s",
                 h2d_bytes_per_step=int(Dh.numel() * Dh.element_size()),
                 d2h_bytes_per_step=int(Vh.numel() * Vh.element_size())),
        gpu_launches=int(st.launches_per_invert) * args.steps,
        roofline=roof,
        kernel_rows=dict(bound="issue/latency (2D FFTs of the window products)", ms=k3_ms,
                         table_bytes=k3_bytes,
                         table_write_gbs=k3_bytes / (k3_ms / 1e3) / 1e9 if k3_ms > 0 else None,
                         hbm_peak_gbs=peaks.get("hbm_gbs")),
        stage_ms=stage_ms, clocks=clk, cpu_baseline=cpu)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main_grad(args, world, rank, local):
    """Misfit gradients on the production geometry (FP32): 512 x 512, 128 frequencies 3-60 Hz,
    256 depths of 8 m, 20 layers; data = Born data of a 3 % random field plus 20 dB noise,
    model = half that field.  One step = one evaluation of J = ||F V - D||^2, dJ/dV (adjoint
    Born) and dJ/dc for the 20 layer velocities (reverse-mode depth march)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import Config, Solver, EDT_MIXED
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    wl = synth.preset(WORKLOAD)
    wl.cutoff = 0.0
    rng = synth.rng_for(3, salt=line_salt(rank))
    Vt = synth.perturbation_random_field(rng, wl.nx, wl.dx, wl.nz, wl.dz, wl.z0, wl.layer_top,
                                         wl.layer_vel)
    s = Solver(Config.from_workload(wl, precision=EDT_MIXED), device=dev)
    D = s.forward(torch.from_numpy(Vt.astype(np.float32)).to(dev), out_dtype=torch.complex64)
    gen = torch.Generator(device=dev)
    gen.manual_seed(synth.SEED_BASE + 3 + 1000 * rank)
    p_sig = (D.abs() ** 2).mean(dim=(1, 2), keepdim=True)
    sd = torch.sqrt(p_sig / 10 ** (wl.snr_db / 10) / 2)
    D = (D + torch.complex(torch.randn(D.shape, device=dev, generator=gen),
                           torch.randn(D.shape, device=dev, generator=gen)) * sd).contiguous()
    V = torch.from_numpy((0.5 * Vt).astype(np.float32)).to(dev).contiguous()
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        s.misfit_grad(V, D)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, gV, gc = s.misfit_grad(V, D)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world)
    value = job_throughput(world, 1, args.steps, ms_total)
    # end to end: pinned host inputs in, J and both gradients back to pinned host memory
    Dh = D.cpu().pin_memory()
    Vh = V.cpu().pin_memory()
    gVh = torch.empty_like(Vh).pin_memory()
    gch = torch.empty((len(wl.layer_vel),), dtype=torch.float64).pin_memory()
    Jh = torch.empty((), dtype=torch.float64).pin_memory()
    Dd, Vd = torch.empty_like(D), torch.empty_like(V)
    torch.cuda.synchronize()
    barrier()
    h0 = torch.cuda.Event(enable_timing=True)
    h1 = torch.cuda.Event(enable_timing=True)
    h0.record(stream)
    for _ in range(args.steps):
        Dd.copy_(Dh, non_blocking=True)
        Vd.copy_(Vh, non_blocking=True)
        J, gV, gc = s.misfit_grad(Vd, Dd)
        Jh.copy_(J, non_blocking=True)
        gVh.copy_(gV, non_blocking=True)
        gch.copy_(gc, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(h0.elapsed_time(h1), world)
    # adjoint of the production inversion (cut on, as edt_invert runs it): dL/dD for a
    # loss of V, timed beside the inversion it differentiates
    inv = Solver(Config.from_workload(synth.preset(WORKLOAD), precision=EDT_MIXED), device=dev)
    Vout = torch.empty((wl.nx, wl.nz), device=dev, dtype=torch.float32)
    Vbar = torch.randn((wl.nx, wl.nz), device=dev, generator=gen, dtype=torch.float32)
    for _ in range(3):
        inv.invert(D, out=Vout)
        inv.invert_adjoint(Vbar, out_dtype=torch.complex64)
        inv.invert_vjp(Vbar, want_D=False)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a2 = torch.cuda.Event(enable_timing=True)
    a3 = torch.cuda.Event(enable_timing=True)
    a4 = torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(args.steps):
        inv.invert(D, out=Vout)
    a1.record(stream)
    for _ in range(args.steps):
        Dbar = inv.invert_adjoint(Vbar, out_dtype=torch.complex64)
    a2.record(stream)
    for _ in range(args.steps):
        _, gc_solve = inv.invert_vjp(Vbar, want_D=False)
    a3.record(stream)
    for _ in range(args.steps):
        Dbar, gc_solve = inv.invert_vjp(Vbar, out_dtype=torch.complex64)
    a4.record(stream)
    torch.cuda.synchronize()
    adj = dict(invert_ms=a0.elapsed_time(a1) / args.steps, invert_adjoint_ms=a1.elapsed_time(a2) / args.steps,
               invert_grad_c_ms=a2.elapsed_time(a3) / args.steps,
               invert_vjp_both_ms=a3.elapsed_time(a4) / args.steps,
               note="after edt_invert on the production inversion (cut on, one refinement step): "
                    "edt_invert_adjoint (dL/dD through the damped solve, c64 Dbar); edt_invert_vjp "
                    "with dL/dc only (rows, normal-matrix and damping derivatives, reverse depth "
                    "march) and with both outputs")
    del inv
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    nf, N, nz = len(wl.freq_hz), wl.nx, wl.nz
    # four contractions over (f, p, q, z): residual, adjoint Born, and the two legs of dJ/dg,
    # each a complex product (6 flops) and a complex multiply-add (8 flops) per term
    flops = 56.0 * nf * N * N * nz
    peak = 152 * 128 * 2 * 2.07 / 1e3        # FP32 FMA lanes x 2 flops x 2.07 GHz -> TFLOP/s
    achieved = flops / (ms_total / args.steps / 1e3) / 1e12
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_cpu_baseline(None, dict(workload="differentiation_2d", freq=127))
        except Exception as ex:
            cpu = dict(value=None, unit="gradients/s", cores=0, kind="oracle", sample=str(ex)[:300])
    line = dict(
        metric="misfit_gradients_per_sec", value=value, unit="gradients/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=ms_total / args.steps,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32+f64acc",
        data="synthetic (Born data of a seeded 3% random field + 20 dB noise; model = half the field)",
        config=dict(workload=(f"differentiation_2d: {N}x{N} dx {wl.dx} m, {nf} freqs "
                              f"{wl.freq_hz.min():g}-{wl.freq_hz.max():g} Hz, nz {nz} dz {wl.dz} m, "
                              f"{len(wl.layer_vel)} layers; J, dJ/dV, dJ/dc per step"),
                    l2="inputs larger than L2 (268 MB data)", parallelism=f"replicas x{world}"),
        model_pts_per_sec=world * N * nz * args.steps / (ms_total / 1e3),
        e2e=dict(value=job_throughput(world, 1, args.steps, ms_e2e), unit="gradients/s",
                 h2d_bytes_per_step=int(D.numel() * D.element_size() + V.numel() * V.element_size()),
                 d2h_bytes_per_step=int(gV.numel() * gV.element_size() + gc.numel() * 8 + 8)),
        gpu_launches=None,
        roofline=dict(bound="alu", kernel="grad_residual + grad_vhat + grad_gbar (whole call)",
                      achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                      traffic=None, peak_source="derived: 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz",
                      flops_per_launch=flops),
        J=float(J), solve_adjoint=adj, clocks=clk, cpu_baseline=cpu)
    line["gpu_launches"] = int(s.stats().launches_per_grad) * args.steps
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main_stream(args, world, rank, local):
    """Streaming batched solves: 4096 independent 1D subproblems (depth counts uniform 64-512,
    rows uniform 128-4096, random layered references of 5-30 layers, complex64 data) arriving
    in Poisson bursts of 32-512.  One step = the whole stream.

    value: subproblems / device time in which the batches' launches ran (the union of their
    intervals: consecutive batches overlap on the two arenas' streams; inputs resident, the
    host-device copies outside those intervals); e2e: the same stream submitted through
    edt_stream_submit from host arrays burst after burst with no pause, host wall time from the
    first submit to the last result; latency: the bursts submitted at Poisson arrival times at
    70 % of the saturated burst rate, completion (CUDA event) minus scheduled arrival."""
    import numpy as np
    import torch
    import torch.distributed as dist
    from synth import stream as ss
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import Stream
    from paper_0905_0238_gb300.edt import edt_stream_request_bytes
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    n_total = 4096
    subs = ss.stream_requests(n_total, salt=rank)
    sizes, _ = ss.burst_schedule(n_total, rate_hz=1.0, salt=rank)
    cuts = np.concatenate([[0], np.cumsum(sizes)])
    bursts = [subs[cuts[i]:cuts[i + 1]] for i in range(len(sizes))]
    rb = np.array([edt_stream_request_bytes(x) for x in subs], dtype=np.int64)
    burst_bytes = max(int(rb[cuts[i]:cuts[i + 1]].sum()) for i in range(len(sizes)))
    s = Stream(max_batch=512, workspace_bytes=2 * (burst_bytes + (64 << 20)), device=dev)

    def run_all():
        t0 = time.perf_counter()
        tickets = [s.submit(bb) for bb in bursts]
        out = [s.wait(t) for t in tickets]
        return time.perf_counter() - t0, out

    for _ in range(max(3, args.warmup)):
        run_all()
    st0 = s.stats()
    clocks = Clocks(local)
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    s.epoch()
    wall = []
    for _ in range(args.steps):
        t, out = run_all()
        wall.append(t)
    barrier()
    clk = clocks.stop()
    st1 = s.stats()
    # device time: union of the intervals in which some batch's launches ran (the two arenas'
    # streams overlap consecutive batches); host-device copies outside those intervals
    dev_ms = max_over_ranks(st1["busy_ms"], world)
    sum_ms = st1["compute_ms"] - st0["compute_ms"]
    value = world * n_total * args.steps / (dev_ms / 1e3)
    wall_s = max_over_ranks(sum(wall), world)
    e2e = world * n_total * args.steps / wall_s
    bad = sum(int(np.count_nonzero(o[1])) for o in out)
    # per-launch split of one pass (CUDA events between the launches)
    s.set_profiling(True)
    run_all()
    prof, nb = s.read_profile()
    s.set_profiling(False)
    # open-loop latency at 70 % of the saturated burst rate
    rate = 0.7 * len(bursts) / (sum(wall) / len(wall))
    _, arrive = ss.burst_schedule(n_total, rate_hz=rate, salt=rank)
    s.epoch()
    t_epoch = time.perf_counter()
    tickets = []
    for bb, ta in zip(bursts, arrive):
        now = time.perf_counter() - t_epoch
        if ta > now:
            time.sleep(ta - now)
        tickets.append(s.submit(bb))
    lat = []
    for t, ta, bb in zip(tickets, arrive, bursts):
        _, _, done_ms = s.wait(t)
        lat += [done_ms - 1e3 * ta] * len(bb)
    lat = np.array(lat)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    # algorithmic work of one pass
    nz = np.array([x.nz for x in subs], dtype=np.float64)
    nr = np.array([x.nrow for x in subs], dtype=np.float64)
    chol_flops = float(np.sum(nz ** 3 / 3 + 4 * nz ** 2))
    gram_flops = float(np.sum(2 * (2 * nr) * nz * (nz + 2)))
    chol_ms = prof.get("chol", 0.0)
    gram_ms = prof.get("st_gram", 0.0)
    kern = max(prof, key=prof.get) if prof else None
    # the blocked factorisation and its solves run in double-float on the FP32 pipes: the
    # FP64-equivalent rate beside the measured FP64 multiply-add rate (what a native FP64
    # factorisation is bounded by) and the measured FP32 rate (the pipe it uses)
    from paper_0905_0238_gb300 import edt as _edt
    fp64_peak, fp32_peak = _edt.edt_measure_fma_rates()
    roof = dict(bound="alu", kernel="chol (double-float blocked Cholesky + solves, all requests of a pass)",
                achieved=chol_flops / (chol_ms / 1e3) / 1e12 if chol_ms else None, peak=fp64_peak,
                unit="TFLOP/s (FP64-equivalent)", traffic=None,
                peak_source="edt_measure_fma_rates: FP64 multiply-add rate measured in this run",
                fp32_peak=fp32_peak, flops_per_pass=chol_flops)
    roof["frac"] = roof["achieved"] / fp64_peak if roof["achieved"] and fp64_peak else None
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16 = peaks.get("bf16_tflops_sustained") or 1686.2
    gram_issued = 0.0
    for x in subs:
        nzt = -(-x.nz // 128)
        kst = -(-x.nrow // 32)
        for ti in range(nzt):
            for tj in range(ti, nzt):
                ncol = 144 if tj == nzt - 1 else 128
                gram_issued += 3 * 2 * 128 * ncol * 64 * kst
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_cpu_baseline(None, dict(workload="streaming", n=n_total, every=512))
        except Exception as ex:
            cpu = dict(value=None, unit="subproblems/s", cores=0, kind="oracle", sample=str(ex)[:300])
    h2d = st1["bytes_in"] - st0["bytes_in"]
    d2h = st1["bytes_out"] - st0["bytes_out"]
    line = dict(
        metric="subproblems_per_sec", value=value, unit="subproblems/s", n_gpus=world,
        steps=args.steps, warmup=args.warmup, ms_per_step=dev_ms / args.steps,
        higher_is_better=True, scaling="weak", vs_baseline=None, dtype="bf16x3+f32+f64",
        data="synthetic (seeded requests: layered references, band rows, complex Gaussian data)",
        config=dict(workload=(f"streaming: {n_total} 1D subproblems, nz U(64,512), rows U(128,4096), "
                              f"5-30 layers, {len(bursts)} Poisson bursts of 32-512; one step = the "
                              f"whole stream"),
                    l2="inputs larger than L2 (each burst's row tables, several GB)",
                    parallelism=f"replicas x{world}", batches_per_pass=nb,
                    launch_ms_summed_over_batches=sum_ms / args.steps,
                    workspace_gb=round(2 * (burst_bytes + (64 << 20)) / 1e9, 2)),
        e2e=dict(value=e2e, unit="subproblems/s", h2d_bytes_per_step=int(h2d // args.steps),
                 d2h_bytes_per_step=int(d2h // args.steps),
                 note="saturated: bursts submitted back to back from host arrays, host wall time"),
        latency_ms=dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                        max=float(lat.max()), offered_bursts_per_s=rate,
                        note="open loop, Poisson burst arrivals at 70 % of the saturated burst rate; "
                             "completion (CUDA event after the result copy) minus arrival"),
        kernels_ms_per_pass={k: v for k, v in prof.items()},
        gram=dict(issued_tflop_per_pass=gram_issued / 1e12, useful_tflop_per_pass=gram_flops / 1e12,
                  achieved_tflops=gram_issued / (gram_ms / 1e3) / 1e12 if gram_ms else None,
                  peak_tflops=bf16, frac=(gram_issued / (gram_ms / 1e3) / 1e12 / bf16) if gram_ms else None),
        dominant_kernel=kern, nonzero_status=bad,
        gpu_launches=int(st1["launches"] - st0["launches"]),
        roofline=roof, clocks=clk, cpu_baseline=cpu)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def main_paper(args, world, rank, local):
    """The paper's own solver on its acquisition shape: a 256-point line (m, h every 50 m), 10
    frequencies 1-10 Hz, 65 depths 800-4000 m every 50 m, two-layer 1500/4000 m/s reference;
    truncated SVD (relative tolerance) with the vertical-wavenumber disk |k| <= 2.2 omega_max /
    c0, FP64 path.  Data: the library's FP64 Born data of three blobs plus the paper's noise
    (5 % of the largest |D| per frequency, uniform phase)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import synth
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import Config, Solver, EDT_FP64
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    wl = synth.preset("paper_2d")
    V0 = synth.perturbation_blobs(synth.rng_for(2, salt=line_salt(rank)), wl.nx, wl.dx, wl.nz, wl.dz, wl.z0,
                                  wl.layer_top, wl.layer_vel)
    s = Solver(Config.from_workload(wl, precision=EDT_FP64, solver=1, **PAPER_TSVD), device=dev)
    D = s.forward(torch.from_numpy(V0).to(dev))
    Dn = D.cpu().numpy()
    Dn = Dn + synth.noise_paper(synth.rng_for(2, salt=7 + rank), Dn)
    D = torch.from_numpy(np.ascontiguousarray(Dn)).to(dev)
    out = torch.empty((wl.nx, wl.nz), device=dev, dtype=torch.float64)
    stream = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        s.invert(D, out=out)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        s.invert(D, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms_total = max_over_ranks(e0.elapsed_time(e1), world)
    value = job_throughput(world, wl.nx, args.steps, ms_total)
    s.set_profiling(True)
    s.invert(D, out=out)
    prof = s.read_profile()
    s.set_profiling(False)
    # end to end through the host-buffer entry point
    Dh = torch.from_numpy(Dn).pin_memory()
    Vh = torch.empty((wl.nx, wl.nz), dtype=torch.float64).pin_memory()
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(args.steps):
        s.invert_host(Dh, Vh)
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks((time.perf_counter() - h0) * 1e3, world)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    stage = prof[0] if isinstance(prof, tuple) else prof
    solve_ms = None
    try:
        solve_ms = dict(stage).get("cholesky")
    except Exception:
        pass
    # Jacobi work model: per sweep (p - 1) rounds x p/2 pairs x 3 p (2 columns of A and W, 2 rows
    # of A) rotations of 6 flops; the converged sweep count is data dependent (5-6 measured on the
    # CPU model of the same iteration), 6 assumed
    p, nsub = wl.nz, wl.nx // 2 + 1
    jac_flops = 6.0 * nsub * (p - 1) * (p / 2) * 3 * p * 6
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        try:
            cpu = run_cpu_baseline(None, dict(workload="paper_2d_tsvd", ms=[1, 32, 64, 96]))
        except Exception as ex:
            cpu = dict(value=None, unit="subproblems/s", cores=0, kind="oracle", sample=str(ex)[:300])
    line = dict(
        metric="subproblems_per_sec", value=value, unit="subproblems/s", n_gpus=world, steps=args.steps,
        warmup=args.warmup, ms_per_step=ms_total / args.steps, higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64", data="synthetic (FP64 Born data of three blobs + the paper's 5 % noise)",
        config=dict(workload=(f"paper_2d_tsvd: {wl.nx}-point line dx {wl.dx} m, {len(wl.freq_hz)} freqs "
                              f"{wl.freq_hz.min():g}-{wl.freq_hz.max():g} Hz, nz {wl.nz} dz {wl.dz} m from "
                              f"{wl.z0 + wl.dz / 2:g} m, 2 layers; truncated SVD sigma = 1e-2 s_max, k_z disk 2.2"),
                    l2="inputs in L2 (5 MB of data)", parallelism=f"replicas x{world}"),
        e2e=dict(value=job_throughput(world, wl.nx, args.steps, ms_e2e), unit="subproblems/s",
                 h2d_bytes_per_step=int(Dn.nbytes), d2h_bytes_per_step=int(wl.nx * wl.nz * 8)),
        stage_ms=dict(stage) if not isinstance(stage, dict) else stage,
        gpu_launches=int(s.stats().launches_per_invert) * args.steps,
        roofline=dict(bound="alu", kernel="solver-variant stage (projection, Jacobi eigen-solver, back-projection)",
                      achieved=(jac_flops / (solve_ms / 1e3) / 1e12) if solve_ms else None, peak=1.25,
                      unit="TFLOP/s", traffic=None,
                      peak_source="nominal GB300 FP64 rate (1.25 TFLOP/s); flops from a 6-sweep Jacobi model",
                      flops_per_launch=jac_flops),
        clocks=clk, cpu_baseline=cpu)
    if line["roofline"]["achieved"]:
        line["roofline"]["frac"] = line["roofline"]["achieved"] / 1.25
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def cholesky_roofline(nz, nsub, chol_ms, chol_fp64=False):
    """Roofline of the damped Cholesky stage.  Algorithmic work per split system: nz^3/3 flops
    for the factorisation and 4 nz^2 for the two right-hand sides' substitutions.  The default
    factorisation runs in double-float on the FP32 pipes, so its FP64-equivalent rate is set
    beside the device's measured FP64 multiply-add rate (what a native FP64 factorisation is
    bounded by) and its measured FP32 rate (the pipe it actually uses)."""
    from paper_0905_0238_gb300 import edt as _edt
    fp64, fp32 = _edt.edt_measure_fma_rates()
    flops = nsub * (nz ** 3 / 3.0 + 4.0 * nz ** 2)
    ach = flops / (chol_ms * 1e-3) / 1e12 if chol_ms > 0 else None
    return dict(bound="fp64 pipe" if chol_fp64 else "fp32 pipe (double-float arithmetic)",
                kernel="chol_kernel" if chol_fp64 else "cdf_* (diag, panel, update, final)",
                achieved=ach, unit="TFLOP/s (FP64-equivalent)", peak=fp64,
                peak_source="edt_measure_fma_rates: FP64 multiply-add rate measured in this run",
                frac=(ach / fp64) if (ach and fp64) else None,
                fp32_peak=fp32, flops_per_call=flops, cholesky_ms=chol_ms)


def main_fma_peak(args, world, rank, local):
    """The device's FP64 and FP32 multiply-add rates (the denominators of the FP64 and
    double-float rooflines), measured by the library's probe."""
    import torch
    from paper_0905_0238_gb300 import build as libbuild
    libbuild.build()
    from paper_0905_0238_gb300 import edt as _edt
    torch.cuda.set_device(local)
    rates = [_edt.edt_measure_fma_rates() for _ in range(max(1, args.steps))]
    fp64 = max(r[0] for r in rates)
    fp32 = max(r[1] for r in rates)
    if rank == 0:
        print(json.dumps(dict(metric="fma_tflops", value=fp64, unit="TFLOP/s (FP64 multiply-add)",
                              n_gpus=1, steps=len(rates), warmup=0, higher_is_better=True,
                              dtype="f64", data="synthetic",
                              config=dict(workload="fma_peak: 8 independent multiply-add chains per "
                                                   "thread, 8 CTAs of 256 threads per SM"),
                              fp32_tflops=fp32, fp64_to_fp32=fp64 / fp32 if fp32 else None)))


def _kernel_source_hash(name):
    import hashlib
    path = os.path.join(ROOT, "paper_0905_0238_gb300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def _traffic_from_profile():
    """DRAM bytes per launch of the Gram kernel from the committed ncu summary, or None when
    the kernel source has changed since those counters were taken."""
    p = os.path.join(ROOT, "profiles", "gram_tc_production_2d.json")
    try:
        prof = json.load(open(p))
        if prof.get("source_sha16") != _kernel_source_hash("gram_tc.cu"):
            return None
        return prof.get("dram_bytes_per_launch")
    except Exception:
        return None


if __name__ == "__main__":
    main()
