#!/usr/bin/env python
"""Throughput benchmark of the spectral-element elastic hot path on GB300.

Workload: the three-layer jittered cube (vp 5000/3500/2000 m/s, side 4 km, interior vertex
jitter up to 10 % of the element size, 256 GLL intervals per side: 64^3 elements at
NGLL=5), Ricker point source at the centre, 256 surface receivers. One step = one explicit
Newmark time step of the whole hot path (Newmark update, matrix-free forces over all
colours with the coloured assembly, source, receivers). Metric: local GLL-point updates
per second = nspec * NGLL^3 * steps / time, summed over ranks (replicas, weak scaling).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--ngll 5] [--impl ours|reference]

Prints one JSON line. ``--impl reference`` times the FP64 CPU oracle (the only
reference this method has) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLL-pt updates/s & %HBM roofline; shots/s batched vs plain at 2e-5 rel L2"
UNIT = "local GLL-pt updates/s"
FALLBACK_HBM_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=1000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--ngll", type=int, default=5)
    p.add_argument("--elems", type=int, default=None,
                   help="elements per side (default: 256 GLL intervals per side); smaller cases for profiling")
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--stiffness-reps", type=int, default=40)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=20.0,
                   help="target time of the all-cores CPU baseline (steps of the full mesh, at most 20)")
    p.add_argument("--shots", type=int, default=32, help="batched-shot measurement (0 = skip)")
    p.add_argument("--shot-steps", type=int, default=100)
    p.add_argument("--no-sweep", action="store_true", help="skip the NGLL 3/5/7/9 (h,p) sweep")
    p.add_argument("--adjoint-steps", type=int, default=800, help="misfit-gradient measurement (0 = skip)")
    p.add_argument("--surrogate-runs", type=int, default=4096, help="surrogate training runs (0 = skip)")
    p.add_argument("--models", type=int, default=16, help="uneven-models group measurement (0 = skip)")
    p.add_argument("--no-iso", action="store_true", help="skip the (h,p) iso-accuracy study")
    p.add_argument("--no-ablation", action="store_true", help="skip the colouring/atomics assembly ablation")
    p.add_argument("--no-tiles", action="store_true", help="skip the element-tile autotuner measurement")
    p.add_argument("--surrogate-epochs", type=int, default=150)
    p.add_argument("--products-only", type=int, default=0, metavar="N",
                   help="only time the surrogate's products (both kernels) on N seeded inputs, print JSON, exit")
    return p.parse_args()


def algorithmic_bytes(nspec: int, ngll: int, nglob: int):
    """Bytes a perfect-reuse implementation moves (FP32 data, int32 ibool):
    per local point 52 B (ibool, 9 inverse-Jacobian terms, J, kappa, mu), per global node
    76 B per step (read u, v, a, 1/M; write u, v, a); the force kernel alone: 52 B per
    local point plus u read once and f written once per node (24 B)."""
    nloc = nspec * ngll ** 3
    return dict(step=52 * nloc + 76 * nglob, forces=52 * nloc + 24 * nglob, nloc=nloc)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s"


def kernel_source_hash() -> str:
    """Hash of the force kernel's sources (template, per-order units, record layout): a
    profile's counters stay valid while it matches."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2606_12850_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if name in ("sem_forces.cuh", "sem_internal.h", "sem_patches.cpp") or (
                name.startswith("sem_forces_") and name.endswith(".cu")):
            with open(os.path.join(csrc, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(ngll: int):
    """DRAM bytes per force-kernel launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"patch_forces_kernel_ngll{ngll}_layered.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_sweep:\s*([0-9.eE+]+)\s+kernel_sources:\s*([0-9a-f]+)", text)
    if not m or m.group(2) != kernel_source_hash():
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.proc = None
        target = str(device)
        try:
            import torch
            pr = torch.cuda.get_device_properties(device)
            target = "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
        except Exception:
            vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
            if vis:
                target = vis.split(",")[device]
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", target, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
                for name, val in zip(names, r[4:8]):
                    if val.strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_throughput(local_ms: float, units_per_rank: float, world: int, device=None):
    """Whole-job throughput of independent replicas: every rank processed units_per_rank
    in local_ms; the job takes the slowest rank's time (max over ranks).
    Returns (units per second over all ranks, max ms)."""
    import torch
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def host_cpu() -> dict:
    """Cores this process may run on and the CPU model (from /proc/cpuinfo)."""
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    model = "unknown"
    try:
        info = open("/proc/cpuinfo").read()
        m = re.search(r"^model name\s*:\s*(.+)$", info, re.M)
        if m:
            model = m.group(1).strip()
        else:  # Arm: implementer and part numbers
            imp = re.search(r"^CPU implementer\s*:\s*(\S+)", info, re.M)
            part = re.search(r"^CPU part\s*:\s*(\S+)", info, re.M)
            if imp and part:
                model = f"Arm implementer {imp.group(1)} part {part.group(1)}"
    except OSError:
        pass
    return {"cores": cores, "model": model}


def compiled_baseline(ngll: int, elems: int | None, seconds: float = 20.0, max_steps: int = 20):
    """The compiled FP64 CPU baseline (oracle/sem_cpu.c, pinned to the numpy oracle) on the
    full workload mesh: all host cores (OpenMP over the elements of one colour) for up to
    ``max_steps`` steps sized to about ``seconds``, and one core for one step. Returns a dict
    with local-pt updates/s per mode, the steps timed and the host description."""
    from oracle import sem_cpu, sem_oracle
    from paper_2606_12850_gb300 import inputs

    w = inputs.layered_cube(ngll, n=elems, nsteps=max_steps)
    t = time.perf_counter()
    m = sem_oracle.build_model(w)
    dt = m.cfl_dt(w.courant)
    src, _ = sem_oracle.locate_workload(m, w)
    setup_s = time.perf_counter() - t
    host = host_cpu()
    nloc = w.mesh.nlocal
    out = {"host": host, "setup_s": setup_s, "mesh": f"{w.mesh.nx}^3 NGLL={ngll}", "nlocal": nloc}
    kw = dict(src_node=int(src[0]), src_force=w.source_force[0], f0=w.f0, t0=w.t0)
    for mode, threads in (("all_cores", host["cores"]), ("one_core", 1)):
        cb = sem_cpu.CpuBaseline(m, threads)
        t = time.perf_counter()
        u, v, a = cb.run(dt, 1, **kw)
        one = time.perf_counter() - t
        steps = 1
        el = one
        if mode == "all_cores":
            steps = int(max(1, min(max_steps, seconds / max(one, 1e-9))))
            t = time.perf_counter()
            cb.run(dt, steps, u=u, v=v, a=a, **kw)
            el = time.perf_counter() - t
        out[mode] = {"threads": threads, "steps": steps, "seconds": el, "updates_per_s": nloc * steps / el}
    return out


def workload_name(args) -> str:
    """The workload both arms quote their metric on (the reference arm on bounded samples)."""
    from paper_2606_12850_gb300 import inputs
    n = args.elems or inputs.LAYERED_ELEMS.get(args.ngll, 64)
    return (f"three-layer jittered cube {n}^3 hex, NGLL={args.ngll}, 4 km "
            "(plain SEM scaling / (h,p) sweep configuration)")


def run_reference(args):
    """The reference arm: the oracle as it stands (its compiled FP64 baseline, pinned to the
    numpy oracle) on the host cores, on the same workload; the whole mesh when K + W steps
    of it fit in about two and a half minutes, else each step on the largest sub-cube of
    the same recipe that does."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import sem_cpu, sem_oracle
    from paper_2606_12850_gb300 import inputs

    budget = 150.0
    host = host_cpu()
    full = args.elems or inputs.LAYERED_ELEMS.get(args.ngll, 64)
    n = full
    while True:
        w = inputs.layered_cube(args.ngll, n=n, nsteps=args.steps)
        m = sem_oracle.build_model(w)
        cb = sem_cpu.CpuBaseline(m, host["cores"])
        dt = m.cfl_dt(w.courant)
        src, _ = sem_oracle.locate_workload(m, w)
        kw = dict(src_node=int(src[0]), src_force=w.source_force[0], f0=w.f0, t0=w.t0)
        t = time.perf_counter()
        u, v, a = cb.run(dt, 1, **kw)
        one = time.perf_counter() - t
        if (args.steps + args.warmup) * one <= budget or n <= 4:
            break
        n = max(4, int(n * ((budget / ((args.steps + args.warmup) * one)) ** (1 / 3))))
    u, v, a = cb.run(dt, max(0, args.warmup - 1), u=u, v=v, a=a, **kw)
    t = time.perf_counter()
    cb.run(dt, args.steps, u=u, v=v, a=a, **kw)
    el = time.perf_counter() - t
    value = w.mesh.nlocal * args.steps / el
    sample = (f"compiled FP64 CPU baseline of the oracle (oracle/sem_cpu.c, pinned to the numpy oracle) on "
              f"{host['cores']} host threads ({host['model']}), each step on the "
              + ("full workload mesh" if n == full else f"{n}^3-element cube of the same recipe (a bounded sample)"))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "ngll": args.ngll,
                   "parallelism": f"{host['cores']} host threads, colour by colour",
                   "sample_per_step": "the full mesh" if n == full else f"{n}^3 elements of the same recipe"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": host["cores"], "kind": "oracle", "sample": sample,
                         "cpu_model": host["model"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def measure_assembly_ablation(device: int, reps: int = 20):
    """Sec. V-D-1's colouring ablation on GB300: one stiffness sweep of the benchmark mesh
    (NGLL 5: 64^3, NGLL 9: 32^3) with the default patch assembly, the element-by-element
    coloured assembly, and the element kernel with float atomics instead of colours (one
    launch, f zeroed first). CUDA events, mean of ``reps`` sweeps after three untimed ones."""
    import torch

    from paper_2606_12850_gb300 import inputs, sem

    out = []
    for ngll in (5, 9):
        w = inputs.layered_cube(ngll, nsteps=10)
        stream = torch.cuda.Stream(device=device)
        s = sem.setup_workload(w, device=device, stream=stream)
        with torch.cuda.stream(stream):
            ud = (torch.rand(4 * w.mesh.nglob, device="cuda") - 0.5) * 2e-3
            fd = torch.empty_like(ud)
        stream.synchronize()
        row = {"ngll": ngll, "elements": f"{w.mesh.nx}^3"}
        for name, asm in (("patch_colours_ms", 0), ("element_colours_ms", 1), ("element_atomic_ms", 3)):
            sem.sem_set_option(s.ctx, sem.SEM_OPT_ASSEMBLY, asm)
            for _ in range(3):
                sem.sem_apply_stiffness_strided(s.ctx, ud, fd, 4)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, b in evs:
                a.record(stream)
                sem.sem_apply_stiffness_strided(s.ctx, ud, fd, 4)
                b.record(stream)
            stream.synchronize()
            row[name] = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        row["atomic_over_element_colours"] = row["element_atomic_ms"] / row["element_colours_ms"]
        out.append(row)
        del s
        torch.cuda.empty_cache()
    return {"rows": out, "paper_lx2": "removing the colouring (atomics) costs 1.16x at p = 15 (Sec. V-D-1)"}


def measure_batched(args, device: int):
    """Many shots on one model vs one shot at a time: the three-layer jittered cube with 48^3
    elements at NGLL=5 and S Ricker sources at seeded random positions. Shots/s are quoted
    for a 1000-step shot; rel_l2 compares the batched seismograms of two shots with their
    plain single-shot runs after the timed steps' worth of steps."""
    import torch

    from paper_2606_12850_gb300 import inputs, sem

    S, K = args.shots, args.shot_steps
    w, pos = inputs.batched_layered_cube(n=48, ngll=5, nshots=S)
    stream = torch.cuda.Stream(device=device)
    plain = sem.setup_workload(w, device=device, stream=stream)
    nodes = sem.sem_locate_nodes(plain.ctx, pos)
    force = np.tile([0.0, 0.0, 1.0e10], (S, 1))
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def timed(ctx, steps):
        a, b = ev(), ev()
        sem.sem_run_dev(ctx, 5, None)
        a.record(stream)
        sem.sem_run_dev(ctx, steps, None)
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b) / steps

    sem.sem_set_source_nodes(plain.ctx, nodes[:1], force[:1], w.f0, w.t0)
    ms_plain = timed(plain.ctx, K)
    batch = sem.setup_workload(w, device=device, stream=stream, src_nodes=nodes[:1], rec_nodes=plain.rec_nodes)
    sem.sem_set_shots(batch.ctx, S)
    sem.sem_set_shot_sources(batch.ctx, np.arange(S), nodes, force, w.f0, w.t0)
    sem.sem_set_state(batch.ctx)
    ms_batch = timed(batch.ctx, K)
    # accuracy: batched vs plain displacement fields of shots 0 and S-1 after 200 steps
    sem.sem_set_state(batch.ctx)
    sem.sem_run(batch.ctx, 200)
    u_b, _, _ = sem.sem_get_state(batch.ctx, want=(True, False, False))
    errs = []
    for sh in (0, S - 1):
        sem.sem_set_source_nodes(plain.ctx, nodes[sh:sh + 1], force[sh:sh + 1], w.f0, w.t0)
        sem.sem_set_state(plain.ctx)
        sem.sem_run(plain.ctx, 200)
        u_p, _, _ = sem.sem_get_state(plain.ctx, want=(True, False, False))
        errs.append(float(np.linalg.norm(u_b[sh] - u_p) / np.linalg.norm(u_p)))
    nloc = w.mesh.nlocal
    return {"model": f"three-layer jittered cube 48^3 hex, NGLL=5, {S} shots at seeded random positions",
            "shots": S, "steps_timed": K, "ms_per_step_batched": ms_batch, "ms_per_step_plain_one_shot": ms_plain,
            "shots_per_s_batched": S / (ms_batch * 1e-3 * 1000), "shots_per_s_plain": 1.0 / (ms_plain * 1e-3 * 1000),
            "speedup": S * ms_plain / ms_batch, "shot_pt_updates_per_s_batched": S * nloc / (ms_batch * 1e-3),
            "rel_l2_vs_plain": max(errs), "rel_l2_what": "displacement of shots 0 and S-1 after 200 steps",
            "shot_steps_for_shots_per_s": 1000}


def measure_hp_sweep(device: int, steps: int = 50):
    """(h,p) cost on GB300 at a fixed number of GLL intervals per side (256, i.e. fixed
    points per wavelength): for NGLL = 3, 5, 7, 9 the throughput, the CFL step, device
    memory and the device time to simulate one second (steps = 1 s / dt)."""
    import torch

    from paper_2606_12850_gb300 import inputs, sem

    out = []
    for ngll in (3, 5, 7, 9):
        w = inputs.layered_cube(ngll)
        stream = torch.cuda.Stream(device=device)
        s = sem.setup_workload(w, device=device, stream=stream)
        info = sem.sem_info(s.ctx)
        sem.sem_run_dev(s.ctx, 5, None)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sem.sem_run_dev(s.ctx, steps, None)
        b.record(stream)
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        nloc = w.mesh.nlocal
        out.append({"ngll": ngll, "elements": f"{w.mesh.nx}^3", "nlocal": nloc, "nglob": w.mesh.nglob,
                    "ms_per_step": ms, "updates_per_s": nloc / (ms * 1e-3), "dt": s.dt,
                    "device_mb": info["device_bytes"] / 1e6, "seconds_per_simulated_second": ms * 1e-3 / s.dt})
        del s
    return out


def measure_adjoint(device: int, nsteps: int = 800, every: int = 50):
    """Cost of one misfit gradient against one plain forward run of the same model: the
    three-layer jittered cube with 32^3 elements at NGLL=5, a 5 % Gaussian velocity anomaly
    in the true model, 64 surface receivers, ``nsteps`` steps with a checkpoint every
    ``every``. The observed data come from the true model; the L2 misfit's gradient in
    (rho, kappa, mu) is taken at the unperturbed layers. ``fd_rel_err`` compares the
    gradient's directional derivative along a seeded per-element direction with a central
    difference of the float32 misfit (step 1e-3), a sanity check at full size; the parity
    bar is the oracle comparison of the tests."""
    import torch

    from paper_2606_12850_gb300 import adjoint, inputs, sem

    w = inputs.perturbed_layered_cube(n=32, ngll=5, nsteps=nsteps, nrec_side=8)
    stream = torch.cuda.Stream(device=device)
    s = sem.setup_workload(w, device=device, stream=stream)  # true model; its dt is the smaller one
    ctx, nrec = s.ctx, len(s.rec_nodes)
    dev = torch.device("cuda", device)
    with torch.cuda.stream(stream):
        d_obs = torch.empty((nrec, 3, nsteps), device=dev)
    sem.sem_run_dev(ctx, nsteps, d_obs)
    sem.sem_sync(ctx)
    rho_b, vp_b, vs_b = (x.astype(np.float64) for x in w.extra["background"])
    mu = rho_b * vs_b ** 2
    kappa = rho_b * vp_b ** 2 - 4.0 / 3.0 * mu
    mat = [torch.from_numpy(x.astype(np.float32)).to(dev) for x in (rho_b, kappa, mu)]
    sim = adjoint.Simulation(ctx, s.dt, nsteps, checkpoint_every=every, device=device)  # keeps all if they fit

    sim.set_material(*mat)  # plain forward of the same model, device-timed
    sem.sem_set_state(ctx)
    with torch.cuda.stream(stream):
        buf = torch.empty((nrec, 3, nsteps), device=dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    sem.sem_run_dev(ctx, nsteps, buf)
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)

    def misfit(seis):
        return 0.5 * s.dt * float(torch.sum((seis.double() - d_obs.double()) ** 2))

    def timed_gradient(sm):
        sm.gradient(s.dt * (sm.forward(*mat) - d_obs))  # warm-up: the allocator's first blocks
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        seis = sm.forward(*mat)
        G = s.dt * (seis - d_obs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        grads = sm.gradient(G)
        t2 = time.perf_counter()
        return seis, grads, 1e3 * (t1 - t0), 1e3 * (t2 - t1)

    # every step's displacement kept on the device (no recomputation), the default when it fits
    seis, (g_rho, g_kappa, g_mu), fwd_ms, bwd_ms = timed_gradient(sim)
    kept = sim.snapshots is not None
    kept_mb = sim.snapshots.numel() * 4 / 1e6 if kept else 0.0
    sim.snapshots = None
    L0 = misfit(seis)
    # checkpoints every `every` steps and recomputed segments (when memory is short)
    sim_ck = adjoint.Simulation(ctx, s.dt, nsteps, checkpoint_every=every, device=device, keep_all=False)
    _, g_ck, ck_fwd_ms, ck_bwd_ms = timed_gradient(sim_ck)
    ck_diff = max(float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(g_ck, (g_rho, g_kappa, g_mu)))

    # float32 directional finite difference along a seeded per-element direction
    nspec = w.mesh.nspec
    r = [inputs.uniform(9, (nspec, 1), -1.0, 1.0, stream=k) for k in (1, 2, 3)]
    base = (rho_b, kappa, mu)
    dirs = [p_ * r_ for p_, r_ in zip(base, r)]
    predicted = float(sum(np.sum(g * d) for g, d in zip((g_rho, g_kappa, g_mu), dirs)))
    h = 1e-3
    Ls = []
    for sg in (+1, -1):
        pert = [torch.from_numpy((p_ + sg * h * d).astype(np.float32)).to(dev) for p_, d in zip(base, dirs)]
        sim.set_material(*pert)
        sem.sem_set_state(ctx)
        sem.sem_run_dev(ctx, nsteps, buf)
        sem.sem_sync(ctx)
        Ls.append(misfit(buf))
    fd = (Ls[0] - Ls[1]) / (2 * h)
    nglob = w.mesh.nglob
    return {"model": f"{w.name}, {nrec} surface receivers", "nsteps": nsteps,
            "plain_forward_ms": plain_ms, "mode": "every displacement kept" if kept else "checkpointed",
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "gradient_ms": fwd_ms + bwd_ms, "gradient_over_plain_forward": (fwd_ms + bwd_ms) / plain_ms,
            "snapshots_mb": kept_mb,
            "checkpointed": {"checkpoint_every": every, "forward_ms": ck_fwd_ms, "backward_ms": ck_bwd_ms,
                             "gradient_over_plain_forward": (ck_fwd_ms + ck_bwd_ms) / plain_ms,
                             "checkpoint_mb": len(sim_ck.checkpoints) * 3 * 3 * nglob * 4 / 1e6,
                             "segment_mb": (every + 2) * 3 * nglob * 4 / 1e6,
                             "max_rel_l2_vs_kept": ck_diff},
            "misfit": L0,
            "fd_directional": fd, "adjoint_directional": predicted,
            "fd_rel_err": abs(fd - predicted) / abs(fd) if fd else None,
            "timing": "plain forward: CUDA events; gradient: wall clock including host synchronisation, "
                      "after one untimed gradient"}


def measure_tiles(device: int, reps: int = 10):
    """Element tiles per NGLL picked by the autotuner (sem_tune_patch_shape): every brick shape
    of the order's patch CTA timed on the three-layer jittered cube at 128 GLL intervals per
    side (32^3 / 22^3 / 16^3 elements at NGLL 5 / 7 / 9), ms of one time step's sweep."""
    from paper_2606_12850_gb300 import inputs, sem

    out = []
    for ngll, n in ((5, 32), (7, 22), (9, 16)):
        w = inputs.layered_cube(ngll, n=n, nsteps=10)
        ctx = sem.sem_create(ngll, device)
        rows, best = sem.sem_tune_patch_shape(ctx, w.mesh.ibool, w.mesh.nglob, w.rho, w.vp, w.vs,
                                              ctrl=w.mesh.ctrl, reps=reps)
        tiny = inputs.structured_hex_mesh((2, 2, 2), ngll, 1.0)  # the order's default brick
        info = sem.sem_patch_plan(ngll, tiny.ibool, tiny.nglob)[2]
        default = (info["bx"], info["by"], info["bz"])
        ms = dict(rows)
        out.append({"ngll": ngll, "elements": f"{n}^3",
                    "shapes_ms": {"x".join(map(str, k)): v for k, v in rows},
                    "chosen": "x".join(map(str, best)), "default": "x".join(map(str, default)),
                    "chosen_over_default": ms[tuple(default)] / ms[best]})
        del ctx
    return out


def measure_models(device: int, count: int = 16, steps: int = 50):
    """Many independent models on one GPU: homogeneous cubes of 8^3 .. 40^3 elements with
    NGLL cycling through 4 .. 8, each autotuned (contraction form), stepped one after
    another (each with its own CUDA graphs) against all together (sem_group_step: one graph
    launch per ten steps, every model a branch of its own)."""
    import torch

    from paper_2606_12850_gb300 import inputs, sem

    sizes = np.linspace(8, 40, count).round().astype(int)
    orders = [4 + k % 5 for k in range(count)]
    stream = torch.cuda.Stream(device=device)
    setups, desc, tuned = [], [], []
    for n, ngll in zip(sizes, orders):
        w = inputs.homogeneous_cube(int(n), ngll, nsteps=steps)
        s = sem.setup_workload(w, device=device, stream=stream)
        ms, choice = sem.sem_autotune(s.ctx, reps=3)
        setups.append(s)
        desc.append(f"{n}^3/{ngll}")
        tuned.append({"model": f"{n}^3 NGLL {ngll}", "line_owners_ms": ms[0], "per_point_ms": ms[1],
                      "form": "line owners" if choice == 1 else "per point"})
    nloc = sum(int(s.ctx.nspec) * int(s.ctx.ngll) ** 3 for s in setups)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for s in setups:  # warm-up (graphs)
        sem.sem_run_dev(s.ctx, 12, None)
    stream.synchronize()
    a, b = ev(), ev()
    a.record(stream)
    for s in setups:
        sem.sem_run_dev(s.ctx, steps, None)
    b.record(stream)
    b.synchronize()
    seq_ms = a.elapsed_time(b)
    group = sem.Group([s.ctx for s in setups])

    def group_time(mode):
        group.set_option(sem.SEM_GROUP_MODE, mode)
        group.step(12)
        group.sync()
        torch.cuda.synchronize()
        t = time.perf_counter()
        group.step(steps)
        group.sync()
        return 1e3 * (time.perf_counter() - t)

    persistent_ms = group_time(1)
    info = group.info()
    group_ms = group_time(0)  # the default mode
    return {"models": desc, "steps": steps, "nlocal_total": nloc, "sequential_ms": seq_ms, "group_ms": group_ms,
            "group_mode": "graph branches (default)",
            "speedup": seq_ms / group_ms, "group_updates_per_s": nloc * steps / (group_ms * 1e-3),
            "sequential_updates_per_s": nloc * steps / (seq_ms * 1e-3),
            "persistent_ms": persistent_ms, "persistent_speedup": seq_ms / persistent_ms,
            "persistent_sweep_launches_per_step": info["sweep_launches"], "autotune": tuned,
            "timing": "sequential: CUDA events on the models' stream; group: wall clock around "
                      "sem_group_step and sem_group_sync"}


def plane_wave_error(ngll: int, nz: int, periods: float, steps_per_period: int, device: int = 0) -> float:
    """Waveform error (Sec. V-C-1: squared-norm ratio against the analytic solution, all
    stations on a line along z) of a P plane wave of wavelength 1 km (vp 3 km/s) travelling
    ``periods`` periods through a periodic 2 x 2 x nz-element box 8 wavelengths long, from its
    exact initial displacement and velocity (acceleration from the discrete operator)."""
    from paper_2606_12850_gb300 import inputs, sem
    lam, vp = 1000.0, 3000.0
    h = 8 * lam / nz
    mesh = inputs.structured_hex_mesh((2, 2, nz), ngll, (2 * h, 2 * h, 8 * lam), periodic=True)
    one = np.ones(mesh.nspec)
    ctx = sem.sem_create(ngll, device)
    sem.sem_set_mesh_corners(ctx, mesh.ibool, mesh.ctrl, mesh.nglob)
    sem.sem_set_material(ctx, inputs.per_point(mesh, 2500 * one), inputs.per_point(mesh, vp * one),
                         inputs.per_point(mesh, 1730 * one))
    k = 2 * np.pi / lam
    w = vp * k
    period = 2 * np.pi / w
    dt = period / steps_per_period
    n = int(round(periods * steps_per_period))
    sem.sem_set_dt(ctx, dt)
    X = sem.sem_node_xyz(ctx, np.arange(mesh.nglob))
    u0 = np.zeros((mesh.nglob, 3), dtype=np.float32)
    v0 = np.zeros((mesh.nglob, 3), dtype=np.float32)
    u0[:, 2] = np.sin(k * X[:, 2])
    v0[:, 2] = -w * np.cos(k * X[:, 2])
    Lxy = mesh.lengths[0]
    on_x = np.isclose(np.mod(X[:, 0] + 0.5 * Lxy, Lxy), 0.5 * Lxy)  # x = 0 or its periodic image
    on_y = np.isclose(np.mod(X[:, 1] + 0.5 * Lxy, Lxy), 0.5 * Lxy)
    rec = np.nonzero(on_x & on_y)[0]
    if rec.size == 0:
        raise RuntimeError("no station line found")
    sem.sem_set_receiver_nodes(ctx, rec)
    sem.sem_set_state(ctx, u0, v0, None)
    sem.sem_init_acceleration(ctx)
    seis = sem.sem_run(ctx, n)
    t = dt * np.arange(1, n + 1)
    theory = np.sin(k * X[rec, 2][:, None] - w * t[None, :])
    wz = seis[:, 2, :].astype(np.float64)
    return float(np.sum((wz - theory) ** 2) / np.sum(theory ** 2))


def measure_iso_accuracy(device: int, target: float = 1e-2, periods: float = 20.0, steps_per_period: int = 400):
    """The (h, p) iso-accuracy study (Sec. V-C-1) on the GPU, elastic: for every order the
    largest element (fewest elements per wavelength) whose plane-wave error after
    ``periods`` periods stays within ``target``, at one time step for all (400 per period,
    its temporal error far below the target); then the cost of p = 4 against p = 7 and
    p = 9 on one domain at those element sizes: time per step and device memory at the
    common time step (the paper's comparison, p = 15 being beyond this build's orders)."""
    import torch

    from paper_2606_12850_gb300 import inputs, sem

    candidates = [3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 36, 40, 48, 56, 64]
    frontier = []
    for ngll in (3, 4, 5, 6, 7, 8, 9, 10):
        tried = []
        for nz in candidates:
            err = plane_wave_error(ngll, nz, periods, steps_per_period, device)
            tried.append((nz / 8.0, err))
            if err <= target:
                break
        epw, err = tried[-1]
        frontier.append({"ngll": ngll, "p": ngll - 1, "elements_per_wavelength": epw,
                         "h_over_wavelength": 1.0 / epw, "error": err, "error_sqrt": float(np.sqrt(err)),
                         "met": err <= target,
                         "tried": [[a, b] for a, b in tried]})
    # cost on one domain: p = 4 on 64^3 elements, the others scaled by the frontier's h ratio
    lam, vp = 1000.0, 3000.0
    dt = 2 * np.pi / (vp * 2 * np.pi / lam) / steps_per_period
    h = {f["p"]: lam / f["elements_per_wavelength"] for f in frontier}
    side = 64 * h[4]
    costs = []
    stream = torch.cuda.Stream(device=device)
    for p in (4, 7, 9):
        n = max(2, int(round(side / h[p])))
        w = inputs.homogeneous_cube(n, p + 1, side=side, vp=vp, vs=1730.0, nsteps=100)
        s = sem.setup_workload(w, device=device, stream=stream, dt=dt)
        info = sem.sem_info(s.ctx)
        sem.sem_run_dev(s.ctx, 10, None)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        sem.sem_run_dev(s.ctx, 100, None)
        b.record(stream)
        b.synchronize()
        costs.append({"p": p, "elements": f"{n}^3", "h_m": side / n, "ms_per_step": a.elapsed_time(b) / 100,
                      "device_mb": info["device_bytes"] / 1e6, "nglob": info["nglob"]})
        del s
    base = costs[0]
    for c in costs:
        c["time_reduction_vs_p4"] = base["ms_per_step"] / c["ms_per_step"]
        c["memory_reduction_vs_p4"] = base["device_mb"] / c["device_mb"]
    return {"target_error": target, "periods": periods, "steps_per_period": steps_per_period,
            "frontier": frontier, "domain_m": side, "dt": dt, "costs": costs,
            "paper_lx2": "p4 -> p7: 3.18x less memory, 3.85x less time; p7 -> p15: 1.8x / 1.4x (acoustic "
                         "frontier, 160 periods, elastic runs of 15 000 steps)"}


def measure_surrogate(device: int, runs: int, epochs: int, heldout: int = 256, batch: int = 256):
    """The learned surrogate of the 16^3 layered medium (NGLL 5, 64 surface receivers, 1000
    steps, Ricker 0.5 Hz): ``runs`` solver runs with seeded random positions and unit moment
    tensors (32 shots per launch), Adam training of the default network, then the held-out
    error per run (relative L2 over receivers, components and samples) against new solver
    runs, next to the answer without learning (the nearest training run), and the time per
    source of the network (batch 4096) against the solver."""
    import torch

    from paper_2606_12850_gb300 import inputs, surrogate

    w = inputs.surrogate_cube()
    solver = surrogate.Solver(w, shots=32, device=device)
    tr = surrogate.generate_runs(solver, runs, seed=1)
    te = surrogate.generate_runs(solver, heldout, seed=2)
    amp = solver.amplitude_model().fit(tr.xyz, surrogate.run_rms(tr.y))
    yn = surrogate.training_targets(tr.y, amp(tr.xyz), 1.0)
    scale = 1.0 / float(yn.pow(2).mean().sqrt())
    yn.mul_(scale)
    spec = surrogate.Spec()
    model = surrogate.Model(spec, max_batch=batch, device=device)
    model.set_params(spec.init_params(1))
    x = torch.from_numpy(tr.x).to(torch.device("cuda", device))
    torch.cuda.synchronize()
    t = time.perf_counter()
    losses = surrogate.train(model, x, yn, epochs=epochs, batch=batch, lr=2e-3, seed=3)
    train_s = time.perf_counter() - t
    del yn
    sur = surrogate.Surrogate(model, scale, w.mesh.lengths[0], amp, solver)
    pred = sur.predict(te.xyz, te.moments)
    err = surrogate.rel_l2_per_run(pred, te.y)
    err_nn = surrogate.rel_l2_per_run(surrogate.nearest_run_baseline(tr, te), te.y)
    n_inf = 4096
    xi = x[:n_inf].contiguous() if runs >= n_inf else x.repeat((n_inf + runs - 1) // runs, 1)[:n_inf].contiguous()
    yi = torch.empty((n_inf, spec.out_c, spec.out_l), device=x.device)
    model.forward(xi, yi)
    model.sync()
    torch.cuda.synchronize()
    t = time.perf_counter()
    model.forward(xi, yi)
    model.sync()
    infer_s = time.perf_counter() - t
    products = compare_products(model, spec, xi, yi, batch)
    solver_ms = 1e3 * (tr.seconds + te.seconds) / (runs + heldout)
    net_ms = 1e3 * infer_s / n_inf
    return {"medium": w.name, "train_runs": runs, "heldout_runs": heldout,
            "network": f"MLP 9-512-512, seed [64][125], conv decoder x2 x2 x2 to 1000 samples, "
                       f"6 x 192 channels combined with the moment tensor; {model.nparams} parameters, bf16 "
                       "weights and operands, fp32 accumulate, tcgen05 products (TMEM accumulators)",
            "epochs": epochs, "batch": batch, "train_s": train_s, "final_loss": losses[-1],
            "generation_s": tr.seconds + te.seconds, "solver_ms_per_run": solver_ms,
            "network_ms_per_source_batch4096": net_ms, "speedup_per_source": solver_ms / net_ms,
            "heldout_rel_l2": {"median": float(np.median(err)), "mean": float(err.mean()),
                               "p90": float(np.percentile(err, 90))},
            "nearest_run_rel_l2": {"median": float(np.median(err_nn)), "mean": float(err_nn.mean())},
            "products": products,
            "timing": "wall clock with device synchronisation"}


def product_flops(spec) -> int:
    """Multiply-add FLOPs (2 per multiply-add) of the network's products for one input: the
    three dense layers and the decoder's width-3 convolutions."""
    f = spec.in_dim * spec.hidden + spec.hidden * spec.hidden + spec.hidden * spec.c0 * spec.l0
    cin, length = spec.c0, spec.l0
    for co, up in zip(spec.stage_cout, spec.stage_up):
        length *= up
        f += co * cin * 3 * length
        cin = co
    return 2 * f


def compare_products(model, spec, xi, yi, batch: int, reps: int = 5):
    """The same forward (len(xi) inputs) and loss-gradient step (``batch`` inputs) with each
    product kernel: tcgen05 with TMEM accumulators (the default) and warp-level mma.sync;
    median wall clock of ``reps`` synchronised repetitions after one warm-up. The loss step
    takes the network's own outputs as targets (its gradients are not applied)."""
    xb = xi[:batch].contiguous()
    tb = yi[:batch].clone()
    flops = product_flops(spec)
    out = {}
    for kind, name in ((1, "tcgen05"), (0, "mma_sync")):
        model.product = kind
        res = {}
        for what, fn, n, mult in (("forward", lambda: model.forward(xi, yi), len(xi), 1),
                                  ("loss_grad", lambda: model.loss_grad(xb, tb), batch, 3)):
            fn()
            model.sync()
            times = []
            for _ in range(reps):
                t0 = time.perf_counter()
                fn()
                model.sync()
                times.append(time.perf_counter() - t0)
            ms = 1e3 * float(np.median(times))
            res[what] = {"batch": n, "ms": ms, "product_tflops": mult * flops * n / (ms * 1e-3) / 1e12}
        out[name] = res
    model.product = 1
    out["product_gflop_per_input"] = flops / 1e9
    out["speedup_forward"] = out["mma_sync"]["forward"]["ms"] / out["tcgen05"]["forward"]["ms"]
    out["speedup_loss_grad"] = out["mma_sync"]["loss_grad"]["ms"] / out["tcgen05"]["loss_grad"]["ms"]
    return out


def run_ours(args):
    import torch

    from paper_2606_12850_gb300 import build, inputs, sem

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()

    K, W = args.steps, args.warmup
    w = inputs.layered_cube(args.ngll, n=args.elems, nsteps=K)
    mesh = w.mesh
    stream = torch.cuda.Stream(device=local)
    s = sem.setup_workload(w, device=local, stream=stream)
    ctx = s.ctx
    info = sem.sem_info(ctx)
    pinfo = sem.sem_patch_info(ctx)
    ncolors = pinfo["colors"]
    alg = algorithmic_bytes(mesh.nspec, mesh.ngll, mesh.nglob)
    nrec = len(s.rec_nodes)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    with torch.cuda.stream(stream):
        seis_w = torch.empty(max(1, nrec * 3 * W), device="cuda")
        seis = torch.empty(max(1, nrec * 3 * K), device="cuda")
    sem.sem_run_dev(ctx, W, seis_w)
    barrier()
    clocks = ClockSampler(local)
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    sem.sem_run_dev(ctx, K, seis)
    end.record(stream)
    end.synchronize()
    clock_info = clocks.stop()
    ms = start.elapsed_time(end)
    barrier()
    value, ms = replica_throughput(ms, alg["nloc"] * K, world, device="cuda")
    launches = K * (ncolors + 1) + 2  # per step: receiver sampling + one launch per patch colour

    # the dominant kernel (force kernel over all colours) timed alone on the same stream
    # (the solver's own [nglob][4] field layout, so this is the kernel the time step runs)
    with torch.cuda.stream(stream):
        ud = (torch.rand(4 * mesh.nglob, device="cuda") - 0.5) * 2e-3
        fd = torch.empty_like(ud)
    stream.synchronize()
    for _ in range(3):
        sem.sem_apply_stiffness_strided(ctx, ud, fd, 4)
    reps = max(1, args.stiffness_reps)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:
        a.record(stream)
        sem.sem_apply_stiffness_strided(ctx, ud, fd, 4)
        b.record(stream)
    stream.synchronize()
    forces_ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    peak, peak_src = measured_peaks()
    forces_gbs = alg["forces"] / (forces_ms / 1e3) / 1e9
    # the dominant kernel of the timed step: the force sweep with the Newmark update fused in
    # (all colour launches of one step), timed with CUDA events around each step's sweep
    sweep_ms, rest_ms = sem.sem_profile_steps(ctx, max(10, args.stiffness_reps // 2))
    achieved = alg["step"] / (sweep_ms / 1e3) / 1e9
    traffic = profiled_traffic(args.ngll)
    step_gbs = alg["step"] * K / (ms / 1e3) / 1e9

    # end to end through the C ABI with host buffers: initial state up, K steps, seismograms
    # and final displacement down (pinned host memory)
    e2e = None
    if not args.no_e2e:
        pin = lambda shape: torch.zeros(shape, dtype=torch.float32, pin_memory=True).numpy()
        u0, v0, a0 = pin((mesh.nglob, 3)), pin((mesh.nglob, 3)), pin((mesh.nglob, 3))
        seis_h = pin((nrec, 3, K))
        u_out = pin((mesh.nglob, 3))
        barrier()
        t = time.perf_counter()
        sem.sem_set_state(ctx, u0, v0, a0)
        sem.sem_run(ctx, K, out=seis_h)
        lib = sem.lib()
        rc = lib.sem_get_state(ctx.handle, u_out.ctypes.data_as(sem._P), None, None)
        if rc != 0:
            raise RuntimeError(sem.sem_last_error(ctx))
        el = time.perf_counter() - t
        e2e_value, _ = replica_throughput(1e3 * el, alg["nloc"] * K, world, device="cuda")
        h2d = 3 * mesh.nglob * 3 * 4
        d2h = nrec * 3 * K * 4 + mesh.nglob * 3 * 4
        e2e = {"value": e2e_value, "unit": UNIT,
               "h2d_bytes_per_step": h2d / K, "d2h_bytes_per_step": d2h / K,
               "what": "sem_set_state (u,v,a from pinned host) + sem_run (K steps, seismograms to host) + "
                       "sem_get_state (u to host), wall clock"}

    batched = None
    if args.shots > 1:
        dt_main = s.dt
        del s, ctx
        batched = measure_batched(args, local)
    else:
        dt_main = s.dt

    sweep = None
    if not args.no_sweep:
        sweep = measure_hp_sweep(local)

    adj = None
    if args.adjoint_steps > 0:
        adj = measure_adjoint(local, args.adjoint_steps)

    iso = None
    if not args.no_iso:
        iso = measure_iso_accuracy(local)

    ablation = None
    if not args.no_ablation:
        ablation = measure_assembly_ablation(local)

    models = None
    if args.models > 0:
        models = measure_models(local, args.models)

    tiles = None
    if not args.no_tiles:
        tiles = measure_tiles(local)

    sur = None
    if args.surrogate_runs > 0:
        sur = measure_surrogate(local, args.surrogate_runs, args.surrogate_epochs)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = compiled_baseline(args.ngll, args.elems, seconds=args.cpu_seconds)
        h = cb["host"]
        cpu = {"value": cb["all_cores"]["updates_per_s"], "unit": UNIT, "cores": h["cores"], "kind": "oracle",
               "sample": (f"compiled FP64 CPU baseline of the oracle (oracle/sem_cpu.c, pinned to the numpy oracle), "
                          f"the full {cb['mesh']} workload mesh, {cb['all_cores']['steps']} steps on "
                          f"{h['cores']} host threads (OpenMP over the elements of one colour)"),
               "cpu_model": h["model"],
               "one_core": {"value": cb["one_core"]["updates_per_s"], "steps": 1},
               "all_cores": cb["all_cores"], "setup_s": cb["setup_s"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "ngll": mesh.ngll, "nspec": mesh.nspec, "nglob": mesh.nglob, "nlocal": alg["nloc"],
                       "ncolors": ncolors, "nrec": nrec, "dt": dt_main,
                       "l2": "inputs larger than L2: 1.7 GB of element records stream every step",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": f"patch_forces_kernel<{mesh.ngll}, fused Newmark> (all {ncolors} patch-colour "
                                   f"launches of one time step; bricks of {pinfo['bx']}x{pinfo['by']}x{pinfo['bz']} "
                                   "elements; forces, sources, corrector and predictor)",
                         "algorithmic_bytes": alg["step"],
                         "bytes_rule": "52 B per local point + 76 B per global node (one time step)",
                         "sweep_ms": sweep_ms, "rest_of_step_ms": rest_ms, "peak_source": peak_src},
            "forces_only": {"kernel": f"patch_forces_kernel<{mesh.ngll}> (stiffness application alone)",
                            "ms": forces_ms, "achieved": forces_gbs, "frac": forces_gbs / peak,
                            "algorithmic_bytes": alg["forces"],
                            "bytes_rule": "52 B per local point + 24 B per global node"},
            "hbm_roofline_step": {"achieved": step_gbs, "frac": step_gbs / peak, "unit": "GB/s",
                                  "bytes_per_step": alg["step"]},
            "global_pt_updates_per_s": world * mesh.nglob * K / (ms / 1e3),
            "e2e": e2e, "cpu_baseline": cpu, "gpu_launches": launches, "clocks": clock_info,
            "batched_shots": batched, "uneven_models": models, "element_tiles": tiles, "hp_sweep": sweep, "iso_accuracy": iso,
            "assembly_ablation": ablation,
            "adjoint": adj,
            "surrogate": sur,
            "kernel_sources": kernel_source_hash(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_products_only(n: int):
    """The default surrogate network with seeded weights (init_params(1)) on n seeded inputs:
    forward and loss-gradient step with each product kernel (compare_products)."""
    import torch

    from paper_2606_12850_gb300 import build, inputs, surrogate

    build.build()
    spec = surrogate.Spec()
    model = surrogate.Model(spec, max_batch=min(n, 256))
    model.set_params(spec.init_params(1))
    x = torch.from_numpy(inputs.uniform(3, (n, spec.in_dim), -1, 1).astype(np.float32)).cuda()
    y = torch.empty((n, spec.out_c, spec.out_l), device="cuda")
    print(json.dumps(compare_products(model, spec, x, y, min(n, 256))))
    return 0


def main():
    args = parse_args()
    if args.products_only > 0:
        return run_products_only(args.products_only)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
