"""Benchmark of the D3Q19 pseudopotential MRT step on GB300.

Workload (the 256^3 throughput configuration): one periodic 256^3 box, a
Carnahan-Starling droplet R = 40 at the centre, T = 0.7 T_c, a = 1, b = 4, R = 1,
G = -1, s_nu = 1.0, other rates 1.1, 1000 steps.  At this temperature the
square-root pseudopotential needs the thermodynamic-consistency term of Eq. 16
(sigma = 0.105 for droplets, 0.116 for flat interfaces, Sec. IV D): without it
the vapour density turns negative within ten steps, in the FP64 oracle as well.
The initial tanh profile (Eq. 59) has width W = 3, close to the interface this
model settles to: a W = 5 profile leaves a shell that relaxes by sending a
converging density wave into the droplet, which focuses at the centre of an
R = 40 droplet and makes the run non-finite after about 55 steps (FP64
included); with W = 3 all forms run the 1000 steps.  The headline line is
the non-orthogonal operator with FP32 arithmetic and storage, stepped as the
library steps it by default: one launch per step of the work-list single pass
(the fused pass and the next step's psi pass as interleaved tile jobs).  The
``forms`` object adds both operators in FP64, FP32 (also as the two-pass step)
and FP16 storage, the D3Q15 variant of the non-orthogonal operator in the same
three precisions, all on the same box, and the batched and served forms.  A
"step" is one lattice time step over the whole box; MLUPS = 1e-6 * nodes *
steps / second.  Timing: the median of --repeats regions of --steps steps, each
bracketed by CUDA events on the launch stream with nothing else recorded inside
(the kernel split comes from a separate region with per-launch events).

  python bench.py [--gpus N --steps K --warmup W --repeats R] [--impl reference]
                  [--forms headline|batch|batched|all] [--op nonorth|orth|nonorth_d3q15] [--prec f64|f32|f16]
                  [--mode default|two-pass|queue|lagged|onchip|single|tma]

Under torchrun (N > 1) each rank runs its own box on its own GPU (replicas,
weak scaling); the timed region is bracketed by barriers and the max over
ranks is taken.
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

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")  # CPU oracle leg: single-threaded numpy
os.environ.setdefault("OMP_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "MLUPS and % of HBM roofline per D3Q19 step (FP64 vs FP32/FP16); p50/p99 job latency"
UNIT = "MLUPS"
EDGE = 256
T_OVER_TC = 0.7
A, B, R_GAS, G = 1.0, 4.0, 1.0, -1.0
RATES = dict(s_e=1.1, s_nu=1.0, s_q=1.1, s_pi=1.1, s_eps=1.1, s_m=1.1)
SIGMA_DROPLET, SIGMA_FLAT = 0.105, 0.116
W_DROPLET, W_FLAT = 5.0, 2.0  # a = 0.25 droplet forms (batched, served, precision study), flat slab
W_HEADLINE = 3.0                # the a = 1 droplet of the 256^3 throughput box
# algorithmic bytes per node of the fused pass: 19 populations read + 19 written + psi(x) read
FUSED_BYTES = {"f64": 19 * 8 * 2 + 8, "f32": 19 * 4 * 2 + 4, "f16": 19 * 2 * 2 + 4}
# ... and of the psi pass: 19 populations read + psi written
PSI_BYTES = {"f64": 19 * 8 + 8, "f32": 19 * 4 + 4, "f16": 19 * 2 + 4}
# the same for the D3Q15 variant (15 populations per node)
FUSED_BYTES_Q15 = {"f64": 15 * 8 * 2 + 8, "f32": 15 * 4 * 2 + 4, "f16": 15 * 2 * 2 + 4}
PSI_BYTES_Q15 = {"f64": 15 * 8 + 8, "f32": 15 * 4 + 4, "f16": 15 * 2 + 4}
# minimum bytes per lattice update: populations read and written once, psi read and written once
STEP_MIN_BYTES = {"f64": 19 * 8 * 2 + 16, "f32": 19 * 4 * 2 + 8, "f16": 19 * 2 * 2 + 8}
STEP_MIN_BYTES_Q15 = {"f64": 15 * 8 * 2 + 16, "f32": 15 * 4 * 2 + 8, "f16": 15 * 2 * 2 + 8}
HEADLINE = ("nonorth", "f32")
# DRAM bytes per node of the fused pass, from one ncu capture of the current kernel at 256^3 (dram__bytes_read
# + dram__bytes_write over the nodes); null for forms without such a capture.
FUSED_DRAM_BYTES = {("nonorth", "f32"): 152.6, ("nonorth", "f16"): 77.4}
# DRAM bytes per node of one launch of the work-list single pass at 256^3 (ncu dram__bytes_read.sum +
# dram__bytes_write.sum of one launch over the nodes), from a capture of the current kernel only
QUEUE_DRAM_BYTES = {("nonorth", "f32"): 170.1}
# FP64 instructions per node of the fused pass (ncu instruction counts at 128^3 over the nodes) and the FP64
# issue peak of one GB300: 2 per SM per clock x 152 SMs x 2070 MHz.
FUSED_FP64_INSTR = {"nonorth": 255.0, "orth": 309.0, "nonorth_d3q15": 207.0}
FP64_PEAK_GINSTR = 2 * 152 * 2070e6 / 1e9
PREC_TEXT = {"f64": "FP64 compute and storage", "f32": "FP32 compute and storage",
             "f16": "FP32 compute, FP16 storage"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling (200 ms) while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
            os.unlink(self.path)
        except Exception:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def make_lattice(op, prec, edge, sigma=SIGMA_DROPLET):
    from paper_1805_08643_gb300 import thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    Tc = thermo.critical_temperature(A, B, R_GAS)
    rl, rv = thermo.coexistence_cs(T_OVER_TC, A, B, R_GAS)
    lat = Lattice((edge,) * 3, operator=op, precision=prec, eos="cs", a=A, b=B, R=R_GAS,
                  T=T_OVER_TC * Tc, G=G, rates=Rates(**RATES), sigma=sigma)
    return lat, rl, rv


MODES = {"default": None, "two-pass": 0, "single": 1, "tma": "tma", "onchip": "onchip", "lagged": "lagged",
         "queue": "queue"}


def time_form(op, prec, edge, steps, warmup, world, clocks_index=None, field="droplet", mode="default",
              eos_arith="f64", repeats=5):
    """Device time of one form: `repeats` regions of `steps` steps each (CUDA events on the launch stream,
    nothing else recorded inside them; barrier + synchronize around each), median per step; then, outside
    those regions, one region of the same steps with per-launch events for the kernel split."""
    import torch

    lat, rl, rv = make_lattice(op, prec, edge, SIGMA_DROPLET if field == "droplet" else SIGMA_FLAT)
    if MODES[mode] is not None:
        m = MODES[mode]
        lat.set_tuning(m if isinstance(m, str) else bool(m), 1, 0)
    if eos_arith != "f64":
        lat.set_eos_arith(eos_arith)
    if field == "droplet":
        lat.init_droplet((edge / 2,) * 3, 40.0 * edge / 256, W_HEADLINE, rl, rv)
    else:
        lat.init_flat(2, edge / 4, 3 * edge / 4, W_FLAT, rl, rv)
    lat.step(warmup)
    stream = torch.cuda.current_stream()
    clk = Clocks(clocks_index) if clocks_index is not None else None
    times = []
    barrier(world)
    torch.cuda.synchronize()
    if clk:
        clk.__enter__()
    for _ in range(repeats):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier(world)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier(world)
        times.append(e0.elapsed_time(e1))
    if clk:
        clk.__exit__()
    status = lat.check()
    # kernel split, from a separate region with per-launch events
    lat.set_profiling(True)
    lat.kernel_times()
    lat.step(steps)
    kt = lat.kernel_times()
    lat.set_profiling(False)
    tuning = lat.tuning()
    lat.close()
    return {"ms": statistics.median(times), "region_ms": times, "kt": kt, "clocks": clk.summary() if clk else None,
            "status": status, "single_pass": tuning["single_pass"]}


def e2e_run(op, prec, edge, steps):
    """Through the C ABI with host buffers: H2D of the initial density, the steps, D2H of rho and u."""
    import torch

    lat, rl, rv = make_lattice(op, prec, edge)
    from paper_1805_08643_gb300.lbm import lib

    n = edge ** 3
    rho0 = torch.empty(n, dtype=torch.float64).pin_memory()
    # synthetic input: the same droplet as a host field (Eq. 59 profile from the seeded recipe)
    x = np.arange(edge, dtype=np.float64)
    d = np.minimum(np.abs(x - edge / 2), edge - np.abs(x - edge / 2))
    r = np.sqrt(d[None, None, :] ** 2 + d[None, :, None] ** 2 + d[:, None, None] ** 2)
    rho0.numpy()[:] = (0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2.0 * (r - 40.0 * edge / 256) / W_HEADLINE)).ravel()
    rho_out = torch.empty(n, dtype=torch.float64).pin_memory()
    u_out = torch.empty(3 * n, dtype=torch.float64).pin_memory()
    import ctypes

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = lib.lbm_init_field(lat.handle, ctypes.c_void_p(rho0.data_ptr()), 0, rv)
    st |= lib.lbm_step(lat.handle, steps)
    st |= lib.lbm_moments(lat.handle, ctypes.c_void_p(rho_out.data_ptr()), ctypes.c_void_p(u_out.data_ptr()), 0)
    t1 = time.perf_counter()
    lat.close()
    assert st == 0, "e2e C-ABI calls failed"
    return t1 - t0, 8 * n, 32 * n


def batched_run(steps, warmup, n_boxes=512, tuning=None):
    """The batched workload: n_boxes periodic boxes (edges 32/48/64/96, every edge even), stepped as the
    autotuner picks: the work list (one launch per step) or the two-pass pair kernels (a flat fused grid per
    operator, then the psi pass over work items: three launches per step).  tuning = (tile, z_planes) fixes the
    choice instead (no autotuning launches: for launch lists)."""
    import torch

    from paper_1805_08643_gb300 import synth, thermo, tune
    from paper_1805_08643_gb300.lbm import Batch, Rates

    specs = synth.batched_boxes(n_boxes)
    a = 0.25  # stable over T/T_c in [0.6, 0.9] with W = 5 and sigma = 0.105
    Tc = thermo.critical_temperature(a, B, R_GAS)
    batch = Batch("f32", "cs", hbm_budget_bytes=200 << 30)
    nodes = 0
    for k, sp in enumerate(specs):
        rl, rv = thermo.coexistence_cs(sp.T_over_Tc, a, B, R_GAS)
        box = batch.add((sp.edge,) * 3, "nonorth" if k % 2 == 0 else "orth", a=a, b=B, R=R_GAS,
                        T=sp.T_over_Tc * Tc, G=G, rates=Rates(**RATES), sigma=SIGMA_DROPLET)
        batch.init_droplet(box, (sp.edge / 2,) * 3, sp.radius, W_DROPLET, rl, rv)
        nodes += sp.edge ** 3
    if tuning is None:
        tile, zc, table = tune.tune_batch(batch)
    else:
        (tile, zc), table = tuning, {}
        for box in batch.grids:
            batch.set_tuning(tile, box, zc)
    steps += steps % 2
    batch.step(max(2, warmup + warmup % 2))
    stream = batch.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    stream.synchronize()
    e0.record(stream)
    batch.step(steps)
    e1.record(stream)
    stream.synchronize()
    ms = e0.elapsed_time(e1)
    status = batch.check()
    info = batch.info()
    batch.close()
    return {"mlups": nodes * steps / (ms / 1e3) / 1e6, "ms_per_step": ms / steps, "boxes": n_boxes, "nodes": nodes,
            "work_items": info["work_items"], "tile": tune.TILES[tile], "z_planes": zc,
            "step_gbs": (FUSED_BYTES["f32"] + PSI_BYTES["f32"]) * nodes / (ms / steps / 1e3) / 1e9,
            "bytes_per_lup": FUSED_BYTES["f32"] + PSI_BYTES["f32"],
            "tuning_ms_per_step": {f"{tune.TILES[t]}/z{z}": round(v, 3) for (t, z), v in table.items()},
            "operators": "alternating non-orthogonal / orthogonal", "status": status,
            "physics": "a=0.25, W=5, sigma=0.105, T/Tc~U[0.6,0.9], R~U[6,edge/3], FP32"}


def served_run(n_jobs=24, load=1.0, max_steps=20000, tol=1e-7):
    """The served workload, scaled down: Poisson droplet / slab jobs, edges U[48, 96], continuous batching."""
    from paper_1805_08643_gb300 import synth
    from paper_1805_08643_gb300.serve import BatchBackend, Server

    # offered load relative to a capacity estimate: GPU rate 20 GLUPS over jobs of mean edge^3 x max_steps
    mean_nodes = (96 ** 4 - 48 ** 4) / (4 * 48)
    capacity = 20e9 / (mean_nodes * max_steps)
    jobs = synth.job_stream(n_jobs, rate_per_s=load * capacity, edge_lo=48, edge_hi=96)
    be = BatchBackend("f32", hbm_budget_bytes=64 << 30)
    rep = Server(be, check_every=100, tol=tol, max_steps=max_steps, min_steps=200).run(jobs)
    be.close()
    out = rep.summary()
    out.update({"offered_jobs_per_s": load * capacity, "tol_max_du_per_100_steps": tol, "max_steps": max_steps,
                "workload": f"{n_jobs} jobs, edge U[48,96], droplet or slab, T/Tc U[0.6,0.9], "
                            "operator random, FP32, a=0.25, W=5"})
    return out


def serve_study(n_jobs=200, loads=(0.25, 0.5, 1.0, 1.5, 2.0), max_steps=100_000, tol=1e-8, pilot_jobs=32,
                capacity=None):
    """The served configuration: Poisson streams of droplet / slab jobs, box edges U[48, 192], T/T_c U[0.6, 0.9],
    random operator, FP32, run until max|du| < tol per 100 steps (converged) or max_steps (truncated, reported
    apart); offered rate swept as multiples of the measured service capacity.  Capacity: a pilot of
    `pilot_jobs` jobs of the same distribution (another seed), all present at the start, served to completion:
    jobs / wall time (or `capacity` jobs/s, from an earlier pilot).  Per rate: p50 / p99 arrival-to-convergence
    latency, truncated jobs, aggregate MLUPS."""
    from paper_1805_08643_gb300 import synth
    from paper_1805_08643_gb300.serve import BatchBackend, Server

    lo, hi = 48, 192
    budget = 96 << 30
    t0 = time.perf_counter()
    pilot_summary = None
    if capacity is None:
        pilot = synth.job_stream(pilot_jobs, rate_per_s=1e9, edge_lo=lo, edge_hi=hi, seed=synth.SEED + 1)
        be = BatchBackend("f32", hbm_budget_bytes=budget)
        prep = Server(be, check_every=100, tol=tol, max_steps=max_steps, min_steps=200).run(pilot)
        be.close()
        capacity = pilot_jobs / prep.wall_s
        pilot_summary = {"jobs": pilot_jobs, **prep.summary()}
    rows = []
    for load in loads:
        if n_jobs < 1:
            break
        jobs = synth.job_stream(n_jobs, rate_per_s=load * capacity, edge_lo=lo, edge_hi=hi)
        be = BatchBackend("f32", hbm_budget_bytes=budget)
        rep = Server(be, check_every=100, tol=tol, max_steps=max_steps, min_steps=200).run(jobs)
        be.close()
        rows.append({"load": load, "offered_jobs_per_s": load * capacity, **rep.summary()})
        print(json.dumps({"progress": rows[-1]}), file=sys.stderr, flush=True)
    return {"study": "serve", "jobs_per_rate": n_jobs, "edge": [lo, hi], "tol_max_du_per_100_steps": tol,
            "max_steps": max_steps, "capacity_jobs_per_s": capacity,
            "pilot": pilot_summary,
            "workload": "droplet or slab, T/Tc U[0.6,0.9], operator random, FP32, a=0.25, W=5, "
                        "sigma=0.105 (droplet) / 0.116 (slab)", "rates": rows,
            "seconds": time.perf_counter() - t0}


def precision_study(edge=512, steps=5000):
    """FP32 and FP16-storage forms against the FP64 form on the 27-droplet workload.

    512^3 box, 27 droplets on a jittered 3x3x3 lattice (R ~ U[12, 40], seed 1805),
    T = 0.6 T_c, a = 0.25 (a = 1 is unstable here), W = 5, sigma = 0.105, s_nu = 1.0,
    other rates 1.1, non-orthogonal operator.  Per form: density ratio (mean of the
    droplet-centre densities over the vapour median), Laplace Delta p of each droplet
    and the maximum spurious |u|, with errors relative to the FP64 run.
    """
    import torch

    from paper_1805_08643_gb300 import synth, thermo
    from paper_1805_08643_gb300.lbm import Lattice, Rates

    a = 0.25
    Tc = thermo.critical_temperature(a, B, R_GAS)
    T = 0.6 * Tc
    rl, rv = thermo.coexistence_cs(0.6, a, B, R_GAS)
    centres, radii = synth.random_droplets(box=edge)

    def p_eos(r):
        e = B * r / 4
        return r * R_GAS * T * (1 + e + e * e - e ** 3) / (1 - e) ** 3 - a * r * r

    out = {}
    for prec in ("f64", "f32", "f16"):
        lat = Lattice((edge,) * 3, operator="nonorth", precision=prec, a=a, T=T, G=G, rates=Rates(**RATES),
                      sigma=SIGMA_DROPLET)
        lat.init_droplets(centres, radii, W_DROPLET, rl, rv)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(steps)
        status = lat.check()
        t1 = time.perf_counter()
        rho, u = lat.moments()
        diag = lat.diag()
        lat.close()
        del lat
        torch.cuda.empty_cache()
        idx = np.rint(centres).astype(int) % edge
        rho_in = rho[idx[:, 2], idx[:, 1], idx[:, 0]]
        vap = rho[rho < 0.5 * (rl + rv)]
        rho_out = float(np.median(vap))
        umag = np.sqrt((u * u).sum(0))
        out[prec] = {"rho_in": rho_in, "rho_out": rho_out, "dp": p_eos(rho_in) - p_eos(rho_out),
                     "umax": float(umag.max()), "mass": diag["mass"], "seconds": t1 - t0,
                     "mlups": edge ** 3 * steps / (t1 - t0) / 1e6, "status": status}
        del rho, u, umag, vap
    ref = out["f64"]
    table = {}
    for prec, r in out.items():
        ratio = float(np.mean(r["rho_in"]) / r["rho_out"])
        ratio_ref = float(np.mean(ref["rho_in"]) / ref["rho_out"])
        dp_err = np.abs(r["dp"] - ref["dp"]) / np.abs(ref["dp"])
        table[prec] = {"density_ratio": ratio, "density_ratio_rel_err": abs(ratio / ratio_ref - 1),
                       "laplace_dp_rel_err_max": float(dp_err.max()), "laplace_dp_rel_err_mean": float(dp_err.mean()),
                       "max_spurious_u": r["umax"], "max_spurious_u_abs_err": abs(r["umax"] - ref["umax"]),
                       "rel_mass_vs_fp64": r["mass"] / ref["mass"] - 1, "seconds": r["seconds"],
                       "mlups": r["mlups"], "status": r["status"]}
    return {"study": "precision", "edge": edge, "steps": steps, "droplets": len(radii),
            "physics": "T=0.6Tc, a=0.25, W=5, sigma=0.105, s_nu=1.0, other rates 1.1, non-orthogonal",
            "forms": table}


def lattice_name(op):
    return "D3Q15" if op == "nonorth_d3q15" else "D3Q19"


def workload_text(op, prec, edge):
    """The headline workload, named by what it is (shared by both arms)."""
    op_text = {"nonorth": "non-orthogonal", "orth": "orthogonal", "nonorth_d3q15": "non-orthogonal"}[op]
    return (f"{lattice_name(op)} {op_text} MRT + CS pseudopotential, {edge}^3 periodic box, "
            f"droplet R={40.0 * edge / 256:g} W={W_HEADLINE:g}, T=0.7Tc, sigma=0.105 (Eq. 16), {PREC_TEXT[prec]}")


def oracle_for(op):
    """The oracle module of the operator's lattice and the operator name its Params take."""
    if op == "nonorth_d3q15":
        from oracle import d3q15 as D

        return D, "nonorth"
    from oracle import lbm_oracle as L

    return L, op


def oracle_slab(op, nz, edge=EDGE, z0=None):
    """Oracle state of the nz planes [z0, z0 + nz) of the edge^3 droplet box (default: through its centre),
    run as a box of its own (periodic in z): a timing sample whose work per node is the full box's."""
    from oracle import lbm_oracle as L
    from oracle import maxwell

    O, oop = oracle_for(op)
    Tc = L.critical_temperature(A, B, R_GAS)
    rl, rv = maxwell.coexistence_cs(T_OVER_TC, A, B, R_GAS)
    p = L.Params(grid=(edge, edge, nz), operator=oop, a=A, b=B, R=R_GAS, T=T_OVER_TC * Tc, G=G,
                 sigma=SIGMA_DROPLET, **RATES)
    if z0 is None:
        z0 = edge // 2 - nz // 2
    rho = slab_density(edge, z0, nz, 40.0 * edge / 256, W_HEADLINE, rl, rv)
    return O, p, O.equilibrium_state(p, rho)


def slab_density(edge, z0, nz, R, W, rl, rv):
    """Planes [z0, z0 + nz) of the Eq. 59 droplet centred in the edge^3 box (periodic minimum-image
    distances over the full box), computed for the slab alone (no full-box array)."""
    c = edge / 2

    def d(v):
        a = np.abs(v - c)
        return np.minimum(a, edge - a)

    x = d(np.arange(edge, dtype=np.float64))
    z = d(np.arange(z0, z0 + nz, dtype=np.float64))
    r = np.sqrt(z[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2)
    return 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2.0 * (r - R) / W)


def _oracle_job(job):
    """One CPU-baseline task (in a spawned process): build its oracle state, time `steps` steps of it."""
    kind, op, edge, nz, z0, steps = job
    if kind == "parity":  # the 32^3 parity workload: T = 0.8 T_c, droplet R = 8, W = 2, no Eq. 16 term
        from oracle import lbm_oracle as L
        from oracle import maxwell

        O, oop = oracle_for(op)
        Tc = L.critical_temperature(A, B, R_GAS)
        rl, rv = maxwell.coexistence_cs(0.8, A, B, R_GAS)
        p = L.Params(grid=(edge,) * 3, operator=oop, a=A, b=B, R=R_GAS, T=0.8 * Tc, G=G, s_e=1.1, s_nu=1.0,
                     s_q=1.1, s_pi=1.1, s_eps=1.1, s_m=1.1)
        f = O.equilibrium_state(p, L.droplet_density((edge,) * 3, (edge / 2,) * 3, 8.0, 2.0, rl, rv))
        nodes = edge ** 3
    else:
        O, p, f = oracle_slab(op, nz, edge, z0)
        nodes = edge * edge * nz
    t0 = time.perf_counter()
    for _ in range(steps):
        f = O.step(p, f)
    return nodes * steps, time.perf_counter() - t0


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(op=None):
    """The FP64 oracle, as it stands (single-threaded numpy per process), on the host's cores.

    Samples (about 15-20 s of CPU work on 16 Grace cores):
      * all cores, 256^3 x 10 steps: as many nodes as the whole headline box, as `cores` copies of the
        256 x 256 x (256 / cores) slab through the droplet centre, one process each (the line's value);
      * all cores, 512^3 x 2 steps: the same at 512^3 (R = 80), 4 x `cores` copies of a centre slab of 8 planes;
      * all cores, 32^3 x 200 steps: the parity workload, one full copy per process;
      * one core: 256 x 256 x 8 slab through the droplet centre, 3 steps.
    A slab runs as a periodic box of its own, so its work per node is the full box's; centred on the
    droplet, its periodic seam joins two planes at about the same distance from the centre (slabs cut
    elsewhere would join liquid to vapour across the seam and leave the EOS domain within steps).
    Processes are spawned (no fork after CUDA initialisation)."""
    import multiprocessing as mp

    op = op or HEADLINE[0]
    cores = cpu_cores()
    ctx = mp.get_context("spawn")
    out = {}

    def run(name, jobs, procs, what):
        t0 = time.perf_counter()
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_job, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        lups = sum(r[0] for r in res)
        out[name] = {"value": lups / wall / 1e6, "unit": UNIT, "cores": procs, "seconds": wall, "sample": what}

    n256 = max(1, min(cores, EDGE))
    nz256 = EDGE // n256
    run("256^3x10", [("slab", op, EDGE, nz256, None, 10) for _ in range(n256)], n256,
        f"{EDGE}^3 nodes x 10 FP64 oracle steps: {n256} copies of the periodic {EDGE}x{EDGE}x{nz256} slab through "
        f"the droplet centre, in {n256} spawned processes")
    n512 = 4 * n256
    run("512^3x2", [("slab", op, 512, 512 // n512, None, 2) for _ in range(n512)], n256,
        f"512^3 nodes x 2 FP64 oracle steps: {n512} copies of the periodic 512x512x{512 // n512} slab through the "
        f"centre of the 512^3 droplet box (R=80), on {n256} processes")
    run("32^3x200", [("parity", op, 32, 32, 0, 200) for _ in range(n256)], n256,
        f"the 32^3 parity workload (T=0.8Tc, R=8, W=2), 200 FP64 oracle steps, one full copy per process, "
        f"{n256} processes")
    run("1core", [("slab", op, EDGE, 8, None, 3)], 1,
        f"{EDGE}x{EDGE}x8 slab through the droplet centre, 3 FP64 oracle steps, one process")
    head = out["256^3x10"]
    return {"value": head["value"], "unit": UNIT, "cores": head["cores"], "kind": "oracle",
            "sample": head["sample"] + f" ({lattice_name(op)} {op} operator, single-threaded numpy per process)",
            "samples": out}


class _SlabWorker:
    """A spawned process that holds one oracle slab and steps it on request (reference arm)."""

    def __init__(self, ctx, op, nz, z0):
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_slab_worker_main, args=(child, op, nz, z0), daemon=True)
        self.proc.start()

    def close(self):
        try:
            self.conn.send(None)
        except Exception:
            pass
        self.proc.join(timeout=30)


def _slab_worker_main(conn, op, nz, z0):
    O, p, f = oracle_slab(op, nz, EDGE, z0)
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg is None:
            return
        f = O.step(p, f)
        conn.send(1)


def reference_arm(args, world, rank):
    """The oracle on the host cores, on this benchmark's workload: every step, one FP64 oracle step of
    `cores` periodic z-slabs of 256 x 256 x 2 around the droplet centre, one spawned process each."""
    if rank != 0:
        return
    import multiprocessing as mp

    cores = cpu_cores()
    nz = 2
    ctx = mp.get_context("spawn")
    z_lo = EDGE // 2 - cores * nz // 2
    workers = [_SlabWorker(ctx, args.op, nz, max(0, z_lo + k * nz) % (EDGE - nz + 1)) for k in range(cores)]
    try:
        for w in workers:
            assert w.conn.recv() == "ready"

        def step():
            for w in workers:
                w.conn.send(1)
            for w in workers:
                w.conn.recv()

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        dt = time.perf_counter() - t0
    finally:
        for w in workers:
            w.close()
    nodes = EDGE * EDGE * nz * cores
    v = nodes * args.steps / dt / 1e6
    sample = (f"each step: one FP64 oracle step (numpy, as it stands) of each of {cores} periodic "
              f"{EDGE}x{EDGE}x{nz} z-slabs of the {EDGE}^3 droplet box, one spawned process per core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": reference_workload_text(args.op, cores, nz), "edge": EDGE,
                                        "operator": args.op, "precision": "f64", "parallelism": f"{cores} host processes"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def reference_workload_text(op, cores, nz):
    op_text = {"nonorth": "non-orthogonal", "orth": "orthogonal", "nonorth_d3q15": "non-orthogonal"}[op]
    return (f"{lattice_name(op)} {op_text} MRT + CS pseudopotential, droplet R=40 W=3 of the {EDGE}^3 periodic box, "
            f"T=0.7Tc, sigma=0.105 (Eq. 16); the FP64 oracle on {cores} z-slabs of {EDGE}x{EDGE}x{nz} per step "
            f"(FP64 compute and storage)")


def form_entry(op, prec, edge, steps, warmup, world, hbm_peak, mode="default", field="droplet", eos_arith="f64",
               repeats=3):
    """One line of the `forms` object: throughput, whole-step bandwidth against the minimum bytes per update,
    and the kernel split."""
    r = time_form(op, prec, edge, steps, warmup, world, field=field, mode=mode, eos_arith=eos_arith, repeats=repeats)
    n = edge ** 3
    q15 = op == "nonorth_d3q15"
    fb = (FUSED_BYTES_Q15 if q15 else FUSED_BYTES)[prec]
    pb = (PSI_BYTES_Q15 if q15 else PSI_BYTES)[prec]
    smin = (STEP_MIN_BYTES_Q15 if q15 else STEP_MIN_BYTES)[prec]
    ms_step = r["ms"] / steps
    kt = r["kt"]
    f_ms = kt["fused_ms"] / max(kt["fused_launches"], 1)
    e = {"mlups": n * steps / (r["ms"] / 1e3) / 1e6, "ms_per_step": ms_step,
         "step": "work-list single pass (one launch)" if r["single_pass"] == "queue" else
                 ("two-pass (psi pass + fused pass)" if not r["single_pass"] else f"single pass ({r['single_pass']})"),
         "bytes_per_lup_min": smin, "whole_step_gbs_at_min_bytes": smin * n / (ms_step / 1e3) / 1e9,
         "whole_step_frac_of_hbm": smin * n / (ms_step / 1e3) / 1e9 / hbm_peak, "status": r["status"]}
    if not r["single_pass"]:
        p_ms = kt["psi_ms"] / max(kt["psi_launches"], 1)
        e.update({"fused_ms": f_ms, "psi_ms": p_ms, "fused_gbs": fb * n / (f_ms / 1e3) / 1e9,
                  "hbm_frac_fused": fb * n / (f_ms / 1e3) / 1e9 / hbm_peak, "bytes_per_lup_two_pass": fb + pb})
    if prec == "f64" and op in FUSED_FP64_INSTR:
        e["fp64_alu_frac_fused"] = FUSED_FP64_INSTR[op] * n / (f_ms / 1e3) / 1e9 / FP64_PEAK_GINSTR
    if eos_arith != "f64":
        e["note"] = "EOS radicand in compensated FP32 pairs instead of FP64"
    return e


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--repeats", type=int, default=5, help="timed regions of --steps steps; the median is reported")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--edge", type=int, default=EDGE)
    ap.add_argument("--op", default=HEADLINE[0], choices=["nonorth", "orth", "nonorth_d3q15"])
    ap.add_argument("--prec", default=HEADLINE[1], choices=["f64", "f32", "f16"])
    ap.add_argument("--mode", default="default", choices=sorted(MODES),
                    help="step kernels: the library default (work-list single pass for FP32 storage, two-pass "
                         "otherwise), or one of the lbm_set_tuning modes")
    ap.add_argument("--forms", default="all",
                    help="'all', 'headline', 'batched' (headline + batched + served) or 'batch' (headline + batched)")
    ap.add_argument("--batch-boxes", type=int, default=512, help="boxes of the batched form")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--eos-arith", default="f64", choices=["f64", "f32x2"],
                    help="EOS radicand arithmetic of the psi pass (FP32 / FP16 forms)")
    ap.add_argument("--study", default=None, choices=["precision", "serve"],
                    help="run a study instead of the benchmark line (minutes)")
    ap.add_argument("--study-steps", type=int, default=5000)
    ap.add_argument("--serve-jobs", type=int, default=200, help="jobs per offered rate of --study serve")
    ap.add_argument("--batch-tuning", default=None,
                    help="TILE,Z: fixed step kind and z planes of the batched form (default: autotuned)")
    ap.add_argument("--serve-capacity", type=float, default=None,
                    help="service capacity (jobs/s) of --study serve; default: measure it with a pilot")
    ap.add_argument("--serve-loads", default="0.25,0.5,1,1.5,2",
                    help="offered rates of --study serve, as multiples of the measured capacity")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    args.repeats = max(1, args.repeats)
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return

    import torch

    from __graft_entry__ import build

    build()
    torch.cuda.set_device(local)
    if args.study == "precision":
        if rank == 0:
            print(json.dumps(precision_study(args.edge if args.edge != EDGE else 512, args.study_steps)))
        return
    if args.study == "serve":
        if rank == 0:
            print(json.dumps(serve_study(n_jobs=args.serve_jobs,
                                         loads=tuple(float(v) for v in args.serve_loads.split(",")),
                                         capacity=args.serve_capacity)))
        return
    n = args.edge ** 3
    hbm_peak, peak_kind = peaks()

    op, prec = args.op, args.prec
    r = time_form(op, prec, args.edge, args.steps, args.warmup, world, clocks_index=local, mode=args.mode,
                  eos_arith=args.eos_arith, repeats=args.repeats)
    ms = max_over_ranks(r["ms"], world)  # median region of this rank, max over ranks
    ms_step = ms / args.steps
    value = sum_over_ranks(n * args.steps / (ms / 1e3) / 1e6, world)  # all ranks' nodes / max time
    kt = r["kt"]
    fused_ms = kt["fused_ms"] / max(kt["fused_launches"], 1)
    psi_ms = kt["psi_ms"] / max(kt["psi_launches"], 1)
    q15 = op == "nonorth_d3q15"
    smin = (STEP_MIN_BYTES_Q15 if q15 else STEP_MIN_BYTES)[prec]
    single = r["single_pass"]

    if prec == "f64" and op in FUSED_FP64_INSTR:
        ach = FUSED_FP64_INSTR[op] * n / (fused_ms / 1e3) / 1e9
        roofline = {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_GINSTR, "unit": "G FP64 instr/s",
                    "frac": ach / FP64_PEAK_GINSTR, "traffic": None,
                    "peak_kind": "derived: 2 FP64/SM/clk x 152 x 2070 MHz",
                    "kernel": "fused force+collide+stream", "fp64_instr_per_node": FUSED_FP64_INSTR[op],
                    "fused_ms": fused_ms, "psi_ms": psi_ms}
        launches = 2 * args.steps
    elif single == "queue":
        # one launch per step: the kernel's average launch duration is the step time
        achieved = smin * n / (ms_step / 1e3) / 1e9
        dram = QUEUE_DRAM_BYTES.get((op, prec)) if args.edge == EDGE else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": dram * n if dram else None, "peak_kind": peak_kind,
                    "kernel": "work-list single pass (fused pass + next step's psi pass, one launch per step)",
                    "bytes_per_node": smin, "kernel_ms": ms_step,
                    "kernel_ms_profiled": fused_ms}
        launches = args.steps
    else:
        fused_bytes = (FUSED_BYTES_Q15 if q15 else FUSED_BYTES)[prec]
        achieved = fused_bytes * n / (fused_ms / 1e3) / 1e9
        dram = FUSED_DRAM_BYTES.get((op, prec)) if args.edge == EDGE and not single else None
        roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                    "frac": achieved / hbm_peak, "traffic": dram * n if dram else None, "peak_kind": peak_kind,
                    "kernel": f"single pass ({single})" if single else "fused force+collide+stream",
                    "bytes_per_node": fused_bytes, "fused_ms": fused_ms, "psi_ms": psi_ms}
        launches = args.steps if single else 2 * args.steps
    whole = {"bytes_per_lup_min": smin, "gbs_at_min_bytes": smin * n / (ms_step / 1e3) / 1e9,
             "frac_of_hbm": smin * n / (ms_step / 1e3) / 1e9 / hbm_peak}

    forms = {}
    if args.forms == "all":
        E = args.edge
        K, W = args.steps, args.warmup
        k64 = max(10, K // 8)
        for fop in ("nonorth", "orth"):
            for fprec in ("f64", "f32", "f16"):
                forms[f"{fop}_{fprec}_droplet"] = form_entry(fop, fprec, E, k64 if fprec == "f64" else K, W, world,
                                                             hbm_peak)
            forms[f"{fop}_f32_droplet_two_pass"] = form_entry(fop, "f32", E, K, W, world, hbm_peak, mode="two-pass")
        for fprec in ("f64", "f32", "f16"):
            forms[f"nonorth_d3q15_{fprec}_droplet"] = form_entry("nonorth_d3q15", fprec, E, k64 if fprec == "f64" else K,
                                                                 W, world, hbm_peak)
        for fprec in ("f32", "f16"):
            forms[f"nonorth_{fprec}_droplet_eos_f32x2"] = form_entry("nonorth", fprec, E, K, W, world, hbm_peak,
                                                                     eos_arith="f32x2")
        for fprec in ("f64", "f32"):
            forms[f"nonorth_{fprec}_flat"] = form_entry("nonorth", fprec, E, k64 if fprec == "f64" else K, W, world,
                                                        hbm_peak, field="flat")

    if args.forms in ("all", "batched", "batch"):
        bt = tuple(int(v) for v in args.batch_tuning.split(",")) if args.batch_tuning else None
        forms[f"batched_{args.batch_boxes}"] = batched_run(args.steps, args.warmup, args.batch_boxes, bt)
    if args.forms in ("all", "batched"):
        forms["served"] = served_run()

    e2e = None
    if not args.no_e2e:
        e2e_steps = args.steps
        t_e2e, h2d, d2h = e2e_run(op, prec, args.edge, e2e_steps)
        e2e = {"value": sum_over_ranks(n * e2e_steps / max_over_ranks(t_e2e, world) / 1e6, world), "unit": UNIT,
               "h2d_bytes_per_step": h2d / e2e_steps, "d2h_bytes_per_step": d2h / e2e_steps,
               "note": "lbm_init_field from pinned host rho, lbm_step(K), lbm_moments to pinned host"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(op)

    if rank != 0:
        return
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == "f64" else "f32", "data": "synthetic",
        "config": {"workload": workload_text(op, prec, args.edge),
                   "edge": args.edge, "operator": op, "precision": prec,
                   "step": "work-list single pass" if single == "queue" else (f"single pass ({single})" if single
                                                                            else "two-pass"),
                   "parallelism": f"replicas{world}" if world > 1 else "single",
                   "l2": f"inputs larger than L2 (populations {(15 if q15 else 19) * n * {'f64': 8, 'f32': 4, 'f16': 2}[prec] / 1e9:.2f} GB per buffer)"},
        "timing": f"median of {args.repeats} regions of {args.steps} steps (CUDA events on the launch stream, "
                  f"barrier + synchronize around each); kernel split from a separate region",
        "region_ms": r["region_ms"],
        "roofline": roofline,
        "whole_step": whole,
        "clocks": r["clocks"],
        "e2e": e2e,
        "gpu_launches": launches,
        "forms": forms,
        "status": r["status"],
    }
    if cpu:
        out["cpu_baseline"] = cpu
    print(json.dumps(out))


if __name__ == "__main__":
    main()
