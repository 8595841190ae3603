"""Throughput of the EAM hot path on one GB300 (atom-steps/s), with its roofline.

Headline workload: fcc Cu 50x50x50 cells = 500,000 atoms, Sutton-Chen EAM as 5,000-knot
cubic tables (cutoff 2a), 300 K seeded velocities, velocity-Verlet NVE with dt = 2 fs, a
0.3 Å skin and a list rebuild whenever an atom has moved more than skin/2.  One step is the
whole path: half kick + drift + skin check, [link-cell binning, sort, list build], density
pass, force pass + half kick.  All steps of one md_step call run in one persistent launch.
The headline is the FP64 path (the paper's arithmetic), with its roofline against the FP64
FMA rate measured in the same run by the library's own FMA-chain kernel; the mixed path (FP32
pair/density terms, FP64 positions, integration, density sum and reductions) is reported in
the same line as its speedup over FP64 at its stated force error and NVE drift.  The other
workloads print one line each ("extra <name>: {...}") before the headline line: bcc Fe 2,000
atoms (FP64), 256 bcc Fe replicas of 2,000-54,000 atoms in one batch under a captured CUDA
graph, bcc Fe-C 4.2M atoms with a z strain ramp, the table-versus-explicit potential
comparison, the neighbour walks, and the learned surrogate on 1,024,000-atom bcc Fe next to
FP64 and mixed EAM (force RMSE, ms per step, NVE drift); a summary of the surrogate line is
carried in the headline line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]
  python bench.py --surrogate-only            # the surrogate comparison alone
  python bench.py --profile-case --cells 40   # short mixed-EAM run for ncu captures
  python bench.py --surrogate-profile bf16    # short surrogate run for ncu captures

Under torchrun each rank advances its own replica (different seed) on its own GPU; there is
no exchange on the data path (replicas only); timings are reduced with a max over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
import argparse
import ctypes as C
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1107_2619_gb300 import inputs as I  # noqa: E402

METRIC = "atom-steps/s (EAM force+integrate, 1 GB300) & HBM roofline fraction; surrogate speedup at force err"
UNIT = "atom-steps/s"
CELLS = 50
SEED = 2
WORKLOAD = ("fcc Cu 50x50x50 cells = 500,000 atoms, Sutton-Chen EAM as 5,000-knot cubic tables "
            "(cutoff 2a, shifted force), 300 K, NVE velocity Verlet dt = 2 fs, skin 0.3 Å")


def _config(precision, cells=CELLS):
    return {"workload": WORKLOAD, "n_atoms": 4 * cells ** 3, "precision": precision, "seed": SEED,
            "rebuild": "when an atom moved > skin/2 (checked every step)",
            "l2": "inputs larger than L2: the neighbour list alone is 4 B x 140 x 500k = 280 MB per pass"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


# FP64 operations per list entry of the FP64 passes, counted from the pair code (an add or a
# multiply is 1 flop, an FMA 2; conversions and rounding to integer not counted).  Entries
# inside r_cut: density 35 (separation 3, r^2 5, FP64 refinement of the reciprocal square root 6,
# r 1, knot index 3, the cubic of phi 6, the sum 1, the derivative cubics of phi and V 8, their
# scaling by 1/r 2) + force 12 (separation 3, the pair scalar from the cached derivatives 3, the
# force 6).  Entries in the skin shell: 8 in the density pass (up to r^2), and the force pass's 12
# on zero terms.  The half list takes each pair once: half of these per list entry.
FP64_FLOP_IN, FP64_FLOP_SHELL = 47.0, 20.0


def fp64_flop_per_step(sum_counts, w):
    """FP64 flop of one step of the FP64 passes by the per-entry model above; the share of list
    entries inside r_cut is taken as (r_cut / r_list)^3 (uniform density)."""
    rc = float(w.potential.r_cut)
    f_in = (rc / (rc + w.skin)) ** 3
    return sum_counts * (f_in * FP64_FLOP_IN + (1.0 - f_in) * FP64_FLOP_SHELL)


def fp64_peak(md, stream, repeats=3, iters=5000):
    """Best of `repeats` runs of the library's FP64 FMA-chain kernel (md_measure_fp64_peak)."""
    return max(md.md_measure_fp64_peak(iters, stream)[0] for _ in range(repeats))


def _capture(kernel):
    """The committed ncu record of a kernel (profiles/traffic.json) if its sources are unchanged
    since the capture; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)[kernel]
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as fh:
                h.update(fh.read())
        return rec if h.hexdigest() == rec["sha256"] else None
    except Exception:
        return None


def _traffic(kernel, n_atoms, n_steps):
    """DRAM bytes per launch from the committed ncu capture (per atom-step, scaled to this launch)."""
    rec = _capture(kernel)
    return None if rec is None else float(rec["bytes_per_atom_step"]) * n_atoms * n_steps


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, name in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_max(dist, x, device):
    """Max of a float over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(atoms_per_rank, world, steps, ms):
    """Whole-job throughput: the atoms of all ranks x steps / the slowest rank's time."""
    return world * atoms_per_rank * steps / (ms * 1e-3)


def _oracle_rate(n_cells, steps, warmup=0):
    """Oracle atom-steps/s on an fcc Cu cube of n_cells^3 cells (same potential, temperature,
    time step and skin as the benchmark workload): velocity Verlet with the link-cell list."""
    import oracle
    w = I.fcc_cu(n_cells, seed=SEED)
    ref = oracle.forces(w.pos, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max)
    pos, vel, force = w.pos, w.vel, ref["force"]
    if warmup:
        r = oracle.run_vv(pos, vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, warmup,
                          w.skin, w.k_max, force=force)
        pos, vel, force = r["pos"], r["vel"], r["force"]
    t0 = time.perf_counter()
    oracle.run_vv(pos, vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, steps, w.skin,
                  w.k_max, force=force)
    dt = time.perf_counter() - t0
    return w.n_atoms * steps / dt, dt, w.n_atoms, oracle.num_threads()


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from oracle import build as obuild
    obuild.build()
    n_cells = 20  # 32,000 atoms per step sample: the oracle's per-atom cost does not depend on N
    steps = max(1, args.steps)
    value, dt, n, cores = _oracle_rate(n_cells, steps, warmup=args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": _config("fp64 (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: one velocity-Verlet step of an fcc Cu {n_cells}^3-cell "
                                       f"sample ({n} atoms) of the workload; {steps} timed steps after "
                                       f"{args.warmup} warm-up steps, one list build included"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def step_bytes(n, sum_counts, precision):
    """Algorithmic HBM bytes of one step (no rebuild) by the per-atom-step model of the hot-path
    scope (neighbour gathers counted as L2 hits: atoms are in cell order), 8K + 170 for the
    mixed path and 8K + 184 for FP64, K list entries per atom:
      FP64:  list 2 x 4K + own position 2 x 24 + F' write and read 16 + force 24 + velocity
             Verlet position and velocity read and write 96;
      mixed: list 2 x 4K + the FP32 copy (16 written, 2 x 16 read) in place of the own
             positions + F' 16 + force 12 + velocity Verlet 96 ... = 8K + 170.
    The state the kernel actually moves is padded (double4 and float4 records), so its DRAM
    traffic (ncu) runs above this model."""
    per_atom = 170 if precision == "mixed" else 184
    total = 8 * sum_counts + per_atom * n
    return total, 4 * sum_counts + 0.5 * per_atom * n, 4 * sum_counts + 0.5 * per_atom * n


REBUILD_PARTS = ("bin", "tile_sums", "top_scan", "apply", "scatter", "cell_sort", "gather", "copyback", "list")


def rebuild_parts(prof):
    """Sub-phase times of a list rebuild (ms per rebuild) from a profiled run's stamps."""
    nr = max(1, int(prof.get("rebuilds", 0)))
    return {name: prof["ms_rebuild_part"][q] / nr for q, name in enumerate(REBUILD_PARTS)} | {"rebuilds": nr}


def _time_steps(torch, s, stream, k, barrier, clocks_index=None):
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    clk = None
    if clocks_index is not None:
        clk = Clocks(clocks_index).__enter__()
    start.record(stream)
    s.step(k)
    end.record(stream)
    end.synchronize()
    if clk is not None:
        clk.__exit__(None, None, None)
    barrier()
    return start.elapsed_time(end), (clk.summary() if clk is not None else None)


def run_ours(args):
    import torch
    import __graft_entry__ as entry
    from paper_1107_2619_gb300 import md

    world, rank, local = _dist()
    entry.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if dist.is_nccl_available() else "gloo")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return reduce_max(dist, x, "cuda")

    w = I.fcc_cu(args.cells, seed=SEED + rank)
    n = w.n_atoms
    stream = torch.cuda.Stream()
    res, snapshot = {}, {}
    # (label, precision, neighbour walk): FP64 is timed with the full list (each pair from both
    # sides) and with the half list (each pair once, FP64 atomics); the faster is the headline
    legs = {"mixed": ("mixed", args.passes), "fp64": ("fp64", "auto"), "fp64_half": ("fp64", "half"),
            "df": ("df", "auto")}
    if args.profile_case:
        legs = {args.profile_precision: (args.profile_precision.replace("_half", ""),
                                         "half" if args.profile_precision.endswith("_half") else args.passes)}
    for precision, (prec, walk) in legs.items():
        s = md.System(w, precision=prec, stream=stream.cuda_stream, device_inputs=True,
                      passes=walk, lanes_per_atom=args.lanes)
        s.eam_forces()
        lanes = args.lanes or s.tune()
        counts = s.get(md.MD_GET_NBR_COUNT)
        s.step(args.warmup)
        e0 = s.energy()
        launches0 = s.profile()["launches"]
        ms, clocks = _time_steps(torch, s, stream, args.steps, barrier, local)
        ms = max_over_ranks(ms)
        launches = s.profile()["launches"] - launches0
        e1 = s.energy()
        # phase breakdown: a second, profiled run (stamps at phase boundaries), at most 200 steps
        s.set_profiling(True)
        s.step(min(args.steps, 200))
        prof = s.profile()
        s.set_profiling(False)
        prof["rebuilds"] = s.energy()["n_rebuilds"] - e1["n_rebuilds"]
        res[precision] = dict(ms=ms, prof=prof, e0=e0, e1=e1, counts=counts, clocks=clocks,
                              launches=launches, lanes=lanes)
        if args.profile_case:
            pass
        elif precision == "mixed":
            snapshot["pos"] = s.positions()
            snapshot["mixed"] = s.forces()
        else:  # forces of every precision at the same thermalised positions
            s.set_state(pos=snapshot["pos"])
            s.eam_forces()
            snapshot[precision] = s.forces()
        s.close()
    if args.profile_case:
        if rank == 0:
            r = res[args.profile_precision]
            print(json.dumps({"profile_case": True, "precision": args.profile_precision,
                              "list_entries": float(r["counts"].sum()), "n_atoms": n, "ms_per_step": r["ms"] / args.steps,
                              "lanes": r["lanes"], "passes": args.passes, "rebuild_ms_per_rebuild": rebuild_parts(r["prof"]),
                              "phase_ms": {k: r["prof"]["ms_" + k] / max(1, r["prof"]["n_" + k])
                                           for k in ("kick", "rebuild", "density", "force")}}))
        return 0

    # FP64 FMA rate of this GPU (the denominator of the FP64 path's roofline), measured now
    fp64_tflops = fp64_peak(md, stream.cuda_stream)
    fp64_leg = "fp64_half" if res["fp64_half"]["ms"] < res["fp64"]["ms"] else "fp64"

    # end to end through the C ABI with host buffers (FP64 path): state in, one step, state and
    # energies out
    pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
    hp, hv, hf = pin((n, 3)), pin((n, 3)), pin((n, 3))
    s = md.System(w, precision="fp64", lanes_per_atom=res[fp64_leg]["lanes"], passes=legs[fp64_leg][1])
    s.eam_forces()
    s.get(md.MD_GET_POS, hp), s.get(md.MD_GET_VEL, hv), s.get(md.MD_GET_FORCE, hf)
    k_e2e = max(3, min(args.steps, 100))
    for _ in range(3):
        s.step_io(1, hp, hv, hf, hp, hv, hf)
    barrier()
    t0 = time.perf_counter()
    for _ in range(k_e2e):
        s.step_io(1, hp, hv, hf, hp, hv, hf)
    t = max_over_ranks(time.perf_counter() - t0)
    s.close()
    e2e = {"value": world * n * k_e2e / t, "unit": UNIT, "h2d_bytes_per_step": 72 * n,
           "d2h_bytes_per_step": 72 * n + C.sizeof(md.md_energies), "steps": k_e2e,
           "note": "FP64 path (the headline's walk); each step one md_step_io call: positions, velocities "
                   "and forces in from pinned host buffers, md_step(1), the three arrays back into them and "
                   "the energies, one synchronisation; the device reads and writes the pinned buffers "
                   "directly over the host link (caller order, in the sort kernels)"}

    extras = {}
    if not args.no_extras:
        try:
            extras = run_extras(torch, md, stream, barrier, max_over_ranks, world)
        except Exception as exc:  # an extra leg must not hide the headline line
            extras = {"error": f"{type(exc).__name__}: {exc}"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    hbm_peak, peak_src = _peaks()
    sum_counts = float(res["fp64"]["counts"].sum())

    def phases(q):
        p = q["prof"]
        return {k: round(p["ms_" + k] / max(1, p["n_" + k]), 4) for k in ("kick", "rebuild", "density", "force")}

    def hbm(q, precision):
        b = step_bytes(n, sum_counts, precision)[0] * args.steps
        a = b / (q["ms"] * 1e-3) / 1e9
        return {"achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak,
                "model": "8K + 170 B per atom-step" if precision == "mixed" else "8K + 184 B per atom-step",
                "traffic": _traffic("k_step_" + precision, n, args.steps), "peak_source": peak_src}

    r64, r32 = res[fp64_leg], res["mixed"]
    flop = fp64_flop_per_step(sum_counts, w) * args.steps * (0.5 if fp64_leg == "fp64_half" else 1.0)
    achieved = flop / (r64["ms"] * 1e-3) / 1e12
    f64, f32 = snapshot[fp64_leg], snapshot["mixed"]
    ferr = np.abs(f32 - f64)
    cpu = None
    if world == 1:
        try:
            from oracle import build as obuild
            obuild.build()
            v, dt, na, cores = _oracle_rate(20, 60)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"60 velocity-Verlet steps of an fcc Cu 20^3-cell sample ({na} atoms, same "
                             f"potential, temperature, dt and skin; one link-cell list build included), "
                             f"{dt:.1f} s on {cores} OpenMP threads"}
        except Exception as exc:  # the CPU leg must not hide the GPU line
            cpu = {"value": None, "unit": UNIT, "cores": None, "kind": "oracle", "sample": f"failed: {exc}"}

    mixed = {"value": job_value(n, world, args.steps, r32["ms"]), "ms_per_step": r32["ms"] / args.steps,
             "dtype": "f32+f64", "speedup_vs_fp64": r64["ms"] / r32["ms"],
             "force_err_vs_fp64_ev_per_a": {"max": float(ferr.max()), "rms": float(np.sqrt((ferr ** 2).mean())),
                                            "max_force": float(np.abs(f64).max())},
             "nve_drift_ev_per_atom": (r32["e1"]["te"] - r32["e0"]["te"]) / n,
             "lanes_per_atom": r32["lanes"], "phase_ms": phases(r32), "roofline": hbm(r32, "mixed")}
    rdf = res["df"]
    fdf = np.abs(snapshot["df"] - f64)
    df_line = {"value": job_value(n, world, args.steps, rdf["ms"]), "ms_per_step": rdf["ms"] / args.steps,
               "dtype": "f32x2 (double-float pair and density terms) + f64",
               "speedup_vs_fp64": r64["ms"] / rdf["ms"],
               "force_err_vs_fp64_rel_maxnorm": float(fdf.max() / np.abs(f64).max()),
               "nve_drift_ev_per_atom": (rdf["e1"]["te"] - rdf["e0"]["te"]) / n,
               "lanes_per_atom": rdf["lanes"], "phase_ms": phases(rdf)}
    line = {
        "metric": METRIC, "value": job_value(n, world, args.steps, r64["ms"]), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r64["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(_config("fp64: every sum, the integration and every reduction in FP64; the pair terms in FP64 "
                               "arithmetic, 1/r and r^2 formed from exact FP32 pieces to <= 4e-13 relative"),
                       fp64_walk=("half list: each pair once, the neighbour's share by FP64 atomics"
                                  if fp64_leg == "fp64_half" else "full list: each pair from both sides")),
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_tflops, "unit": "TFLOP/s",
                     "frac": achieved / fp64_tflops, "traffic": _traffic("k_step_fp64", n, args.steps),
                     "kernel": "k_step (persistent: all phases of the K steps, stopping at each rebuild request "
                               "for the k_rebuild kernel and resuming), FP64 pipe",
                     "peak_source": "measured in this run: md_measure_fp64_peak (FP64 FMA chains, CUDA events)",
                     "flop_model": "47 FP64 flop per list entry inside r_cut over both passes, 20 in the skin "
                                   "shell (an FMA counts 2); half of it with the half list",
                     "flop_per_launch": flop, "avg_launch_ms": r64["ms"], "hbm": hbm(r64, "fp64")},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": r64["launches"], "clocks": r64["clocks"],
        "nve_drift_ev_per_atom": (r64["e1"]["te"] - r64["e0"]["te"]) / n,
        "lanes_per_atom": r64["lanes"], "phase_ms": phases(r64),
        "rebuilds_in_timed_region": r64["e1"]["n_rebuilds"] - r64["e0"]["n_rebuilds"],
        "neighbours_per_atom": sum_counts / n,
        "mixed": mixed,
        "double_float": df_line,
        "fp64_walks_ms_per_step": {"full_list": res["fp64"]["ms"] / args.steps,
                                   "half_list": res["fp64_half"]["ms"] / args.steps},
    }
    sur = extras.get("surrogate_fe_1m") if isinstance(extras, dict) else None
    if sur and "paths" in sur:
        p = sur["paths"]
        line["surrogate"] = {
            "workload": "bcc Fe 1,024,000 atoms, 600 K", "bf16_ms_per_step": p["surrogate_bf16"]["ms_per_step"],
            "speedup_vs_eam_fp64": sur["speedup_surrogate_bf16_over_eam_fp64"],
            "speedup_vs_eam_mixed": sur["speedup_surrogate_bf16_over_eam_mixed"],
            "force_rmse_ev_per_a": p["surrogate_bf16"]["force_rmse_vs_fp64_ev_per_a"],
            "nve_drift_ev_per_atom": p["surrogate_bf16"]["nve_drift_ev_per_atom"]}
    for name, rec in (extras.items() if isinstance(extras, dict) else []):
        print(f"extra {name}: " + json.dumps(rec), flush=True)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_extras(torch, md, stream, barrier, max_over_ranks, world):
    """The other workloads (not the headline): throughput at their sizes."""
    out = {}
    # bcc Fe 2,000 atoms, FS analytic, FP64, 100 steps of 1 fs
    w = I.bcc_fe(10, seed=1)
    s = md.System(w, precision="fp64", stream=stream.cuda_stream)
    s.eam_forces()
    s.step(10)
    ms, _ = _time_steps(torch, s, stream, 100, barrier)
    ms = max_over_ranks(ms)
    out["fe2k_fp64"] = {"workload": "bcc Fe 10^3 cells = 2,000 atoms, FS analytic, FP64, dt 1 fs",
                        "steps": 100, "ms_per_step": ms / 100, "value": job_value(w.n_atoms, world, 100, ms)}
    s.close()
    # 256 replicas, n ~ U{10..30}, T ~ U[300, 1200] K, seeds 3000 + r, mixed, graph, 500 steps
    ws, temps = I.fe_replicas()
    b = md.Batch(ws, precision="mixed", stream=stream.cuda_stream)
    b.eam_forces()
    lanes = b.tune()
    b.set_graph(True)
    b.step(500)            # warm-up: records the graph of a 500-step call
    e0 = b.energy()
    ms, _ = _time_steps(torch, b, stream, 500, barrier)
    e1 = b.energy()
    ms = max_over_ranks(ms)
    out["replicas256_mixed"] = {"workload": "256 bcc Fe replicas of 2n^3 atoms, n ~ U{10..30}, T ~ U[300,1200] K, "
                                            "FS analytic, mixed, one persistent launch per 500-step call, "
                                            "replayed from a captured CUDA graph",
                                "n_atoms": b.n, "steps": 500, "ms_per_step": ms / 500, "lanes_per_atom": lanes,
                                "value": job_value(b.n, world, 500, ms),
                                "rebuilds": e1["n_rebuilds"] - e0["n_rebuilds"]}
    # the same replicas thermostatted at their temperatures (Nose-Hoover, tau 100 fs)
    b.set_thermostat(temps, tau_fs=100.0)
    b.step(500)            # warm-up: records the graph of a thermostatted 500-step call
    ms, _ = _time_steps(torch, b, stream, 500, barrier)
    ms = max_over_ranks(ms)
    th = b.thermostat()
    out["replicas256_mixed_nvt"] = {"workload": "the 256 replicas above, each under a Nose-Hoover thermostat at its "
                                                "own temperature (tau 100 fs), same launch and graph",
                                    "n_atoms": b.n, "steps": 500, "ms_per_step": ms / 500,
                                    "value": job_value(b.n, world, 500, ms),
                                    "extended_energy_ev": float(th[:, 3].sum())}
    b.close()
    # bcc Fe-C 128^3 + 0.1 % C, tables, 600 K, strain -1e9/s, mixed, 200 steps of 1 fs
    w = I.bcc_fe_c(128, seed=4)
    s = md.System(w, precision="mixed", stream=stream.cuda_stream, device_inputs=True)
    s.eam_forces()
    lanes = s.tune()
    s.step(5)
    ms, _ = _time_steps(torch, s, stream, 200, barrier)
    ms = max_over_ranks(ms)
    e = s.energy()
    out["fe_c_4m_mixed"] = {"workload": "bcc Fe 128^3 cells + 0.1 % C on octahedral sites (4,198,498 atoms), "
                                        "two-species 5,000-knot tables, 600 K, strain rate -1e9/s along z, "
                                        "mixed, dt 1 fs", "n_atoms": w.n_atoms, "steps": 200,
                            "ms_per_step": ms / 200, "lanes_per_atom": lanes,
                            "value": job_value(w.n_atoms, world, 200, ms), "box_z": float(e["box"][2])}
    s.close()
    # the paper's table-lookup vs explicit-evaluation experiment (§5.1): the same 15-term Fe potential
    # as explicit cubic knot sums and as 5,000-knot Hermite tables, bcc Fe 80^3 cells, 300 K
    rec = {"workload": "bcc Fe 80^3 cells (1,024,000 atoms), 300 K, dt 1 fs; Fe as 15 cubic knot terms (8 for "
                       "V, 7 for phi) evaluated term by term, or the same sums as 5,000-knot Hermite tables",
           "steps": 100}
    for label, pot in (("explicit", I.fe_knots()), ("tables", I.fe_knot_tables())):
        w = I.bcc_fe(80, seed=7, potential=pot)
        for prec in ("fp64", "mixed"):
            s = md.System(w, precision=prec, stream=stream.cuda_stream, device_inputs=True)
            s.eam_forces()
            s.tune()
            s.step(5)
            ms, _ = _time_steps(torch, s, stream, 100, barrier)
            ms = max_over_ranks(ms)
            rec[f"{label}_{prec}_ms_per_step"] = ms / 100
            s.close()
    for prec in ("fp64", "mixed"):
        rec[f"explicit_over_tables_{prec}"] = rec[f"explicit_{prec}_ms_per_step"] / rec[f"tables_{prec}_ms_per_step"]
    out["fe_knots_vs_tables_1m"] = rec
    out["cu500k_walks"] = walks_extra(torch, md, stream, barrier, max_over_ranks, world)
    if os.path.exists(SUR_WEIGHTS):
        out["surrogate_fe_1m"] = surrogate_extra(torch, md, stream, barrier, max_over_ranks, world)
    return out


SUR_WEIGHTS = os.path.join(ROOT, "paper_1107_2619_gb300", "data", "surrogate_fe.npz")


def walks_extra(torch, md, stream, barrier, max_over_ranks, world, k_time=200):
    """The headline workload (fcc Cu 50^3 cells, mixed) with each neighbour walk of the step kernel
    (md.h MD_PASSES_*): Verlet list from global memory, list rows as shared-memory stage slots,
    the list-free link-cell walk over the staged cells, and the half list with Newton's third
    law over the staged cells; ms per step and the phase split."""
    w = I.fcc_cu(CELLS, seed=SEED)
    out = {"workload": "fcc Cu 50^3 cells (500,000 atoms), 300 K, dt 2 fs, 5,000-knot tables, mixed",
           "timed_steps": k_time, "walks": {}}
    for walk, lanes in (("list", 0), ("staged", 4), ("cells", 4), ("half", 8)):
        s = md.System(w, precision="mixed", stream=stream.cuda_stream, device_inputs=True, passes=walk,
                      lanes_per_atom=lanes)
        s.eam_forces()
        lanes = lanes or s.tune()
        s.step(10)
        e0 = s.energy()
        ms, _ = _time_steps(torch, s, stream, k_time, barrier)
        ms = max_over_ranks(ms)
        e1 = s.energy()
        s.set_profiling(True)
        s.step(k_time)
        p = s.profile()
        s.set_profiling(False)
        out["walks"][walk] = {"ms_per_step": ms / k_time, "lanes_per_atom": lanes,
                              "value": job_value(w.n_atoms, world, k_time, ms),
                              "rebuilds": e1["n_rebuilds"] - e0["n_rebuilds"],
                              "phase_ms": {k: p["ms_" + k] / max(1, p["n_" + k])
                                           for k in ("kick", "rebuild", "density", "force")},
                              "groups": s.passes()}
        s.close()
    return out


def surrogate_extra(torch, md, stream, barrier, max_over_ranks, world, path=SUR_WEIGHTS, md_steps=1000,
                    k_time=100):
    """Learned surrogate on bcc Fe 80^3 cells (1,024,000 atoms) at 600 K next to plain FS EAM
    (FP64 and mixed) on the same GPU: force RMSE against the FP64 EAM forces at the same
    thermalised positions, ms per velocity-Verlet step, and NVE drift over md_steps steps."""
    import dataclasses
    d = np.load(path)
    th, gmu, ginv = d["theta"], d["gmu"], d["ginv"]
    w = I.bcc_fe(80, seed=6, temperature=600.0, sigma=0.0)
    n = w.n_atoms
    cs = stream.cuda_stream
    out = {"workload": "bcc Fe 80^3 cells (1,024,000 atoms), 600 K (300 mixed-EAM steps from the perfect "
                       "lattice), dt 1 fs, FS Fe; surrogate: 32 RBF descriptors, 32-64-64-1 SiLU network "
                       "trained on 2,000-atom oracle snapshots",
           "n_atoms": n, "timed_steps": k_time, "nve_steps": md_steps, "paths": {}}
    s = md.System(w, precision="mixed", stream=cs, device_inputs=True)
    s.eam_forces()
    s.tune()
    s.step(300)
    w = dataclasses.replace(w, pos=s.positions(), vel=s.velocities())
    s.close()

    def nve(sys_, label):
        sys_.eam_forces()
        F = sys_.forces()
        sys_.step(3)
        ms, _ = _time_steps(torch, sys_, stream, k_time, barrier)
        ms = max_over_ranks(ms)
        te = [sys_.energy()["te"]]
        left = md_steps - k_time - 3
        while left > 0:
            q = min(left, 100)
            sys_.step(q)
            left -= q
            te.append(sys_.energy()["te"])
        te = np.array(te) / n
        rec = {"ms_per_step": ms / k_time, "value": job_value(n, world, k_time, ms),
               "nve_drift_ev_per_atom": float(te[-1] - te[0]),
               "nve_max_dev_ev_per_atom": float(np.abs(te - te[0]).max())}
        out["paths"][label] = rec
        return F, rec

    s = md.System(w, precision="fp64", stream=cs, device_inputs=True)
    f64, _ = nve(s, "eam_fp64")
    s.close()
    frms = float(np.sqrt((f64 ** 2).mean()))
    out["force_rms_ev_per_a"] = frms
    s = md.System(w, precision="mixed", stream=cs, device_inputs=True)
    s.tune()
    s.set_graph(True)
    f, rec = nve(s, "eam_mixed")
    rec["force_rmse_vs_fp64_ev_per_a"] = float(np.sqrt(((f - f64) ** 2).mean()))
    s.close()
    for net in ("bf16", "fp32"):
        s = md.SurrogateSystem(w, th, gmu, ginv, net=net, stream=cs, device_inputs=True)
        s.set_graph(True)
        f, rec = nve(s, "surrogate_" + net)
        rec["force_rmse_vs_fp64_ev_per_a"] = float(np.sqrt(((f - f64) ** 2).mean()))
        rec["force_max_err_vs_fp64_ev_per_a"] = float(np.abs(f - f64).max())
        s.close()
    p = out["paths"]
    out["speedup_surrogate_bf16_over_eam_fp64"] = p["eam_fp64"]["ms_per_step"] / p["surrogate_bf16"]["ms_per_step"]
    out["speedup_surrogate_bf16_over_eam_mixed"] = p["eam_mixed"]["ms_per_step"] / p["surrogate_bf16"]["ms_per_step"]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=CELLS, help="fcc Cu cube edge in cells (profiling cases)")
    ap.add_argument("--profile-case", action="store_true",
                    help="mixed path only, no e2e/CPU/extra legs: a short run for ncu captures")
    ap.add_argument("--no-extras", action="store_true", help="skip the non-headline workloads")
    ap.add_argument("--passes", choices=["auto", "list", "staged", "cells", "half"], default="auto",
                    help="neighbour walk of the mixed-precision step kernel (md.h MD_PASSES_*)")
    ap.add_argument("--profile-precision", choices=["mixed", "fp64", "fp64_half", "df"], default="mixed",
                    help="precision of the --profile-case run")
    ap.add_argument("--lanes", type=int, default=0, choices=[0, 1, 2, 4, 8, 16, 32],
                    help="lanes per atom (0: the autotuner's choice)")
    ap.add_argument("--surrogate-only", action="store_true",
                    help="run only the learned-surrogate comparison and print its record")
    ap.add_argument("--sur-weights", default=SUR_WEIGHTS, help="trained surrogate (.npz: theta, gmu, ginv)")
    ap.add_argument("--surrogate-profile", choices=["bf16", "fp32"], default=None,
                    help="a short surrogate run on bcc Fe 80^3 cells (no graph) for ncu captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.surrogate_profile:
        import torch
        from paper_1107_2619_gb300 import md
        d = np.load(args.sur_weights)
        w = I.bcc_fe(80, seed=6, temperature=600.0, sigma=0.05)
        stream = torch.cuda.Stream()
        s = md.SurrogateSystem(w, d["theta"], d["gmu"], d["ginv"], net=args.surrogate_profile,
                               stream=stream.cuda_stream, device_inputs=True)
        s.eam_forces()
        s.step(args.warmup)
        ms, _ = _time_steps(torch, s, stream, args.steps, lambda: None)
        print(json.dumps({"surrogate_profile": args.surrogate_profile, "n_atoms": w.n_atoms,
                          "ms_per_step": ms / args.steps}))
        s.close()
        return 0
    if args.surrogate_only:
        import torch
        from paper_1107_2619_gb300 import md
        stream = torch.cuda.Stream()
        print(json.dumps({"surrogate_fe_1m": surrogate_extra(torch, md, stream, lambda: None, lambda x: x, 1,
                                                             args.sur_weights)}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
