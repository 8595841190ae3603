"""Throughput of the EAM hot path on one GB300 (atom-steps/s), with its roofline.

Workload: fcc Cu 50x50x50 cells = 500,000 atoms, Sutton-Chen EAM as 5,000-knot cubic tables
(cutoff 2a), 300 K seeded velocities, velocity-Verlet NVE with dt = 2 fs; the list has a
0.3 Å skin and is rebuilt whenever an atom has moved more than skin/2.  One step is the
whole path: half kick + drift + skin check, [link-cell binning, sort, list build], density
pass, force pass + half kick.  The headline is the mixed path (FP32 pair/density terms,
FP64 positions/integration/density sum/reductions); the FP64 path is timed beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

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

METRIC = "atom-steps/s (EAM force+integrate, 1 GB300)"
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


def _traffic(kernel):
    """DRAM bytes per launch from a committed ncu capture, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            t = json.load(fh)
        rec = t[kernel]
        with open(os.path.join(ROOT, rec["source"]), "rb") as fh:
            h = hashlib.sha256(fh.read()).hexdigest()
        return float(rec["bytes_per_launch"]) if h == rec["sha256"] else None
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

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
        self.lines = []
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


def _algorithmic_bytes(kernel, n, sum_counts, energy_fraction):
    """HBM bytes one launch must move (neighbour gathers are L2 hits: cell-sorted atoms).
    density (mixed): list 4/neighbour + count 4 + own posf 16 + rho, F', E_i writes 24 + pass-2 copy 16.
    force (mixed):   list 4/neighbour + count 4 + own p2f 16 + force r/w 64 + velocity r/w 64
                     (+ E_i r/w 16 on the energy step)."""
    if kernel == "density":
        return 4 * sum_counts + 60 * n
    return 4 * sum_counts + (148 + 16 * energy_fraction) * n


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
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    w = I.fcc_cu(args.cells, seed=SEED + rank)
    n = w.n_atoms
    stream = torch.cuda.Stream()
    res = {}
    snapshot = {}
    for precision in (("mixed",) if args.profile_case else ("mixed", "fp64")):
        s = md.System(w, precision=precision, stream=stream.cuda_stream, device_inputs=True)
        s.eam_forces()
        lanes = s.tune()
        counts = s.get(md.MD_GET_NBR_COUNT)
        s.step(args.warmup)
        e0 = s.energy()
        s.set_profiling(True)
        launches0 = s.profile()["launches"]
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        with Clocks(local) as clk:
            start.record(stream)
            s.step(args.steps)
            end.record(stream)
            end.synchronize()
        barrier()
        ms = max_over_ranks(start.elapsed_time(end))
        prof = s.profile()
        e1 = s.energy()
        res[precision] = dict(ms=ms, prof=prof, e0=e0, e1=e1, counts=counts, clocks=clk.summary(),
                              launches=prof["launches"] - launches0, lanes=lanes)
        # forces of both precisions at the same thermalised positions (the mixed run's last state)
        if precision == "mixed":
            snapshot["pos"] = s.positions()
            snapshot["mixed"] = s.forces()
        else:
            s.set_state(pos=snapshot["pos"])
            s.eam_forces()
            snapshot["fp64"] = s.forces()
        s.close()
    if args.profile_case:
        if rank == 0:
            r = res["mixed"]
            print(json.dumps({"profile_case": True, "n_atoms": n, "ms_per_step": r["ms"] / args.steps,
                              "lanes": r["lanes"], "kernel_ms": {k: r["prof"]["ms_" + k] / max(1, r["prof"]["n_" + k])
                                                               for k in ("kick", "rebuild", "density", "force")}}))
        return 0

    # end to end through the C ABI with host buffers: state in, one step, state and energies out
    e2e = None
    if rank == 0 or world > 1:
        pin = lambda shape: torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()
        hp, hv, hf = pin((n, 3)), pin((n, 3)), pin((n, 3))
        s = md.System(w, precision="mixed")
        s.eam_forces()
        s.get(md.MD_GET_POS, hp), s.get(md.MD_GET_VEL, hv), s.get(md.MD_GET_FORCE, hf)
        k_e2e = max(3, min(args.steps, 200))
        for _ in range(3):
            s.set_state(hp, hv, hf), s.step(1), s.get(md.MD_GET_POS, hp), s.get(md.MD_GET_VEL, hv)
            s.get(md.MD_GET_FORCE, hf), s.energy()
        barrier()
        t0 = time.perf_counter()
        for _ in range(k_e2e):
            s.set_state(hp, hv, hf)
            s.step(1)
            s.get(md.MD_GET_POS, hp)
            s.get(md.MD_GET_VEL, hv)
            s.get(md.MD_GET_FORCE, hf)
            s.energy()
        t = max_over_ranks(time.perf_counter() - t0)
        s.close()
        e2e = {"value": world * n * k_e2e / t, "unit": UNIT, "h2d_bytes_per_step": 72 * n,
               "d2h_bytes_per_step": 72 * n + C.sizeof(md.md_energies), "steps": k_e2e,
               "note": "each step: md_set_state(pos, vel, force from pinned host), md_step(1), "
                       "md_get(pos, vel, force into pinned host), md_energy"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    hbm_peak, peak_src = _peaks()
    r = res["mixed"]
    p = r["prof"]
    sum_counts = float(r["counts"].sum())
    kern = "force" if p["ms_force"] >= p["ms_density"] else "density"
    avg_ms = p["ms_" + kern] / max(1, p["n_" + kern])
    nbytes = _algorithmic_bytes(kern, n, sum_counts, 1.0 / max(1, args.steps))
    achieved = nbytes / (avg_ms * 1e-3) / 1e9
    kname = "k_force32" if kern == "force" else "k_density32"
    traffic = _traffic(kname)

    f64, f32 = snapshot["fp64"], snapshot["mixed"]
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

    def path_summary(pr):
        q = res[pr]
        de = (q["e1"]["te"] - q["e0"]["te"]) / n
        return {"value": world * n * args.steps / (q["ms"] * 1e-3), "ms_per_step": q["ms"] / args.steps,
                "nve_drift_ev_per_atom": de, "steps_timed": args.steps, "lanes_per_atom": q["lanes"],
                "rebuilds_in_timed_region": q["e1"]["n_rebuilds"] - q["e0"]["n_rebuilds"],
                "kernel_ms_per_step": {k: q["prof"]["ms_" + k] / max(1, q["prof"]["n_" + k])
                                       for k in ("kick", "rebuild", "density", "force")}}

    line = {
        "metric": METRIC, "value": world * n * args.steps / (r["ms"] * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"] / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": _config("mixed: FP32 pair/density terms, FP64 integration and sums"),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "kernel": kname,
                     "algorithmic_bytes_per_launch": nbytes, "avg_launch_ms": avg_ms,
                     "peak_source": peak_src},
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": r["launches"], "clocks": r["clocks"],
        "mixed_path": path_summary("mixed"), "fp64_path": path_summary("fp64"),
        "mixed_vs_fp64_force_error_ev_per_a": {"state": "positions after the mixed run's timed steps",
                                               "max": float(ferr.max()),
                                               "rms": float(np.sqrt((ferr ** 2).mean())),
                                               "max_force": float(np.abs(f64).max())},
        "neighbours_per_atom": sum_counts / n,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cells", type=int, default=CELLS, help="fcc Cu cube edge in cells (profiling cases)")
    ap.add_argument("--profile-case", action="store_true",
                    help="mixed path only, no e2e/CPU legs: a short run for ncu captures")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
