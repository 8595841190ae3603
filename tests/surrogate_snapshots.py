"""Training snapshots for the learned surrogate of bcc Fe, from the FP64 oracle.

Independent velocity-Verlet trajectories of 2,000-atom bcc Fe (10^3 cells, Finnis-Sinclair),
target temperatures spread evenly over 300-1500 K, lattice parameters spread over
2.8665 x (1 +- 0.5 %), started from the perfect lattice with Maxwell-Boltzmann velocities at
twice the target temperature (equipartition halves it), equilibrated, then sampled every
`every` steps.  Each snapshot keeps positions, box, potential energy, forces and the target
temperature.  The trajectories run in a spawn process pool, one OpenMP thread each.

Writes one .npz (pos [S][N][3], box [S][3], pe [S], force [S][N][3], temperature [S]) that
the package's training driver reads:
    python tests/surrogate_snapshots.py --out DIR/frames.npz [--frames 10000]
    python -m paper_1107_2619_gb300.train_surrogate --frames DIR/frames.npz --out DIR
"""
import argparse
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"


def trajectory(args):
    """Frames of one oracle trajectory: list of (pos, box, pe, force, T)."""
    t, n_traj, frames, every, equil, seed = args
    import oracle
    from paper_1107_2619_gb300 import inputs as I
    oracle.lib().orc_set_threads(1)
    T = 300.0 + 1200.0 * t / max(n_traj - 1, 1)
    u = I.random_uniform(seed, 500 + t, 1)[0]
    a = 2.8665 * (1.0 + 0.01 * (u - 0.5))
    w = I.bcc_fe(10, seed=seed * 100000 + t, temperature=2.0 * T, sigma=0.0, a=a)
    m = w.potential.masses
    st = oracle.run_vv(w.pos, w.vel, w.species, m, w.box, w.potential, 1.0, equil, 0.3, 32)
    out = []
    for _ in range(frames):
        st = oracle.run_vv(st["pos"], st["vel"], w.species, m, w.box, w.potential, 1.0, every, 0.3, 32,
                           force=st["force"])
        out.append((st["pos"].astype(np.float64), w.box.copy(), float(st["energies"][-1][0]),
                    st["force"].astype(np.float64), T))
    return out


def generate(n_frames, per_traj=50, every=20, equil=300, seed=5, procs=None):
    """n_frames oracle snapshots as a dict of stacked arrays."""
    n_traj = (n_frames + per_traj - 1) // per_traj
    jobs = [(t, n_traj, per_traj, every, equil, seed) for t in range(n_traj)]
    with mp.get_context("spawn").Pool(procs or os.cpu_count() or 4, initializer=_worker_init) as pool:
        res = pool.map(trajectory, jobs, chunksize=1)
    fr = [f for traj in res for f in traj][:n_frames]
    return dict(pos=np.stack([f[0] for f in fr]), box=np.stack([f[1] for f in fr]),
                pe=np.array([f[2] for f in fr]), force=np.stack([f[3] for f in fr]),
                temperature=np.array([f[4] for f in fr]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--per-traj", type=int, default=50)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--equil", type=int, default=300)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    args = ap.parse_args()
    t0 = time.time()
    d = generate(args.frames, args.per_traj, args.every, args.equil, args.seed, args.procs)
    recipe = ("oracle FP64 FS-Fe velocity Verlet, dt 1 fs, 10^3 bcc cells, T 300-1500 K, "
              f"a = 2.8665 (1 +- 0.5 %), {args.equil} equilibration steps, a frame every "
              f"{args.every} steps, {args.per_traj} frames per trajectory, seed {args.seed}")
    np.savez(args.out, recipe=np.array(recipe), seconds=np.array(time.time() - t0), **d)
    print(f"{d['pe'].size} oracle frames in {time.time() - t0:.1f} s -> {args.out}", flush=True)


if __name__ == "__main__":
    main()
