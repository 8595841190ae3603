"""Train the learned per-atom surrogate of bcc Fe on oracle snapshots, on the GPU.

Training data (the oracle, FP64, Finnis-Sinclair Fe): independent velocity-Verlet
trajectories of 2,000-atom bcc Fe (10^3 cells), target temperatures spread evenly over
300-1500 K, lattice parameters spread over 2.8665 x (1 +- 0.5 %), started from the perfect
lattice with Maxwell-Boltzmann velocities at twice the target temperature (equipartition
halves it), equilibrated, then sampled every `every` steps.  Each snapshot keeps positions,
box, potential energy and forces.  The trajectories run in a spawn process pool, one OpenMP
thread each, before any GPU call.

Training (the library's own kernels, md_sur_*): the snapshots become the replicas of one
batch context, the descriptors are standardised over the training set, and Adam steps on
minibatches of `batch` snapshots follow a stepped learning-rate schedule.  The last `val`
snapshots (after a seeded shuffle) are held out and only evaluated.

Writes an .npz with theta, gmu, ginv and a .json summary (losses, timings, data recipe).
    python tests/surrogate_train_fe.py --out DIR [--frames 10000] [--iters 16000]
"""
import argparse
import json
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
    """Frames of one oracle trajectory: list of (pos, box, pe, force)."""
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


def generate(n_frames, per_traj, every, equil, seed, procs):
    n_traj = (n_frames + per_traj - 1) // per_traj
    jobs = [(t, n_traj, per_traj, every, equil, seed) for t in range(n_traj)]
    with mp.get_context("spawn").Pool(procs, initializer=_worker_init) as pool:
        res = pool.map(trajectory, jobs, chunksize=1)
    return [f for traj in res for f in traj][:n_frames]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", required=True)
    ap.add_argument("--frames", type=int, default=10000)
    ap.add_argument("--per-traj", type=int, default=50)
    ap.add_argument("--every", type=int, default=20)
    ap.add_argument("--equil", type=int, default=300)
    ap.add_argument("--val", type=int, default=500)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--iters", type=int, default=16000)
    ap.add_argument("--w-e", type=float, default=10.0)
    ap.add_argument("--w-f", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)

    t0 = time.time()
    frames = generate(args.frames, args.per_traj, args.every, args.equil, args.seed, args.procs)
    t_data = time.time() - t0
    print(f"{len(frames)} oracle frames in {t_data:.1f} s", flush=True)

    from paper_1107_2619_gb300 import inputs as I
    from paper_1107_2619_gb300 import md
    perm = np.argsort(I.random_u64(args.seed, 900, len(frames)), kind="stable")
    frames = [frames[i] for i in perm]
    n = len(frames)
    n_train = n - args.val
    proto = I.bcc_fe(10, seed=0)
    ws = [I.Workload(name=f"frame {k}", pos=f[0], vel=np.zeros_like(f[0]), species=proto.species,
                     box=f[1], potential=proto.potential, skin=0.3, k_max=32, dt_fs=1.0, steps=0,
                     temperature=f[4]) for k, f in enumerate(frames)]
    eref = np.array([f[2] for f in frames])
    fref = np.concatenate([f[3] for f in frames])
    theta = I.sur_init_weights(args.seed, I.SUR_FE).astype(np.float32)
    theta[-1] = np.float32(eref[:n_train].sum() / (n_train * proto.n_atoms))   # b3 = mean energy per atom

    t1 = time.time()
    b = md.SurrogateBatch(ws, theta, net="fp32")
    b.standardize()
    b.set_reference(eref, fref)
    t_setup = time.time() - t1
    schedule = [(3e-3, 0.25), (1e-3, 0.25), (3e-4, 0.25), (1e-4, 0.25)]
    log = []
    v0, _ = b.loss_grad(n_train, n, args.w_e, args.w_f)
    log.append(dict(iter=0, val=v0.tolist()))
    t2 = time.time()
    done = 0
    for k, (lr, frac) in enumerate(schedule):
        iters = int(round(args.iters * frac))
        for chunk in range(4):
            it = iters // 4
            tl = b.train(it, args.batch, lr, args.w_e, args.w_f, seed=args.seed * 1000003 + done,
                         rep_begin=0, rep_end=n_train)
            done += it
            vl, _ = b.loss_grad(n_train, n, args.w_e, args.w_f)
            log.append(dict(iter=done, lr=lr, train_batch=tl.tolist(), val=vl.tolist()))
            print(f"iter {done:6d} lr {lr:.0e} batch {tl} val {vl}", flush=True)
    t_train = time.time() - t2
    theta, gmu, ginv = b.sur_params()
    # RMS force error (eV/Å) and energy error per atom (eV) on the held-out frames
    val_f_rmse = float(np.sqrt(log[-1]["val"][1] / args.w_f))
    val_e_rmse = float(np.sqrt(log[-1]["val"][0] / args.w_e))
    b.close()
    np.savez(os.path.join(args.out, "surrogate_fe.npz"), theta=theta, gmu=gmu, ginv=ginv)
    summary = dict(
        data=dict(frames=n, train=n_train, val=args.val, atoms_per_frame=proto.n_atoms,
                  recipe="oracle FP64 FS-Fe velocity Verlet, dt 1 fs, 10^3 bcc cells, T 300-1500 K, "
                         f"a = 2.8665 (1 +- 0.5 %), {args.equil} equilibration steps, a frame every "
                         f"{args.every} steps, {args.per_traj} frames per trajectory", seed=args.seed,
                  seconds=t_data, procs=args.procs),
        training=dict(optimizer="Adam (beta1 0.9, beta2 0.999, eps 1e-8)", batch_frames=args.batch,
                      iters=done, schedule=schedule, w_e=args.w_e, w_f=args.w_f, seconds=t_train,
                      setup_seconds=t_setup, net="FP32 (CUDA cores)"),
        val_force_rmse_ev_per_a=val_f_rmse, val_energy_rmse_ev_per_atom=val_e_rmse,
        val_force_rms_ev_per_a=float(np.sqrt((np.concatenate([f[3] for f in frames[n_train:]]) ** 2).mean())),
        log=log)
    with open(os.path.join(args.out, "surrogate_fe.json"), "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "log"}))


if __name__ == "__main__":
    main()
