"""Train the learned per-atom surrogate of bcc Fe on the GPU with the library's own kernels.

Input: reference snapshots of 2,000-atom bcc Fe (10^3 cells, Finnis-Sinclair EAM) as one .npz
with pos [S][N][3] (Å), box [S][3] (Å), pe [S] (eV), force [S][N][3] (eV/Å) and
temperature [S] (K).  The shipped network was trained on 10,000 snapshots of FP64 reference
trajectories (the recipe is stored in the .npz and copied to the summary).

Training (md_sur_*): the snapshots become the replicas of one batch context, the descriptors
are standardised over the training set, and Adam steps on minibatches of `batch` snapshots
follow a stepped learning-rate schedule.  The last `val` snapshots (after a seeded shuffle)
are held out and only evaluated.

Writes surrogate_fe.npz (theta, gmu, ginv) and surrogate_fe.json (losses, timings, recipe):
    python -m paper_1107_2619_gb300.train_surrogate --frames FRAMES.npz --out DIR [--iters 16000]
"""
import argparse
import json
import os
import time

import numpy as np

from . import inputs as I
from . import md

SCHEDULE = [(3e-3, 0.25), (1e-3, 0.25), (3e-4, 0.25), (1e-4, 0.25)]


def train(frames: dict, iters: int = 16000, batch: int = 16, val: int = 500, w_e: float = 10.0,
          w_f: float = 1.0, seed: int = 5, schedule=SCHEDULE, log_fn=print):
    """Train from a dict of snapshot arrays; returns (theta, gmu, ginv, summary)."""
    n = int(frames["pe"].shape[0])
    perm = np.argsort(I.random_u64(seed, 900, n), kind="stable")
    pos, box = frames["pos"][perm], frames["box"][perm]
    eref, fref = np.asarray(frames["pe"], np.float64)[perm], frames["force"][perm]
    temps = frames["temperature"][perm]
    n_train = n - val
    proto = I.bcc_fe(10, seed=0)
    ws = [I.Workload(name=f"frame {k}", pos=pos[k], vel=np.zeros_like(pos[k]), species=proto.species,
                     box=box[k], potential=proto.potential, skin=0.3, k_max=32, dt_fs=1.0, steps=0,
                     temperature=float(temps[k])) for k in range(n)]
    theta = I.sur_init_weights(seed, I.SUR_FE).astype(np.float32)
    theta[-1] = np.float32(eref[:n_train].sum() / (n_train * proto.n_atoms))   # b3 = mean energy per atom

    t1 = time.time()
    b = md.SurrogateBatch(ws, theta, net="fp32")
    b.standardize()
    b.set_reference(eref, fref.reshape(-1, 3))
    t_setup = time.time() - t1
    log = []
    v0, _ = b.loss_grad(n_train, n, w_e, w_f)
    log.append(dict(iter=0, val=v0.tolist()))
    t2 = time.time()
    done = 0
    for lr, frac in schedule:
        n_it = int(round(iters * frac))
        for _chunk in range(4):
            it = n_it // 4
            tl = b.train(it, batch, lr, w_e, w_f, seed=seed * 1000003 + done, rep_begin=0, rep_end=n_train)
            done += it
            vl, _ = b.loss_grad(n_train, n, w_e, w_f)
            log.append(dict(iter=done, lr=lr, train_batch=tl.tolist(), val=vl.tolist()))
            if log_fn:
                log_fn(f"iter {done:6d} lr {lr:.0e} batch {tl} val {vl}")
    t_train = time.time() - t2
    theta, gmu, ginv = b.sur_params()
    b.close()
    summary = dict(
        data=dict(frames=n, train=n_train, val=val, atoms_per_frame=proto.n_atoms),
        training=dict(optimizer="Adam (beta1 0.9, beta2 0.999, eps 1e-8)", batch_frames=batch, iters=done,
                      schedule=list(schedule), w_e=w_e, w_f=w_f, seconds=t_train, setup_seconds=t_setup,
                      net="FP32 (CUDA cores)"),
        # RMS force error (eV/Å) and energy error per atom (eV) on the held-out frames
        val_force_rmse_ev_per_a=float(np.sqrt(log[-1]["val"][1] / w_f)),
        val_energy_rmse_ev_per_atom=float(np.sqrt(log[-1]["val"][0] / w_e)),
        val_force_rms_ev_per_a=float(np.sqrt((fref[n_train:] ** 2).mean())),
        log=log)
    return theta, gmu, ginv, summary


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--frames", required=True, help=".npz of reference snapshots")
    ap.add_argument("--out", required=True)
    ap.add_argument("--val", type=int, default=500)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--iters", type=int, default=16000)
    ap.add_argument("--w-e", type=float, default=10.0)
    ap.add_argument("--w-f", type=float, default=1.0)
    ap.add_argument("--seed", type=int, default=5)
    args = ap.parse_args()
    os.makedirs(args.out, exist_ok=True)
    d = np.load(args.frames)
    frames = {k: d[k] for k in ("pos", "box", "pe", "force", "temperature")}
    theta, gmu, ginv, summary = train(frames, args.iters, args.batch, args.val, args.w_e, args.w_f, args.seed)
    if "recipe" in d:
        summary["data"]["recipe"] = str(d["recipe"])
    np.savez(os.path.join(args.out, "surrogate_fe.npz"), theta=theta, gmu=gmu, ginv=ginv)
    with open(os.path.join(args.out, "surrogate_fe.json"), "w") as fh:
        json.dump(summary, fh, indent=1)
    print(json.dumps({k: v for k, v in summary.items() if k != "log"}))


if __name__ == "__main__":
    main()
