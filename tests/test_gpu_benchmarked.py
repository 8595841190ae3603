"""Oracle parity of the configurations the benchmark times, in the launch configuration it
times them: mixed-precision batches of uneven replicas replayed from a captured CUDA graph
(NVE and Nose-Hoover, list rebuilds inside the replays), the whole 256-replica batch of
5,151,202 atoms sampled replica by replica, and the learned surrogate on 1,024,000-atom bcc Fe
(bf16 tensor-core and FP32 networks) under graph replay.

Mixed bound: each replica's forces against the bound derived per atom for that replica's
atoms, box and FP32 coordinates (tests/mixed_bound.py); PE within 1e-6 relative.
"""
import numpy as np
import pytest

import oracle
from mixed_bound import assert_mixed_forces
from paper_1107_2619_gb300 import inputs as I, md

MIXED_PE_TOL = 1e-6

pytestmark = pytest.mark.gpu

SPEC = dict(I.SUR_FE)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _check_replica_state(w, pos, f, img, pe, lanes):
    """Forces and PE of one replica at the GPU's own final positions against the oracle."""
    assert_mixed_forces(w, pos, f, img, lanes=lanes, pe=pe, pe_tol=MIXED_PE_TOL)


def test_mixed_batch_of_uneven_replicas_under_graph_replay_matches_oracle():
    """The first six replicas of the 256-replica recipe (9,826-43,904 atoms, 300-1,115 K),
    mixed precision, autotuned lanes, three replays of a captured 10-step call (30 steps, list
    rebuilds inside): every replica's trajectory against the oracle's FP64 velocity Verlet, then
    its forces and PE at the GPU's final positions."""
    ws, _ = I.fe_replicas(range(6))
    with md.Batch(ws, precision="mixed") as b:
        b.eam_forces()
        lanes = b.tune()
        b.set_graph(True)
        for _ in range(3):
            b.step(10)
        e = b.energy()
        pos, f, img = b.positions(), b.forces(), b.get(md.MD_GET_IMAGE)
        per = b.replica_energies()
    assert e["n_rebuilds"] >= 2          # the initial build and at least one inside the replays
    o = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30,
                            w.skin, w.k_max)
        p = pos[o[r]:o[r + 1]]
        assert np.abs(p - ref["pos"]).max() < 1e-4, r
        assert abs(per[r]["pe"] - ref["energies"][-1, 0]) <= 1e-5 * abs(ref["energies"][-1, 0]), r
        _check_replica_state(w, p, f[o[r]:o[r + 1]], img[o[r]:o[r + 1]], per[r]["pe"], lanes)


def test_mixed_batch_under_thermostats_and_graph_replay_matches_oracle():
    """The same launch form with a Nose-Hoover thermostat per replica at its own temperature
    (tau 30 fs): trajectories and thermostat variables against the oracle's NVT integrator
    with the inertia the library set."""
    ws, temps = I.fe_replicas(range(4))
    with md.Batch(ws, precision="mixed") as b:
        b.set_thermostat(temps, tau_fs=30.0)
        b.eam_forces()
        q = b.thermostat()[:, 2]
        b.set_graph(True)
        for _ in range(3):
            b.step(10)
        pos, f, th, img = b.positions(), b.forces(), b.thermostat(), b.get(md.MD_GET_IMAGE)
        per = b.replica_energies()
    o = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        ref = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30,
                             w.skin, w.k_max, float(temps[r]), float(q[r]))
        p = pos[o[r]:o[r + 1]]
        assert np.abs(p - ref["pos"]).max() < 1e-4, r
        assert abs(th[r, 0] - ref["pi"]) <= 1e-4 * max(abs(ref["pi"]), 1e-6), r
        assert abs(th[r, 3] - ref["energies"][-1, 2]) <= 1e-5 * abs(ref["energies"][-1, 2]), r
        _check_replica_state(w, p, f[o[r]:o[r + 1]], img[o[r]:o[r + 1]], per[r]["pe"], 1)


def test_full_size_256_replica_batch_sampled():
    """The benchmark's batch: all 256 replicas (5,151,202 atoms) in one context, mixed, tuned,
    20 steps as two replays of a captured 10-step call.  Sampled outputs the oracle computes one
    replica at a time: the first, the largest, the smallest and the last replica's forces and PE
    at the GPU's final positions, and their neighbour lists (bit-exact as sets) from a build at
    those positions."""
    ws, _ = I.fe_replicas()
    sizes = np.array([w.n_atoms for w in ws])
    assert sizes.sum() == 5151202
    sample = sorted({0, int(sizes.argmax()), int(sizes.argmin()), 255})
    o = np.concatenate([[0], np.cumsum(sizes)])
    with md.Batch(ws, precision="mixed") as b:
        b.eam_forces()
        lanes = b.tune()
        b.set_graph(True)
        b.step(10)
        b.step(10)
        pos, f, img = b.positions(), b.forces(), b.get(md.MD_GET_IMAGE)
        per = b.replica_energies()
        b.build_neighbours()
        cnt, nl = b.neighbours()
    for r in sample:
        w = ws[r]
        p = pos[o[r]:o[r + 1]]
        _check_replica_state(w, p, f[o[r]:o[r + 1]], img[o[r]:o[r + 1]], per[r]["pe"], lanes)
        ref = oracle.forces(p, w.species, w.box, w.potential, skin=w.skin, k_max=w.k_max, method="cells")
        assert np.array_equal(cnt[o[r]:o[r + 1]], ref["count"]), r
        rows = nl[o[r]:o[r + 1]]
        got = [sorted((rows[i, :cnt[o[r] + i]] - o[r]).tolist()) for i in range(w.n_atoms)]
        exp = [sorted(ref["list"][i, :ref["count"][i]].tolist()) for i in range(w.n_atoms)]
        assert got == exp, r


def _fold(theta, gmu, ginv):
    nb, h1 = SPEC["nb"], SPEC["h1"]
    th = np.asarray(theta, np.float64).copy()
    W1 = th[:h1 * nb].reshape(h1, nb) * np.asarray(ginv, np.float64)[None, :]
    th[h1 * nb:h1 * nb + h1] -= W1 @ np.asarray(gmu, np.float64)
    th[:h1 * nb] = W1.ravel()
    return th


@pytest.mark.parametrize("net", ["bf16", "fp32"])
def test_full_size_surrogate_1m_under_graph_replay(net):
    """The surrogate comparison's workload: bcc Fe 80^3 cells (1,024,000 atoms), the shipped
    trained network, graph replay of a 10-step call twice; forces, per-atom energies and the
    total at the GPU's final positions against the oracle's FP64 evaluation of the same
    network (bf16: 3 % of the largest force and 1 % RMS; FP32: 1e-4 of the largest force)."""
    import os
    d = np.load(os.path.join(os.path.dirname(__file__), "..", "paper_1107_2619_gb300", "data",
                             "surrogate_fe.npz"))
    th, gmu, ginv = d["theta"], d["gmu"], d["ginv"]
    w = I.bcc_fe(80, seed=6, temperature=600.0, sigma=0.05)
    with md.SurrogateSystem(w, th, gmu, ginv, net=net) as s:
        s.eam_forces()
        s.set_graph(True)
        s.step(10)
        s.step(10)
        pos, F = s.positions(), s.forces()
        Ei = s.get(md.MD_GET_EATOM)
        pe = s.energy()["pe"]
    ref = oracle.surrogate(pos, w.box, SPEC, _fold(th, gmu, ginv), k_max=64)
    fmax = np.abs(ref["force"]).max()
    if net == "bf16":
        assert np.abs(F - ref["force"]).max() <= 0.03 * fmax
        assert np.sqrt(((F - ref["force"]) ** 2).mean()) <= 0.01 * np.sqrt((ref["force"] ** 2).mean())
        assert np.abs(Ei - ref["e_atom"]).max() <= 0.02 * max(1.0, np.abs(ref["e_atom"]).max())
        assert abs(pe - ref["energy"]) <= 1e-3 * w.n_atoms
    else:
        assert np.abs(F - ref["force"]).max() <= 1e-4 * fmax
        assert np.abs(Ei - ref["e_atom"]).max() <= 2e-5 * max(1.0, np.abs(ref["e_atom"]).max())
        assert abs(pe - ref["energy"]) <= 2e-5 * w.n_atoms
