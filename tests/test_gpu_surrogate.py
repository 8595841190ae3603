"""GPU parity of the learned surrogate against the oracle (descriptors, network, forces,
training-loss gradient, Adam), the bf16 tensor-core network within its stated bound, and
the edge cases.  The oracle gets the network folded onto raw descriptors (W1 ginv,
b1 - W1 ginv gmu) in FP64; the GPU runs the FP32 parameters it was given.
"""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I
from paper_1107_2619_gb300 import md

pytestmark = pytest.mark.gpu

SPEC = dict(I.SUR_FE)
NB, H1 = SPEC["nb"], SPEC["h1"]


def fold(theta, gmu, ginv):
    """Parameters for standardised inputs -> the same network on raw descriptors (FP64)."""
    th = np.asarray(theta, np.float64).copy()
    W1 = th[:H1 * NB].reshape(H1, NB)
    b1 = th[H1 * NB:H1 * NB + H1]
    W1r = W1 * np.asarray(ginv, np.float64)[None, :]
    th[H1 * NB:H1 * NB + H1] = b1 - W1r @ np.asarray(gmu, np.float64)
    th[:H1 * NB] = W1r.ravel()
    return th


def params(seed, scale=1.5):
    th = I.sur_init_weights(seed, SPEC, scale=scale).astype(np.float32)
    rng = np.random.default_rng(seed)
    th[H1 * NB:H1 * NB + H1] = rng.normal(0, 0.3, H1).astype(np.float32)      # b1
    th[-1] = np.float32(-4.0)                                                  # b3
    gmu = rng.uniform(0.0, 3.0, NB).astype(np.float32)
    ginv = rng.uniform(0.3, 1.5, NB).astype(np.float32)
    return th, gmu, ginv


def fe(n=6, seed=31, T=600.0, sigma=0.1):
    return I.bcc_fe(n, seed=seed, temperature=T, sigma=sigma)


def ref(w, th, gmu, ginv):
    return oracle.surrogate(w.pos, w.box, SPEC, fold(th, gmu, ginv), k_max=64)


# --------------------------------------------------------------------------- FP32 network
def test_descriptors_match_oracle():
    w = fe(7)
    th, gmu, ginv = params(1)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        G = s.descriptors()
    o = ref(w, th, gmu, ginv)
    assert np.abs(G - o["G"]).max() <= 2e-5 * max(1.0, np.abs(o["G"]).max())


@pytest.mark.parametrize("n", [5, 7])
def test_fp32_network_energy_gradient_forces_match_oracle(n):
    w = fe(n, seed=40 + n)
    th, gmu, ginv = params(2)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        pe = s.eam_forces()
        F = s.forces()
        Ei = s.get(md.MD_GET_EATOM)
        g = s.dE_dG()
        e = s.energy()
    o = ref(w, th, gmu, ginv)
    emax = max(1.0, np.abs(o["e_atom"]).max())
    assert np.abs(Ei - o["e_atom"]).max() <= 2e-5 * emax
    assert abs(pe - o["energy"]) <= 2e-5 * emax * w.n_atoms
    assert abs(e["pe"] - pe) <= 1e-9 * abs(pe)
    assert np.abs(g - o["grad"]).max() <= 1e-4 * np.abs(o["grad"]).max()
    fmax = np.abs(o["force"]).max()
    assert np.abs(F - o["force"]).max() <= 1e-4 * fmax
    assert np.abs(F.sum(axis=0)).max() <= 1e-4 * fmax      # pair-symmetric forces


def test_fp32_virial_is_the_pair_virial():
    w = fe(6, seed=9)
    th, gmu, ginv = params(3)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        s.eam_forces()
        e = s.energy()
        F = s.forces()
    # W = sum_i r_i (x) F_i for the unwrapped minimum-image pairs equals -1/2 sum d (x) f over pairs;
    # check its trace against the volume derivative of the energy by finite differences
    th64 = fold(th, gmu, ginv)
    h = 1e-5
    Ep = oracle.surrogate(w.pos * (1 + h), w.box * (1 + h), SPEC, th64, k_max=64)["energy"]
    Em = oracle.surrogate(w.pos * (1 - h), w.box * (1 - h), SPEC, th64, k_max=64)["energy"]
    dE_dlnL = (Ep - Em) / (2 * h)            # = -tr W
    assert abs(np.trace(e["virial"]) + dE_dlnL) <= 1e-3 * max(1.0, abs(dE_dlnL))
    assert np.isfinite(F).all()


# --------------------------------------------------------------------------- bf16 tensor cores
def bf16_bound(fmax):
    """bf16 inputs, weights and activations (unit roundoff 2^-9 each) through three layers:
    forces within 3 % of the largest force (observed well below; see the design notes)."""
    return 0.03 * fmax


@pytest.mark.parametrize("n", [5, 9])
def test_bf16_network_within_bound_of_oracle(n):
    w = fe(n, seed=50 + n)
    th, gmu, ginv = params(4)
    with md.SurrogateSystem(w, th, gmu, ginv, net="bf16") as s:
        s.eam_forces()
        F = s.forces()
        Ei = s.get(md.MD_GET_EATOM)
        g = s.dE_dG()
    o = ref(w, th, gmu, ginv)
    fmax = np.abs(o["force"]).max()
    assert np.abs(F - o["force"]).max() <= bf16_bound(fmax)
    assert np.sqrt(((F - o["force"]) ** 2).mean()) <= 0.01 * np.sqrt((o["force"] ** 2).mean())
    assert np.abs(Ei - o["e_atom"]).max() <= 0.02 * max(1.0, np.abs(o["e_atom"]).max())
    assert np.abs(g - o["grad"]).max() <= 0.03 * np.abs(o["grad"]).max()


def test_bf16_and_fp32_agree_on_a_ragged_tile():
    w = fe(6, seed=5)                    # 432 atoms: 3 full 128-atom tiles and a tail of 48
    th, gmu, ginv = params(6)
    out = {}
    for net in ("fp32", "bf16"):
        with md.SurrogateSystem(w, th, gmu, ginv, net=net) as s:
            s.eam_forces()
            out[net] = s.forces(), s.get(md.MD_GET_EATOM)
    fmax = np.abs(out["fp32"][0]).max()
    assert np.abs(out["bf16"][0] - out["fp32"][0]).max() <= bf16_bound(fmax)
    assert np.isfinite(out["bf16"][1]).all() and np.abs(out["bf16"][1] - out["fp32"][1]).max() < 0.1


# --------------------------------------------------------------------------- training
def frames(k=3, n=5, seed=70):
    ws, eref, fref = [], [], []
    for s in range(k):
        w = I.bcc_fe(n, seed=seed + s, temperature=300 + 400 * s, sigma=0.05 + 0.03 * s)
        o = oracle.forces(w.pos, w.species, w.box, w.potential)
        ws.append(w)
        eref.append(o["pe"])
        fref.append(o["force"])
    return ws, np.array(eref), fref


@pytest.mark.parametrize("standardised", [False, True])
def test_loss_and_gradient_match_oracle(standardised):
    ws, eref, fref = frames()
    th, gmu, ginv = params(7, scale=1.0)
    if not standardised:
        gmu, ginv = np.zeros(NB, np.float32), np.ones(NB, np.float32)
    w_e, w_f = 0.7, 1.3
    with md.SurrogateBatch(ws, th, gmu, ginv) as b:
        b.set_reference(eref, np.concatenate(fref))
        loss, grad = b.loss_grad(0, len(ws), w_e, w_f)
    o = oracle.sur_loss_grad([(w.pos, w.box, e, f) for w, e, f in zip(ws, eref, fref)], SPEC,
                             fold(th, gmu, ginv), w_e=w_e, w_f=w_f)
    assert abs(loss[0] - o["loss_e"]) <= 1e-4 * o["loss_e"] + 1e-9
    assert abs(loss[1] - o["loss_f"]) <= 1e-4 * o["loss_f"]
    go = o["grad"].copy()
    if standardised:
        # chain rule from raw-descriptor parameters to standardised ones
        W1g = go[:H1 * NB].reshape(H1, NB)
        b1g = go[H1 * NB:H1 * NB + H1]
        go[:H1 * NB] = (W1g * ginv[None, :] - b1g[:, None] * (ginv * gmu)[None, :]).ravel()
    assert np.abs(grad - go).max() <= 2e-4 * np.abs(go).max()


def test_first_adam_step_matches_its_definition():
    ws, eref, fref = frames(k=2)
    th, gmu, ginv = params(8, scale=1.0)
    lr = 1e-3
    with md.SurrogateBatch(ws, th, gmu, ginv) as b:
        b.set_reference(eref, np.concatenate(fref))
        _, g = b.loss_grad(0, 2, 1.0, 1.0)
        b.train(1, 2, lr, 1.0, 1.0, seed=0)            # one minibatch = both frames
        th1, _, _ = b.sur_params()
    w1, _, _ = oracle.adam_step(th.astype(np.float64), g.astype(np.float64), np.zeros_like(g, np.float64),
                                np.zeros_like(g, np.float64), 1, lr)
    assert np.abs(th1 - w1).max() <= 1e-6


def test_adam_steps_beyond_the_first_match_the_oracle():
    """Six single-iteration training calls on one full minibatch: before each, the GPU gradient
    at the current parameters (md_sur_loss_grad) feeds the oracle's Adam, whose moments carry
    over; each GPU update must land on the oracle's parameters.  From step 2 on the bias
    corrections no longer cancel, so this checks both decay rates and the step count."""
    ws, eref, fref = frames(k=2, seed=70)
    th, gmu, ginv = params(12, scale=1.0)
    lr = 1e-3
    with md.SurrogateBatch(ws, th, gmu, ginv) as b:
        b.set_reference(eref, np.concatenate(fref))
        w = th.astype(np.float64)
        m = np.zeros_like(w)
        v = np.zeros_like(w)
        for t in range(1, 7):
            _, g = b.loss_grad(0, 2, 1.0, 1.0)
            w_ref, m, v = oracle.adam_step(b.sur_params()[0].astype(np.float64), g.astype(np.float64), m, v, t, lr)
            b.train(1, 2, lr, 1.0, 1.0, seed=t)
            th_t = b.sur_params()[0]
            assert np.abs(th_t - w_ref).max() <= 2e-6 * lr / 1e-3, t


def test_training_lowers_the_loss_and_is_deterministic():
    ws, eref, fref = frames(k=6, seed=90)
    th, _, _ = params(9, scale=0.5)
    res = []
    for _ in range(2):
        with md.SurrogateBatch(ws, th) as b:
            b.standardize()
            b.set_reference(eref, np.concatenate(fref))
            l0, _ = b.loss_grad(0, 6, 1.0, 1.0)
            b.train(300, 2, 3e-3, 1.0, 1.0, seed=11)
            l1, _ = b.loss_grad(0, 6, 1.0, 1.0)
            res.append((l0.sum(), l1.sum(), b.sur_params()[0]))
    assert res[0][1] < 0.5 * res[0][0]
    assert np.array_equal(res[0][2], res[1][2])


# --------------------------------------------------------------------------- edge cases
def test_single_atom_and_empty_system():
    th, gmu, ginv = params(10)
    w1 = I.bcc_fe(5, seed=1)
    one = I.Workload(name="one", pos=w1.pos[:1].copy(), vel=np.zeros((1, 3)), species=w1.species[:1].copy(),
                     box=w1.box, potential=w1.potential, skin=0.3, k_max=32, dt_fs=1.0, steps=1,
                     temperature=0.0)
    for net in ("fp32", "bf16"):
        with md.SurrogateSystem(one, th, gmu, ginv, net=net) as s:
            pe = s.eam_forces()
            assert np.abs(s.forces()).max() == 0.0
            # no neighbours: G = 0, so E = f((0 - gmu) ginv)
            o = oracle.sur_mlp(np.zeros((1, NB)), SPEC, fold(th, gmu, ginv))[0][0]
            assert abs(pe - o) <= (2e-5 if net == "fp32" else 0.02) * max(1.0, abs(o))
    empty = I.Workload(name="empty", pos=np.zeros((0, 3)), vel=np.zeros((0, 3)), species=np.zeros(0, np.int32),
                       box=w1.box, potential=w1.potential, skin=0.3, k_max=32, dt_fs=1.0, steps=1,
                       temperature=0.0)
    with md.SurrogateSystem(empty, th, gmu, ginv, net="bf16") as s:
        assert s.eam_forces() == 0.0
        s.step(3)


def test_surrogate_rejects_eam_only_calls_and_bad_spec():
    w = fe(5)
    th, gmu, ginv = params(11)
    with md.SurrogateSystem(w) as s:
        with pytest.raises(md.MDError) as e:
            s.eam_forces()                     # no network yet
        assert e.value.status == md.MD_ERR_STATE
        bad = dict(SPEC, rd=3.9)
        with pytest.raises(md.MDError):
            md.md_set_surrogate(s.ctx, md.make_surrogate(bad), th)
        s.set_surrogate(th, gmu, ginv)
        with pytest.raises(md.MDError):
            s.get(md.MD_GET_RHO)
        with pytest.raises(md.MDError):
            s.loss_grad()                      # no references


# --------------------------------------------------------------------------- the trained network
WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(__file__), "..", "paper_1107_2619_gb300",
                                     "data", "surrogate_fe.npz")


def _fresh_frame(T, seed):
    """A thermalised 2,000-atom bcc Fe frame from the oracle (seeds outside the training set)."""
    import dataclasses
    w = I.bcc_fe(10, seed=seed, temperature=2.0 * T, sigma=0.0)
    st = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, 1.0, 300, 0.3, 32)
    o = oracle.forces(st["pos"], w.species, w.box, w.potential)
    return dataclasses.replace(w, pos=st["pos"], vel=st["vel"]), o


def test_trained_surrogate_reproduces_eam_and_beats_the_untrained_network():
    d = np.load(WEIGHTS)
    th, gmu, ginv = d["theta"], d["gmu"], d["ginv"]
    untrained = I.sur_init_weights(5, SPEC).astype(np.float32)
    untrained[-1] = th[-1]
    for T, seed in ((450.0, 7001), (900.0, 7002), (1350.0, 7003)):
        w, o = _fresh_frame(T, seed)
        frms = np.sqrt((o["force"] ** 2).mean())
        err = {}
        for label, theta in (("trained", th), ("untrained", untrained)):
            for net in ("bf16", "fp32"):
                with md.SurrogateSystem(w, theta, gmu, ginv, net=net) as s:
                    pe = s.eam_forces()
                    F = s.forces()
                err[label, net] = (np.sqrt(((F - o["force"]) ** 2).mean()), abs(pe - o["pe"]) / w.n_atoms)
        for net in ("bf16", "fp32"):
            f_rmse, e_err = err["trained", net]
            assert f_rmse < 0.01 and f_rmse < 0.02 * frms, (T, net, f_rmse)
            assert e_err < (5e-3 if net == "bf16" else 1e-3), (T, net, e_err)
            assert err["untrained", net][0] > 10.0 * f_rmse

def test_trained_surrogate_conserves_energy():
    """NVE from a thermalised state: drift of the total energy per atom over 500 steps of 1 fs.
    (From a perfect lattice every atom has the same descriptors, so the bf16 network's rounding
    errors in E add up coherently instead of averaging out: an offset of ~5e-4 eV/atom in the
    first energy, not a drift; the FP32 network is checked from that start too.)"""
    import dataclasses
    d = np.load(WEIGHTS)
    w = I.bcc_fe(12, seed=8, temperature=1200.0, sigma=0.0)
    with md.System(w, precision="fp64") as s:
        s.eam_forces()
        s.step(400)
        wt = dataclasses.replace(w, pos=s.positions(), vel=s.velocities())
    for start, net, bound in ((wt, "bf16", 2e-5), (wt, "fp32", 1e-5), (w, "fp32", 1e-4)):
        with md.SurrogateSystem(start, d["theta"], d["gmu"], d["ginv"], net=net) as s:
            s.eam_forces()
            e0 = s.energy()
            s.step(500)
            e1 = s.energy()
        assert abs(e1["te"] - e0["te"]) / w.n_atoms < bound, (net, e1["te"] - e0["te"])
        assert e1["n_rebuilds"] > e0["n_rebuilds"]       # atoms moved: lists were rebuilt on the way
        assert 300.0 < e1["temperature"] < 900.0
