"""Pins of the oracle's learned-surrogate functions to facts outside the oracle (CPU only).

The descriptor is pinned by shell sums over a perfect fcc lattice; the network's per-atom
energy and input gradient by PyTorch float64 autograd; forces by central differences of
the total energy, by Newton's third law (zero net force) and, for a gradient that is the
same for every atom, by the equivalent pair potential summed over all pairs; the training
loss gradient by central differences of the loss; Adam by its first-step closed form.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1107_2619_gb300 import inputs as I

SPEC = dict(I.SUR_FE)


def basis_np(r, spec=SPEC):
    mu = spec["mu0"] + spec["dmu"] * np.arange(spec["nb"])
    fc = 0.5 * (np.cos(np.pi * r / spec["rd"]) + 1.0) * (r < spec["rd"])
    return np.exp(-((r[..., None] - mu) ** 2) / (2 * spec["width"] ** 2)) * fc[..., None]


def small_fe(n=4, sigma=0.08, seed=11, a=2.8665):
    w = I.bcc_fe(n, seed=seed, sigma=sigma, a=a)
    return w.pos, w.box


def test_descriptor_of_perfect_fcc_equals_shell_sum():
    a = 3.615
    w = I.fcc_cu(4, seed=1, sigma=0.0, a=a, n_knots=50)
    count, nl, _ = oracle.neighbours(w.pos, w.box, 4.3, 80, "cells")
    G = oracle.sur_descriptors(w.pos, w.box, count, nl, SPEC)
    shells = [(12, a / math.sqrt(2)), (6, a), (24, a * math.sqrt(1.5))]   # 3rd shell 4.43 Å > 4.3 Å
    expect = sum(z * basis_np(np.array([r]))[0] for z, r in shells[:2])
    assert np.allclose(G, expect[None, :], rtol=1e-12, atol=1e-14)


def test_mlp_energy_and_input_gradient_match_torch_autograd():
    rng = np.random.default_rng(3)
    G = rng.normal(size=(50, SPEC["nb"])) * 0.7
    wts = I.sur_init_weights(7, SPEC) + 0.05 * rng.normal(size=I.sur_n_params(SPEC))
    E, g = oracle.sur_mlp(G, SPEC, wts)
    nb, h1, h2 = SPEC["nb"], SPEC["h1"], SPEC["h2"]
    t = torch.tensor(wts)
    o = 0
    W1 = t[o:o + h1 * nb].view(h1, nb); o += h1 * nb
    b1 = t[o:o + h1]; o += h1
    W2 = t[o:o + h2 * h1].view(h2, h1); o += h2 * h1
    b2 = t[o:o + h2]; o += h2
    w3 = t[o:o + h2]; o += h2
    b3 = t[o]
    x = torch.tensor(G, requires_grad=True)
    e = torch.nn.functional.silu(torch.nn.functional.silu(x @ W1.T + b1) @ W2.T + b2) @ w3 + b3
    e.sum().backward()
    assert np.allclose(E, e.detach().numpy(), rtol=1e-13, atol=1e-13)
    assert np.allclose(g, x.grad.numpy(), rtol=1e-12, atol=1e-13)


def _energy(pos, box, wts, spec=SPEC):
    return oracle.surrogate(pos, box, spec, wts, k_max=64, method="brute")["energy"]


def test_surrogate_forces_are_minus_energy_gradient():
    pos, box = small_fe()
    wts = I.sur_init_weights(5, SPEC, scale=2.0)
    out = oracle.surrogate(pos, box, SPEC, wts, k_max=64, method="brute")
    h = 1e-5
    rng = np.random.default_rng(0)
    for i in rng.choice(len(pos), 6, replace=False):
        for a in range(3):
            p1, p2 = pos.copy(), pos.copy()
            p1[i, a] += h
            p2[i, a] -= h
            fd = -(_energy(p1, box, wts) - _energy(p2, box, wts)) / (2 * h)
            assert abs(fd - out["force"][i, a]) < 1e-7 * max(1.0, abs(fd))


def test_surrogate_net_force_is_zero():
    pos, box = small_fe(n=5)
    out = oracle.surrogate(pos, box, SPEC, I.sur_init_weights(9, SPEC, scale=2.0))
    assert np.abs(out["force"].sum(axis=0)).max() < 1e-11 * np.abs(out["force"]).sum()


def test_constant_gradient_gives_pair_potential_forces():
    """With g_i = c for every atom the force is that of the pair potential 2 c.b(r), all pairs."""
    pos, box = small_fe(n=3)
    count, nl, _ = oracle.neighbours(pos, box, 4.3, 80, "brute")
    c = np.linspace(-1.0, 1.0, SPEC["nb"])
    F = oracle.sur_forces(pos, box, count, nl, SPEC, np.tile(c, (len(pos), 1)))
    d = pos[None, :, :] - pos[:, None, :]
    d -= box * np.rint(d / box)
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, 1.0)
    h = 1e-6
    dphi = (basis_np(r + h) - basis_np(r - h)) @ c / (2 * h)    # d/dr of c.b(r)
    np.fill_diagonal(dphi, 0.0)
    expect = (2.0 * dphi / r)[..., None] * d
    assert np.allclose(F, expect.sum(axis=1), rtol=1e-7, atol=1e-9)


def test_descriptor_is_zero_and_flat_at_the_cutoff():
    r = np.array([SPEC["rd"] - 1e-6, SPEC["rd"]])
    b = basis_np(r)
    assert np.abs(b).max() < 1e-10


def _frames(n_frames=2, n=5):
    frames = []
    for s in range(n_frames):
        pos, box = small_fe(n=n, seed=20 + s, sigma=0.1)
        rng = np.random.default_rng(s)
        frames.append((pos, box, -4.0 * len(pos) + rng.normal(), rng.normal(size=pos.shape) * 0.3))
    return frames


def test_loss_gradient_matches_finite_differences():
    frames = _frames()
    wts = I.sur_init_weights(4, SPEC, scale=1.5)
    out = oracle.sur_loss_grad(frames, SPEC, wts, w_e=1.0, w_f=2.0)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(I.sur_n_params(SPEC), 14, replace=False), [I.sur_n_params(SPEC) - 1]])
    for p in idx:
        h = 1e-6
        w1, w2 = wts.copy(), wts.copy()
        w1[p] += h
        w2[p] -= h
        fd = (oracle.sur_loss_grad(frames, SPEC, w1, 1.0, 2.0)["loss"]
              - oracle.sur_loss_grad(frames, SPEC, w2, 1.0, 2.0)["loss"]) / (2 * h)
        assert abs(fd - out["grad"][p]) < 2e-6 * max(1.0, abs(fd)), (p, fd, out["grad"][p])


def test_loss_is_the_stated_mean_squares():
    frames = _frames()
    wts = I.sur_init_weights(4, SPEC)
    out = oracle.sur_loss_grad(frames, SPEC, wts, w_e=0.5, w_f=3.0)
    le, lf, nat = 0.0, 0.0, 0
    for pos, box, e, f in frames:
        s = oracle.surrogate(pos, box, SPEC, wts)
        le += ((s["energy"] - e) / len(pos)) ** 2
        lf += ((s["force"] - f) ** 2).sum()
        nat += len(pos)
    assert math.isclose(out["loss_e"], 0.5 * le / len(frames), rel_tol=1e-12)
    assert math.isclose(out["loss_f"], 3.0 * lf / (3 * nat), rel_tol=1e-12)


def test_adam_first_step_is_signed_learning_rate():
    g = np.array([3.0, -1e-3, 2.5e4])
    w, m, v = oracle.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(w, -0.01 * np.sign(g), rtol=1e-14)


def test_adam_constant_gradient_moves_by_the_learning_rate_at_every_step():
    """With the same gradient at every step the bias-corrected moments are exactly g and g^2
    (m_t = (1 - beta1^t) g, v_t = (1 - beta2^t) g^2), so with eps = 0 every step is -lr sign(g).
    A wrong bias-correction exponent, beta1 and beta2 exchanged in a correction, or a moment
    without its (1 - beta) factor moves by another amount from step 2 on."""
    g = np.array([3.0, -1e-3, 2.5e4, -7.0])
    w, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 31):
        w1, m, v = oracle.adam_step(w, g, m, v, t, lr=0.01, eps=0.0)
        assert np.allclose(w1 - w, -0.01 * np.sign(g), rtol=1e-12, atol=0), t
        w = w1


def test_adam_second_step_after_a_zero_gradient_closed_form():
    """g_1 = g, g_2 = 0: m_2 = beta1 (1 - beta1) g and v_2 = beta2 (1 - beta2) g^2, so the bias-
    corrected moments are beta1 g / (1 + beta1) and beta2 g^2 / (1 + beta2), and the second
    step is lr (beta1 / (1 + beta1)) / sqrt(beta2 / (1 + beta2)) sign(g) = 0.670058... lr sign(g)
    for beta1 = 0.9, beta2 = 0.999 (eps = 0).  This fixes the two decay rates, which a constant
    gradient does not."""
    g = np.array([2.0, -0.5])
    w, m, v = oracle.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, lr=1.0, eps=0.0)
    w2, _, _ = oracle.adam_step(w, np.zeros(2), m, v, 2, lr=1.0, eps=0.0)
    step = (0.9 / 1.9) / math.sqrt(0.999 / 1.999)
    assert abs(step - 0.6700583) < 1e-6
    assert np.allclose(w - w2, step * np.sign(g), rtol=1e-13, atol=0)


def test_adam_is_invariant_to_the_gradient_scale():
    """With eps = 0 the update depends on the gradients only through their ratios."""
    rng = np.random.default_rng(3)
    gs = rng.normal(size=(8, 5))
    wa = wb = np.zeros(5)
    ma = va = mb = vb = np.zeros(5)
    for t in range(1, 9):
        wa, ma, va = oracle.adam_step(wa, gs[t - 1], ma, va, t, lr=0.1, eps=0.0)
        wb, mb, vb = oracle.adam_step(wb, 1e3 * gs[t - 1], mb, vb, t, lr=0.1, eps=0.0)
    assert np.allclose(wa, wb, rtol=1e-12, atol=1e-15)
