"""The surrogate as a torch.autograd.Function (paper_1107_2619_gb300.autograd): its energy and
gradient against the oracle's FP64 evaluation of the same network, against central differences
of its own energy, the chain rule through it, and a descent step on the positions.  The network
is the FP32 one (md_surrogate MD_SUR_FP32), so that finite differences resolve the gradient."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

SPEC = dict(I.SUR_FE)


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()
    return t


def _net(seed=21):
    nb, h1 = SPEC["nb"], SPEC["h1"]
    th = I.sur_init_weights(seed, SPEC, scale=1.5).astype(np.float32)
    rng = np.random.default_rng(seed)
    th[h1 * nb:h1 * nb + h1] = rng.normal(0, 0.3, h1).astype(np.float32)
    th[-1] = np.float32(-4.0)
    gmu = rng.uniform(0.0, 3.0, nb).astype(np.float32)
    ginv = rng.uniform(0.3, 1.5, nb).astype(np.float32)
    return th, gmu, ginv


def _fold(th, gmu, ginv):
    nb, h1 = SPEC["nb"], SPEC["h1"]
    t = np.asarray(th, np.float64).copy()
    W1 = t[:h1 * nb].reshape(h1, nb) * np.asarray(ginv, np.float64)[None, :]
    t[h1 * nb:h1 * nb + h1] -= W1 @ np.asarray(gmu, np.float64)
    t[:h1 * nb] = W1.ravel()
    return t


def test_energy_and_gradient_match_the_oracle(torch):
    from paper_1107_2619_gb300.autograd import SurrogateEnergy
    w = I.bcc_fe(6, seed=31, temperature=600.0, sigma=0.1)
    th, gmu, ginv = _net()
    ref = oracle.surrogate(w.pos, w.box, SPEC, _fold(th, gmu, ginv), k_max=64)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda", requires_grad=True)
        U = SurrogateEnergy.apply(pos, s)
        U.backward()
        g = pos.grad.cpu().numpy()
        f_lib = s.forces()
    assert abs(U.item() - ref["energy"]) <= 2e-5 * w.n_atoms
    assert np.array_equal(g, -f_lib)
    assert np.abs(-g - ref["force"]).max() <= 1e-4 * np.abs(ref["force"]).max()


def test_gradient_matches_central_differences_of_the_energy(torch):
    """Directional derivatives along seeded random displacement fields: (U(r + h d) - U(r - h d)) / 2h
    against <dU/dr, d>, h = 1e-3 Å (the list is kept: the displacements stay inside the skin)."""
    from paper_1107_2619_gb300.autograd import SurrogateEnergy
    w = I.bcc_fe(6, seed=32, temperature=600.0, sigma=0.1)
    th, gmu, ginv = _net(22)
    h = 1e-3
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda", requires_grad=True)
        U = SurrogateEnergy.apply(pos, s)
        (g,) = torch.autograd.grad(U, pos)
        for k in range(4):
            d = torch.tensor(I.random_normal(500 + k, 1, 3 * w.n_atoms).reshape(-1, 3), dtype=torch.float64,
                             device="cuda")
            up = SurrogateEnergy.apply(pos.detach() + h * d, s).item()
            um = SurrogateEnergy.apply(pos.detach() - h * d, s).item()
            fd = (up - um) / (2 * h)
            an = float((g * d).sum())
            assert abs(fd - an) <= 2e-3 * max(1.0, abs(an)), (k, fd, an)


def test_chain_rule_and_a_descent_step(torch):
    """The incoming gradient scales the returned one (a loss 3 U gives -3 F), and gradient descent
    on the positions through the Function lowers the energy."""
    from paper_1107_2619_gb300.autograd import SurrogatePotential
    w = I.bcc_fe(5, seed=33, temperature=300.0, sigma=0.12)
    th, gmu, ginv = _net(23)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        model = SurrogatePotential(s)
        pos = torch.tensor(w.pos, dtype=torch.float64, device="cuda", requires_grad=True)
        (3.0 * model(pos)).backward()
        f = model.forces(pos)
        assert torch.equal(pos.grad, -3.0 * f)
        opt = torch.optim.SGD([pos], lr=2e-3)
        u0 = model(pos).item()
        for _ in range(5):
            opt.zero_grad()
            model(pos).backward()
            opt.step()
        assert model(pos).item() < u0


def test_rejects_host_or_single_precision_positions(torch):
    from paper_1107_2619_gb300.autograd import SurrogateEnergy
    w = I.bcc_fe(5, seed=34)
    th, gmu, ginv = _net(24)
    with md.SurrogateSystem(w, th, gmu, ginv, net="fp32") as s:
        with pytest.raises(ValueError):
            SurrogateEnergy.apply(torch.tensor(w.pos, dtype=torch.float64), s)
        with pytest.raises(ValueError):
            SurrogateEnergy.apply(torch.tensor(w.pos, dtype=torch.float32, device="cuda"), s)
