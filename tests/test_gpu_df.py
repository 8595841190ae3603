"""The double-float precision (md.h MD_PREC_DF: pair and density terms as pairs of FP32 numbers on
the FP32 pipes) against the FP64 oracle at the FP64 path's own bars: forces, energies, virial and
rho within 1e-10 relative (max-norm), trajectories within 1e-9 Å, neighbour lists exact, at
every lane count, in the step kernel as benchmarked at full size (fcc Cu 500,000 atoms), under
the predictor-corrector, in a batch of replicas, and the combinations it does not take."""
import numpy as np
import pytest

import oracle
from paper_1107_2619_gb300 import inputs as I, md

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1107_2619_gb300 import build
    build.build()


def _check_forces(w, s, pe, pos=None, box=None):
    pos = w.pos if pos is None else pos
    box = w.box if box is None else box
    ref = oracle.forces(pos, w.species, box, w.potential, skin=w.skin, k_max=w.k_max, method="cells")
    f = s.forces()
    fs = np.abs(ref["force"]).max()
    assert np.abs(f - ref["force"]).max() <= TOL * fs
    assert abs(pe - ref["pe"]) <= TOL * abs(ref["pe"])
    return ref


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("case", ["cu", "fe"])
def test_forces_energies_virial_match_oracle(lanes, case):
    w = I.fcc_cu(8, seed=2, sigma=0.03) if case == "cu" else I.bcc_fe(10, seed=11, tables=True)
    with md.System(w, precision="df", lanes_per_atom=lanes) as s:
        pe = s.eam_forces()
        e = s.energy()
        rho = s.get(md.MD_GET_RHO)
        ref = _check_forces(w, s, pe)
    assert np.abs(rho - ref["rho"]).max() <= TOL * np.abs(ref["rho"]).max()
    ws = np.abs(ref["virial"]).max()
    assert np.abs(e["virial"] - ref["virial"]).max() <= TOL * ws


def test_trajectory_with_rebuilds_matches_oracle():
    """fcc Cu 8^3 tables, 40 velocity-Verlet steps in one launch with rebuilds every 8."""
    w = I.fcc_cu(8, seed=5, sigma=0.03)
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 40, w.skin,
                        w.k_max, rebuild_every=8)
    with md.System(w, precision="df", rebuild_every=8) as s:
        s.step(40)
        pos, vel, e = s.positions(), s.velocities(), s.energy()
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert np.abs(vel - ref["vel"]).max() < 1e-11
    assert abs(e["pe"] - ref["energies"][-1, 0]) <= TOL * abs(ref["energies"][-1, 0])
    assert abs(e["ke"] - ref["energies"][-1, 1]) <= 1e-9 * ref["energies"][-1, 1]


def test_predictor_corrector_matches_oracle():
    w = I.bcc_fe(8, seed=6, tables=True)
    ref = oracle.run_pc3(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 50, w.skin,
                         w.k_max)
    with md.System(w, precision="df", integrator="pc3") as s:
        s.step(50)
        pos = s.positions()
    assert np.abs(pos - ref["pos"]).max() < 1e-9


def test_batch_of_replicas_matches_oracle():
    ws = [I.bcc_fe(5 + r, seed=3200 + r, temperature=300.0 + 400.0 * r, tables=True) for r in range(3)]
    with md.Batch(ws, precision="df") as b:
        b.step(30)
        pos = b.positions()
    o = np.concatenate([[0], np.cumsum([w.n_atoms for w in ws])])
    for r, w in enumerate(ws):
        ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 30, w.skin,
                            w.k_max)
        assert np.abs(pos[o[r]:o[r + 1]] - ref["pos"]).max() < 1e-9, r


def test_full_size_cu500k_step_kernel_as_benchmarked():
    """fcc Cu 50^3 = 500,000 atoms (180.75 Å box: the largest coordinates of the benchmark), the
    autotuner's lanes, one persistent launch of 30 steps with rebuilds: the last force pass at the
    GPU's own final positions, the energies and every neighbour list against the oracle."""
    w = I.fcc_cu(50, seed=2)
    with md.System(w, precision="df") as s:
        s.eam_forces()
        s.tune()
        s.step(30)
        e = s.energy()
        pos = s.positions()
        ref = _check_forces(w, s, e["pe"], pos=pos)
        s.build_neighbours()
        cg = s.get(md.MD_GET_NBR_COUNT)
    assert e["n_rebuilds"] >= 1
    assert np.array_equal(cg, ref["count"])


def test_combinations_it_does_not_take():
    for w in (I.bcc_fe(6, seed=7), I.bcc_fe_c(6, seed=8)):   # analytic FS; two species
        with pytest.raises(md.MDError) as ex:
            md.System(w, precision="df")
        assert ex.value.status == md.MD_ERR_ARG
    with pytest.raises(md.MDError) as ex:
        md.System(I.fcc_cu(7, seed=9), precision="df", passes="staged")
    assert ex.value.status == md.MD_ERR_ARG
