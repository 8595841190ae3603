"""md_step in segments (the FP64 step kernel on systems of at least 32,768 atoms): the step kernel
stops at a step that needs a list rebuild, the cooperative rebuild kernel builds the list (§3.2.1)
and a launch resumes the call at that step; rebuilds beyond the segments enqueued fall back to the
step kernel's own rebuild phases.  Trajectories with frequent rebuilds against the oracle at the
FP64 bars (positions within 1e-9 Å, energies within 1e-10), in both FP64 walks, across two calls,
under the strain ramp and the thermostat, and with the profiling stamps on."""
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


def _cu():
    w = I.fcc_cu(21, seed=41, sigma=0.02, temperature=600.0)   # 37,044 atoms
    assert w.n_atoms >= 32768
    return w


@pytest.mark.parametrize("walk", ["list", "half"])
def test_rebuild_every_other_step_across_two_calls(walk):
    """14 steps with a rebuild every second step (more rebuilds than the first call enqueues
    segments), then 6 more in a second call: positions and energies against one oracle run."""
    w = _cu()
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 20, w.skin,
                        w.k_max, rebuild_every=2)
    with md.System(w, precision="fp64", passes=walk, rebuild_every=2) as s:
        s.step(14)
        e1 = s.energy()
        s.step(6)
        e2 = s.energy()
        pos = s.positions()
    assert e1["n_rebuilds"] >= 7 and e2["n_rebuilds"] >= e1["n_rebuilds"] + 3
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    assert abs(e1["pe"] - ref["energies"][13, 0]) <= TOL * abs(ref["energies"][13, 0])
    assert abs(e2["pe"] - ref["energies"][19, 0]) <= TOL * abs(ref["energies"][19, 0])


def test_strain_ramp():
    w = _cu()
    w.strain_rate_zz = -1.0e9
    ref = oracle.run_vv(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 12, w.skin,
                        w.k_max, rebuild_every=3, strain_rate_zz=w.strain_rate_zz)
    with md.System(w, precision="fp64", passes="half", rebuild_every=3) as s:
        s.step(12)
        e = s.energy()
        pos = s.positions()
        s.eam_forces()   # energies and virial at the final, strained state
        ev = s.energy()
    assert e["n_rebuilds"] >= 4
    assert np.array_equal(e["box"], ref["box"])
    assert np.abs(pos - ref["pos"]).max() < 1e-9
    # the pair walk's virial (atoms' x (x) F plus the image-shift terms of boundary pairs; under the
    # ramp every warp takes the minimum image) against the oracle's pair form, same state
    fv = oracle.forces(pos, w.species, e["box"], w.potential, skin=w.skin, k_max=w.k_max)
    for got in (e, ev):   # the step kernel's last step, the stand-alone passes
        assert np.abs(got["virial"] - fv["virial"]).max() <= TOL * np.abs(fv["virial"]).max()
        assert abs(got["pe"] - fv["pe"]) <= TOL * abs(fv["pe"])


def test_thermostat():
    w = I.fcc_cu(21, seed=42, sigma=0.0, temperature=300.0)
    with md.System(w, precision="fp64", passes="half") as s:
        s.set_thermostat(1500.0, tau_fs=20.0)
        s.eam_forces()
        q = s.thermostat()[0, 2]
        s.step(24)
        e = s.energy()
        pos = s.positions()
    ref = oracle.run_nvt(w.pos, w.vel, w.species, w.potential.masses, w.box, w.potential, w.dt_fs, 24, w.skin,
                         w.k_max, 1500.0, q)
    assert e["n_rebuilds"] >= 1
    assert np.abs(pos - ref["pos"]).max() < 1e-8


def test_profiling_stamps_cover_the_rebuild_kernel():
    w = _cu()
    with md.System(w, precision="fp64", passes="half", rebuild_every=2) as s:
        s.eam_forces()
        s.set_profiling(True)
        s.step(8)
        p = s.profile()
    parts = np.array(p["ms_rebuild_part"])
    assert (parts >= 0).all() and parts[-1] > 0      # the list build of the rebuild kernel is timed
    assert p["ms_density"] > 0 and p["ms_force"] > 0
    assert abs(p["ms_rebuild"] - parts.sum()) <= 1e-6 * max(1.0, p["ms_rebuild"])
