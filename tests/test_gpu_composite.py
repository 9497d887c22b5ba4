"""Composite particles on the GPU against the FP64 oracle, through the C ABI.

Bit-exact from one state: member contact keys, gaps, normals (the member
positions X + R(q) d are rounded as written on both sides) and colours.
Impulses and velocities after a step with FP64 sweeps: 1e-10 relative to the
largest, positions and orientations likewise (the one-contact solve brackets
the same sliding roots and refines them differently: bisection on the host,
Newton steps inside the bracket on the device)."""
import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu

REL = 1e-10


@pytest.fixture(scope="module")
def nb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def _rel_close(a, b, rel=REL):
    scale = max(float(np.abs(b).max()) if b.size else 0.0, 1e-300)
    err = float(np.abs(a - b).max()) if b.size else 0.0
    assert err <= rel * scale, (err, scale)


def _with(sc, **kw):
    return dict(sc, params=dict(sc["params"], **kw))


def _step_and_compare(g, o, sweeps, tol=0.0, rel=REL, exact=True):
    sg = g.step(sweeps, tol)
    so = o.step(sweeps, tol)
    assert sg["n_contacts"] == so["n_contacts"]
    assert sg["n_colours"] == so["n_colours"]
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    if exact:
        assert np.array_equal(cg["xi"], co["xi"]) and np.array_equal(cg["normal"], co["normal"])
        assert np.array_equal(cg["colour"], co["colour"])
        assert sg["sweeps_done"] == so["sweeps_done"]
    _rel_close(cg["impulse"], co["impulse"], rel)
    bg, bo = g.get_bodies(), o.get_bodies()
    _rel_close(bg["vel"], bo["vel"], rel)
    _rel_close(bg["angvel"], bo["angvel"], rel)
    # positions and orientations move by dt v' and dt Q w' / 2: they inherit
    # the velocities' tolerance
    assert np.abs(bg["pos"] - bo["pos"]).max() <= rel * max(1.0, np.abs(bo["pos"]).max())
    assert np.abs(bg["quat"] - bo["quat"]).max() <= rel
    return sg, so, bo


def _pile(seed=1, **kw):
    """Composites of 2-4 members falling onto each other in a walled box."""
    sc = scenes.composite_gas(6, 5, 5, seed=seed, spacing=1.02, v_max=0.5, dt=2e-2, mu=0.4, omega=1.0,
                              gravity=(0.0, 0.0, -9.81), **kw)
    sc["vel"][:, 2] -= 3.0
    return sc


@pytest.mark.parametrize("schedule", ["windows", "global"])
@pytest.mark.parametrize("mu", [0.4, 0.05])
def test_composite_pile_matches_oracle(nb, oracle_mod, mu, schedule):
    """Both schedules of the composite sweep: dependency windows between
    blocks, or a grid barrier after every colour."""
    flags = nb.NBGS_SWEEP_GLOBAL_SYNC if schedule == "global" else 0
    sc = _with(_pile(), mu=mu, sweep_flags=flags)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for _ in range(4):
        sg, so, bo = _step_and_compare(g, o, 40)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
    assert sg["n_contacts"] > 150


def test_composite_periodic_cloud_with_tolerance(nb, oracle_mod):
    sc = scenes.composite_gas(5, 5, 4, seed=6, spacing=1.02, v_max=1.5, walls=False, dt=2e-2, periodic=(1, 1, 1),
                              omega=0.8)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    total = 0
    for _ in range(4):
        sg, so, bo = _step_and_compare(g, o, 300, tol=1e-9)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
        total += sg["n_contacts"]
    assert total > 40


def test_composite_warm_start(nb, oracle_mod):
    sc = _with(_pile(seed=3), warm_start="prev")
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for k in range(3):   # later steps start from the previous impulses
        _step_and_compare(g, o, 30, rel=REL if k == 0 else 1e-9, exact=k == 0)


def test_fp32_composite_sweeps_against_fp64_oracle(nb, oracle_mod):
    sc = _pile(seed=4)
    g = nb.Scene(_with(sc, precision="fp32"))
    o = oracle_mod.OracleScene(sc)
    g.step(40, 0.0)
    o.step(40, 0.0)
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["colour"], co["colour"])
    _rel_close(cg["impulse"], co["impulse"], 2e-4)
    _rel_close(g.get_bodies()["vel"], o.get_bodies()["vel"], 2e-4)


def test_dumbbell_rests_on_gpu(nb):
    dt, gr = 1e-3, 9.81
    sc = scenes.dumbbell_on_plane(dt=dt)
    s = nb.Scene(sc)
    m = 2 * 4.0 / 3.0 * np.pi * 0.5 ** 3
    for _ in range(20):
        st = s.step(200, 1e-14)
        assert st["n_contacts"] == 2
    c = s.get_contacts()
    assert np.abs(c["impulse"][:, 0] - 0.5 * m * gr * dt).max() <= 1e-10 * m * gr * dt
    b = s.get_bodies()
    assert np.abs(b["vel"]).max() <= 1e-12 and np.abs(b["angvel"]).max() <= 1e-12


def test_free_spin_matches_oracle(nb, oracle_mod):
    """The gyroscopic term of eq. (integrationscheme) and the FP64
    orientation update, 300 steps without contacts."""
    sc = scenes.spinning_body(dt=1e-3)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for _ in range(300):
        g.step(1)
        o.step(1)
    bg, bo = g.get_bodies(), o.get_bodies()
    _rel_close(bg["angvel"], bo["angvel"], 1e-12)
    assert np.abs(bg["quat"] - bo["quat"]).max() <= 1e-12


def test_single_member_composites_on_gpu_equal_spheres(nb):
    """The composite path on one-member bodies against the sphere path on
    the GPU: the same contacts and colours, impulses to rounding."""
    sc = scenes.hcp_packing(4, 4, 3, dt=1e-3, tau=1e-3, mu=0.4, tilt_deg=30.0, v0=0.1)
    a, b = nb.Scene(sc), nb.Scene(scenes.as_composites(sc))
    for _ in range(3):
        a.step(30)
        b.step(30)
    ca, cb = a.get_contacts(), b.get_contacts()
    assert np.array_equal(ca["j1"], cb["j1"]) and np.array_equal(ca["colour"], cb["colour"])
    _rel_close(cb["impulse"], ca["impulse"], 1e-10)
    _rel_close(b.get_bodies()["vel"], a.get_bodies()["vel"], 1e-10)


def test_composite_rejections(nb, tmp_path):
    """What composites do not take fails with NBGS_EINVAL (the first error
    sticks in its scene, so one scene per call)."""
    calls = [lambda s: s.set_subdomains("jacobi"), lambda s: s.save_state(str(tmp_path / "x.ckpt")),
             lambda s: (s.step(5), s.final_residuals())]
    for call in calls:
        s = nb.Scene(scenes.dumbbell_on_plane())
        with pytest.raises(nb.NBGSError) as e:
            call(s)
        assert e.value.status == nb.NBGS_EINVAL


def test_composite_creation_checks_its_arguments(nb):
    good = scenes.dumbbell_on_plane()
    nb.Scene(good).close()
    bad = [dict(good, density=np.array([0.0])),
           dict(good, members=dict(good["members"], body=np.array([0, 1], np.int32))),
           dict(good, members=dict(good["members"], radius=np.array([0.5, -0.1]))),
           dict(good, params=dict(good["params"], subdomains="jacobi"))]
    for sc in bad:
        with pytest.raises(nb.NBGSError):
            nb.Scene(sc)
