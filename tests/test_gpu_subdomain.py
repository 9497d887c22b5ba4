"""Subdomain NBGS and non-linear block Jacobi (Alg. 1 with s_c(j); the
velocity corrections of Sect. 6.3) on the GPU against the FP64 oracle,
through the C ABI.

Bit-exact: contact keys, gaps, normals, s_c(j), colours.  Impulses and
velocities after a step: 1e-10 relative to their largest magnitude (FP64
sweeps).  The two sides add the corrections in the same subdomain order; the
GPU forms each subdomain's correction as the difference of its instance and
the accumulator, the oracle accumulates it directly, which differs by
rounding (~1e-16 per sweep)."""
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


def _step_and_compare(g, o, sweeps, tol=0.0, rel=REL, exact=True):
    """One step on both sides.  exact: the two started from the same state,
    so the geometry is bit-exact; otherwise (a warm-started run carried over
    several steps, whose states differ by rounding) it is compared within rel
    and the sweep counts may differ by one where R_k sits at the tolerance."""
    sg = g.step(sweeps, tol)
    so = o.step(sweeps, tol)
    assert sg["n_contacts"] == so["n_contacts"]
    assert sg["n_colours"] == so["n_colours"]
    assert abs(sg["sweeps_done"] - so["sweeps_done"]) <= (0 if exact else 1)
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    if exact:
        assert np.array_equal(cg["xi"], co["xi"]) and np.array_equal(cg["normal"], co["normal"])
    else:
        _rel_close(cg["xi"], co["xi"], rel)
        _rel_close(cg["normal"], co["normal"], rel)
    assert np.array_equal(cg["colour"], co["colour"])
    assert np.array_equal(g.get_subdomains().astype(np.int64), o.contact_subdomains())
    _rel_close(cg["impulse"], co["impulse"], rel)
    bg, bo = g.get_bodies(), o.get_bodies()
    _rel_close(bg["vel"], bo["vel"], rel)
    _rel_close(bg["angvel"], bo["angvel"], rel)
    assert np.abs(bg["pos"] - bo["pos"]).max() <= 1e-12 * max(1.0, np.abs(bo["pos"]).max())
    return sg, so, bo


def _with(sc, **kw):
    return dict(sc, params=dict(sc["params"], **kw))


@pytest.mark.parametrize("solver", ["persistent", "per_colour"])
@pytest.mark.parametrize("sub,omega", [((2, 2, 2), 1.0), ((3, 2, 1), 0.75), ("jacobi", 0.5), ("jacobi", 1.0)])
def test_config1_subdomains_match_oracle(nb, oracle_mod, solver, sub, omega):
    """1,000 spheres, FP64, 50 sweeps, 4 steps each from the oracle's state,
    a compressed start so that many contacts cross subdomain borders."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2, subdomains=sub, omega=omega)
    g, o = nb.Scene(sc, solver=solver), oracle_mod.OracleScene(sc)
    for _ in range(4):
        sg, so, bo = _step_and_compare(g, o, 50)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
    assert sg["n_contacts"] > 1500
    if sub == "jacobi":
        assert sg["n_colours"] == 1


def test_multi_tile_ragged_subdomains(nb, oracle_mod):
    """9,001 polydisperse spheres (ragged tiles of every pass), a 4 x 3 x 5
    grid, warm start from the previous step."""
    sc = scenes.loose_pour(seed=2, n=9001)
    sc["vel"] = np.random.default_rng(7).normal(0.0, 2.0, sc["vel"].shape)
    sc = _with(sc, dt=0.05, subdomains=(4, 3, 5), omega=0.9, warm_start="prev")
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for k in range(2):   # the second step starts from the first one's impulses
        sg, so, bo = _step_and_compare(g, o, 30, rel=REL if k == 0 else 1e-9, exact=k == 0)
    assert sg["n_contacts"] > 9001
    assert len(np.unique(g.get_subdomains())) == 60


def test_periodic_jacobi_with_warm_start_and_tolerance(nb, oracle_mod):
    sc = _with(scenes.periodic_cloud(seed=11, per_side=8, dt=2e-2), subdomains="jacobi", omega=0.6,
               warm_start="prev")
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for k in range(3):
        sg, so, bo = _step_and_compare(g, o, 400, tol=1e-7, rel=REL if k == 0 else 1e-9, exact=k == 0)
    assert sg["n_contacts"] > 50
    assert 0 < sg["sweeps_done"] < 400


@pytest.mark.parametrize("flags", ["warp", "global", "tma"])
@pytest.mark.parametrize("sub", [(2, 3, 2), "jacobi"])
def test_sweep_schedules_with_subdomains(nb, oracle_mod, flags, sub):
    """Every schedule of the persistent solver: warps with per-sweep grid
    barriers around the reduction, a grid barrier after every colour, and the
    default block windows (here with the shared-memory stage), where the
    reduction is a windowed phase of its own."""
    f = {"warp": nb.NBGS_SWEEP_WARP_SYNC, "global": nb.NBGS_SWEEP_GLOBAL_SYNC, "tma": nb.NBGS_SWEEP_TMA_STAGE}[flags]
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2, subdomains=sub, omega=0.6, sweep_flags=f)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for _ in range(2):
        sg, so, bo = _step_and_compare(g, o, 50)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])


def test_fp32_subdomain_sweeps_against_fp64_oracle(nb, oracle_mod):
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2, subdomains=(2, 2, 2), precision="fp32")
    g = nb.Scene(sc)
    o = oracle_mod.OracleScene(_with(sc, precision="fp64"))
    g.step(50, 0.0)
    o.step(50, 0.0)
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["colour"], co["colour"])
    _rel_close(cg["impulse"], co["impulse"], 1e-4)
    _rel_close(g.get_bodies()["vel"], o.get_bodies()["vel"], 1e-4)


def test_jacobi_column_on_gpu(nb):
    """T6 under non-linear block Jacobi: the unique weights i m g dt."""
    kcol, dt, g = 6, 1e-3, 9.81
    sc = scenes.column(kcol, dt=dt, subdomains="jacobi", omega=0.5)
    m = sc["density"][0] * 4.0 / 3.0 * np.pi * sc["radius"][0] ** 3
    s = nb.Scene(sc)
    st = s.step(100000, 1e-13)
    assert st["residual"] <= 1e-13 and st["n_colours"] == 1
    c = s.get_contacts()
    for j1, j2, p in zip(c["j1"], c["j2"], c["impulse"][:, 0]):
        above = kcol - j1 if j2 == kcol else kcol - j2
        assert abs(p - above * m * g * dt) < 1e-9 * kcol * m * g * dt


@pytest.mark.parametrize("sub", [(2, 2, 2), "jacobi"])
def test_subdomain_momentum_on_gpu(nb, sub):
    sc = scenes.periodic_cloud(seed=5, per_side=6, periodic=(1, 1, 1), dt=2e-2, subdomains=sub, omega=0.7)
    s = nb.Scene(sc)
    m = sc["density"] * 4.0 / 3.0 * np.pi * sc["radius"] ** 3
    P0 = (m[:, None] * s.get_bodies()["vel"]).sum(0)
    scale = (m[:, None] * np.abs(sc["vel"])).sum()
    total = 0
    for _ in range(8):
        total += s.step(20, 0.0)["n_contacts"]
        P1 = (m[:, None] * s.get_bodies()["vel"]).sum(0)
        assert np.abs(P1 - P0).max() <= 1e-13 * scale
    assert total > 100


def test_switching_modes_on_a_live_scene(nb, oracle_mod):
    """set_subdomains between steps: each step equals the oracle run in the
    mode of that step from the same state."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2, omega=0.8)
    g = nb.Scene(sc)
    for sub in ("jacobi", (2, 1, 2), None, "jacobi"):
        b = g.get_bodies()
        o = oracle_mod.OracleScene(_with(sc, subdomains=sub))
        o.set_bodies(b["pos"], b["quat"], b["vel"], b["angvel"])
        g.set_subdomains(sub)
        _step_and_compare(g, o, 40)


def test_network_features_do_not_depend_on_subdomains(nb):
    """The learned warm start reads bodies, not the sweep's instances."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2)
    feats = []
    for sub in (None, (2, 2, 2), "jacobi"):
        s = nb.Scene(_with(sc, subdomains=sub))
        s.detect_contacts()
        s.colour_contacts()
        feats.append(s.mlp_features())   # canonical order
    assert np.array_equal(feats[0], feats[1]) and np.array_equal(feats[0], feats[2])


def test_checkpoint_resume_with_subdomains(nb, tmp_path):
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc = _with(sc, dt=2e-2, subdomains=(2, 2, 1), warm_start="prev", omega=0.9)
    a = nb.Scene(sc)
    for _ in range(2):
        a.step(30, 0.0)
    path = str(tmp_path / "sub.ckpt")
    a.save_state(path)
    b = nb.Scene(_with(sc, subdomains=None))
    b.load_state(path)
    for _ in range(2):
        a.step(30, 0.0)
        b.step(30, 0.0)
    ba, bb = a.get_bodies(), b.get_bodies()
    assert np.array_equal(ba["vel"], bb["vel"]) and np.array_equal(ba["pos"], bb["pos"])
    assert np.array_equal(a.get_subdomains(), b.get_subdomains())


def test_bad_subdomain_arguments(nb):
    sc = scenes.column(3)
    with pytest.raises(Exception):
        nb.Scene(_with(sc, subdomains=(0, 1, 1)))
    s = nb.Scene(sc)
    with pytest.raises(nb.NBGSError):
        s.set_subdomains((1, -1, 1))
    bs = scenes.batch_scenes(2, seed=0)
    g = nb.BatchScene(bs)
    with pytest.raises(nb.NBGSError):
        g.set_subdomains("jacobi")
