"""Parity of the CUDA path with the FP64 CPU oracle, element by element, on
identical seeded inputs, through the C ABI.

Tolerances (FP64 sweeps): contact keys, colours, normals and gaps bit-exact
(both sides round the same expressions the same way); impulses and
velocities after a step within 1e-10 relative to their largest magnitude
(the two sides differ only by FMA contraction and summation order, ~1e-16
per operation, and Gauss-Seidel does not amplify it beyond a few orders);
positions within 1e-12 of the box scale.  FP32 sweeps: stated per workload
below."""
import math

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


def _pair(nb, oracle_mod, sc, solver="persistent"):
    return nb.Scene(sc, solver=solver), oracle_mod.OracleScene(sc)


def _assert_same_contacts(cg, co, exact_geometry=True):
    assert len(cg["j1"]) == len(co["j1"])
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    if exact_geometry:
        assert np.array_equal(cg["xi"], co["xi"])
        assert np.array_equal(cg["normal"], co["normal"])


def _rel_close(a, b, rel=REL):
    scale = max(float(np.abs(b).max()) if b.size else 0.0, 1e-300)
    err = float(np.abs(a - b).max()) if b.size else 0.0
    assert err <= rel * scale, (err, scale)


def _step_and_compare(g, o, sweeps, tol=0.0, rel=REL, exact=True):
    sg = g.step(sweeps, tol)
    so = o.step(sweeps, tol)
    assert sg["n_contacts"] == so["n_contacts"]
    assert sg["n_colours"] == so["n_colours"]
    cg, co = g.get_contacts(), o.get_contacts()
    _assert_same_contacts(cg, co, exact_geometry=exact)
    if exact:
        assert np.array_equal(cg["colour"], co["colour"])
    _rel_close(cg["impulse"], co["impulse"], rel)
    bg, bo = g.get_bodies(), o.get_bodies()
    _rel_close(bg["vel"], bo["vel"], rel)
    _rel_close(bg["angvel"], bo["angvel"], rel)
    assert np.abs(bg["pos"] - bo["pos"]).max() <= 1e-12 * max(1.0, np.abs(bo["pos"]).max())
    assert np.abs(bg["quat"] - bo["quat"]).max() <= 1e-12
    return sg, so, bo


# ---------------------------------------------------------------------------
# per-step parity on the workloads
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("solver", ["persistent", "per_colour"])
def test_config1_steps_match_oracle(nb, oracle_mod, solver):
    """1,000 spheres, FP64, 50 sweeps: 5 steps, each from the oracle's state."""
    sc = scenes.config1(0)
    g, o = _pair(nb, oracle_mod, sc, solver)
    for _ in range(5):
        sg, so, bo = _step_and_compare(g, o, 50)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
    assert sg["n_contacts"] > 30


def test_config1_dense_phase_matches_oracle(nb, oracle_mod):
    """Start from a state with many contacts: every sphere given a strong
    downward velocity so the hulls reach the neighbours."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc["params"]["dt"] = 2e-2
    g, o = _pair(nb, oracle_mod, sc)
    sg, _, _ = _step_and_compare(g, o, 50)
    assert sg["n_contacts"] > 2000


def test_multi_tile_ragged_pour(nb, oracle_mod):
    """9,001 polydisperse spheres (3 radix tiles with a ragged tail, many
    colouring and sweep blocks), large hulls so contacts are dense."""
    sc = scenes.loose_pour(seed=2, n=9001)
    sc["vel"] = np.random.default_rng(7).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    g, o = _pair(nb, oracle_mod, sc)
    sg, _, _ = _step_and_compare(g, o, 30)
    assert sg["n_contacts"] > 9001


def test_periodic_cloud_matches_oracle(nb, oracle_mod):
    sc = scenes.periodic_cloud(seed=11, per_side=8, dt=2e-2)
    g, o = _pair(nb, oracle_mod, sc)
    for _ in range(3):
        sg, so, bo = _step_and_compare(g, o, 25)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
    assert sg["n_contacts"] > 50


def test_hcp_contact_count_on_gpu(nb, oracle_mod):
    for nx, ny, nz in [(4, 4, 10), (6, 4, 5), (8, 8, 3)]:
        sc = scenes.hcp_packing(nx, ny, nz, dt=1e-5, tau=1e-3)
        g = nb.Scene(sc)
        assert g.detect_contacts() == nx * ny * (6 * nz - 1)


def test_tolerance_stop_matches_oracle(nb, oracle_mod):
    sc = scenes.hcp_packing(4, 4, 3, dt=1e-3, tau=1e-3, mu=0.4, tilt_deg=30.0, v0=0.1)
    g, o = _pair(nb, oracle_mod, sc)
    for obj in (g, o):
        obj.detect_contacts()
        obj.colour_contacts()
    kg, rg = g.solve_nbgs(6000, 1e-8)
    ko, ro = o.solve_nbgs(6000, 1e-8)
    assert abs(kg - ko) <= 1 and rg <= 1e-8
    hg, ho = g.residual_history(), o.residual_history()
    m = min(len(hg), len(ho))
    assert np.allclose(hg[:m], ho[:m], rtol=1e-6, atol=1e-14)
    rg_, ro_ = g.final_residuals(), o.final_residuals()
    for k in rg_:
        assert abs(rg_[k] - ro_[k]) <= 1e-6 * max(1.0, ro_[k]) + 1e-9, (k, rg_[k], ro_[k])


def test_warm_start_matches_oracle(nb, oracle_mod):
    sc = scenes.column(5, dt=1e-3, warm_start="prev")
    sc["params"]["tau"] = 0.01
    g, o = _pair(nb, oracle_mod, sc)
    for _ in range(4):
        sg = g.step(3)
        so = o.step(3)
    cg, co = g.get_contacts(), o.get_contacts()
    _rel_close(cg["impulse"], co["impulse"], 1e-9)


def test_empty_scene_and_no_contacts(nb, oracle_mod):
    sc = scenes.sphere_on_plane(gap=1.0)
    g = nb.Scene(sc)
    st = g.step(10, 1e-6)
    assert st["n_contacts"] == 0 and st["n_colours"] == 0
    empty = scenes._scene("empty", scenes.default_params(box_lo=(0, 0, 0), box_hi=(4, 4, 4)), np.zeros((0, 3)),
                          np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0), np.zeros(0), [])
    g = nb.Scene(empty)
    assert g.step(5)["n_contacts"] == 0


# ---------------------------------------------------------------------------
# known-answer tests on the GPU
# ---------------------------------------------------------------------------

def test_T1_T2_on_gpu(nb):
    sc = scenes.sphere_on_plane(dt=1e-3)
    g = nb.Scene(sc)
    for _ in range(200):
        g.step(10, stats=False)
    b = g.get_bodies()
    assert abs(b["pos"][0, 2] - 0.5) <= 1e-12 and np.abs(b["vel"]).max() <= 1e-15
    sc = scenes.head_on(dt=0.01, gap=0.01)
    m = sc["density"] * 4.0 / 3.0 * math.pi * sc["radius"] ** 3
    g = nb.Scene(sc)
    g.step(20)
    b = g.get_bodies()
    assert abs((b["vel"][0, 0] - b["vel"][1, 0]) - 1.0) < 1e-14
    g.step(20)
    b = g.get_bodies()
    vcm = (m[0] * 1.0 + m[1] * -0.5) / m.sum()
    assert np.allclose(b["vel"][:, 0], vcm, rtol=1e-14, atol=1e-15)


def test_T3_rolling_on_gpu(nb):
    mu, g_, v0, dt, r = 0.3, 9.81, 1.0, 1e-3, 0.5
    g = nb.Scene(scenes.sliding(v0=v0, mu=mu, dt=dt, radius=r))
    for _ in range(300):
        g.step(5, stats=False)
    b = g.get_bodies()
    assert abs(b["vel"][0, 0] - 5.0 / 7.0 * v0) < 1e-12


def test_T4_momentum_on_gpu(nb):
    sc = scenes.periodic_cloud(seed=5, per_side=6, periodic=(0, 0, 0), dt=2e-2)
    m = sc["density"] * 4.0 / 3.0 * math.pi * sc["radius"] ** 3
    I = 0.4 * m * sc["radius"] ** 2
    g = nb.Scene(sc)
    b0 = g.get_bodies()
    P0 = (m[:, None] * b0["vel"]).sum(0)
    L0 = (np.cross(b0["pos"], m[:, None] * b0["vel"]) + I[:, None] * b0["angvel"]).sum(0)
    scale = (m[:, None] * np.abs(sc["vel"])).sum()
    for _ in range(10):
        g.step(20, stats=False)
    b = g.get_bodies()
    P1 = (m[:, None] * b["vel"]).sum(0)
    L1 = (np.cross(b["pos"], m[:, None] * b["vel"]) + I[:, None] * b["angvel"]).sum(0)
    assert np.abs(P1 - P0).max() <= 1e-13 * scale
    assert np.abs(L1 - L0).max() <= 1e-11 * scale


def test_T6_column_on_gpu(nb):
    k, dt, gr = 6, 1e-3, 9.81
    sc = scenes.column(k, dt=dt)
    m = sc["density"][0] * 4.0 / 3.0 * math.pi * sc["radius"][0] ** 3
    g = nb.Scene(sc)
    g.detect_contacts()
    g.colour_contacts()
    ks, R = g.solve_nbgs(20000, 1e-13)
    assert R <= 1e-13
    c = g.get_contacts()
    for j1, j2, p in zip(c["j1"], c["j2"], c["impulse"][:, 0]):
        above = k - j1 if j2 == k else k - j2
        assert abs(p - above * m * gr * dt) < 1e-9 * k * m * gr * dt


# ---------------------------------------------------------------------------
# FP32 sweeps
# ---------------------------------------------------------------------------

def test_fp32_sweep_error_vs_fp64_oracle(nb, oracle_mod):
    """FP32 sweeps with FP64 positions: contact sets, colours and geometry
    are still exact when both start from the same float-representable
    velocities; impulses and velocities agree to FP32 accuracy (1e-4 of the
    largest magnitude after 30 sweeps)."""
    sc = scenes.loose_pour(seed=4, n=6000)
    rng = np.random.default_rng(8)
    sc["vel"] = rng.normal(0.0, 2.0, sc["vel"].shape).astype(np.float32).astype(np.float64)
    sc["params"]["dt"] = 0.05
    sc["params"]["precision"] = "fp32"
    g = nb.Scene(sc)
    o = oracle_mod.OracleScene(sc)
    sg, so = g.step(30), o.step(30)
    assert sg["n_contacts"] == so["n_contacts"] > 1000
    cg, co = g.get_contacts(), o.get_contacts()
    _assert_same_contacts(cg, co)
    assert np.array_equal(cg["colour"], co["colour"])
    _rel_close(cg["impulse"], co["impulse"], 1e-4)
    _rel_close(g.get_bodies()["vel"], o.get_bodies()["vel"], 1e-4)


def test_solver_modes_agree(nb):
    """Persistent (grid barrier) and per-colour launches relax the same
    contacts in the same colour order; they differ only in how the compiler
    contracts the arithmetic of the two kernels into FMAs (1e-12)."""
    sc = scenes.loose_pour(seed=5, n=5000)
    sc["vel"] = np.random.default_rng(9).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    out = []
    for solver in ("persistent", "per_colour"):
        g = nb.Scene(sc, solver=solver)
        g.step(20)
        out.append((g.get_bodies(), g.get_contacts()))
    _rel_close(out[0][0]["vel"], out[1][0]["vel"], 1e-12)
    _rel_close(out[0][1]["impulse"], out[1][1]["impulse"], 1e-12)
    assert np.array_equal(out[0][1]["colour"], out[1][1]["colour"])


# ---------------------------------------------------------------------------
# conical hopper walls
# ---------------------------------------------------------------------------

def test_hopper_cone_contacts_match_oracle(nb, oracle_mod):
    """Oracle steps a small hopper until spheres rest on the cone face and
    fall through the orifice; from that state (oracle output as input) one
    step on each side: contact sets, cone normals and gaps bit-exact,
    colours exact, impulses and velocities within 1e-10."""
    sc = scenes.hopper(2500, seed=3, dt=2e-3)
    o = oracle_mod.OracleScene(sc)
    for _ in range(220):   # 0.44 s: ~200 cone and ~100 sphere-sphere contacts
        o.step(20)
    b = o.get_bodies()
    g = nb.Scene(sc)
    g.set_bodies(b["pos"], b["quat"], b["vel"], b["angvel"])
    sg, so, _ = _step_and_compare(g, o, 30)
    c = g.get_contacts()
    n = len(sc["radius"])
    cone_rows = c["j2"] == n + 1
    assert cone_rows.sum() > 100 and sg["n_contacts"] > cone_rows.sum() + 50


def test_hopper_rim_contacts_match_oracle(nb, oracle_mod):
    """Spheres placed under the orifice, pressed against the rim from below
    by an upward gravity: rim contacts (orifice circle) on both sides."""
    sc = scenes.hopper(400, seed=4, dt=2e-3)
    a = math.radians(30.0)
    z_o = 2.0 / math.tan(a)
    rng = np.random.default_rng(11)
    k = 12
    phi = np.linspace(0.0, 2.0 * math.pi, k, endpoint=False)
    ring = np.stack([1.9 * np.cos(phi), 1.9 * np.sin(phi), np.full(k, z_o - 0.45)], -1) + rng.uniform(-0.01, 0.01, (k, 3))
    sc["pos"] = np.concatenate([ring, sc["pos"][k:]])
    sc["params"]["gravity"] = (0.0, 0.0, 9.81)
    g, o = _pair(nb, oracle_mod, sc)
    for _ in range(3):   # each step from the oracle's state
        _, _, bo = _step_and_compare(g, o, 30)
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])
    c = o.get_contacts()
    n = len(sc["radius"])
    rim = (c["j2"] == n + 1) & (c["j1"] < k)
    assert rim.sum() >= k // 2
    # a rim contact's normal points from the orifice circle towards the centre
    assert np.all(c["normal"][rim][:, 2] < 0.0)


def test_sphere_rests_in_cone_on_gpu(nb):
    sc = scenes.sphere_in_cone(radius=0.5, half_angle_deg=30.0, dt=1e-3)
    g = nb.Scene(sc)
    z0 = sc["pos"][0, 2]
    for _ in range(200):
        g.step(10, stats=False)
    b = g.get_bodies()
    assert abs(b["pos"][0, 2] - z0) <= 1e-12 and np.abs(b["vel"]).max() <= 1e-15
    c = g.get_contacts()
    m = 4.0 / 3.0 * math.pi * 0.5 ** 3
    assert len(c["j1"]) == 1 and abs(c["impulse"][0, 0] - m * 9.81 * 1e-3) < 1e-15


def test_colouring_buffers_grow_between_steps(nb, oracle_mod):
    """A step with few contacts sizes the contact buffers; the next step
    has many more contacts (large hulls), so the buffers grow (the
    colouring's lists with them): the result still equals the oracle's."""
    sc = scenes.config1(0)
    g, o = _pair(nb, oracle_mod, sc)
    sg, so, bo = _step_and_compare(g, o, 20)
    few = sg["n_contacts"]
    vel = np.random.default_rng(21).normal(0.0, 40.0, bo["vel"].shape)
    for obj in (g, o):
        obj.set_bodies(bo["pos"], bo["quat"], vel, bo["angvel"])
    sg, so, _ = _step_and_compare(g, o, 20)
    assert sg["n_contacts"] > 20 * max(few, 1)


def test_warp_scheduling_matches_oracle(nb, oracle_mod):
    """NBGS_SWEEP_WARP_SYNC (every warp waits only for the warps whose
    contacts share its bodies) relaxes the same colours in the same order:
    parity with the oracle as for the block-level scheduling."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc["params"]["dt"] = 2e-2
    sc["params"]["sweep_flags"] = 4
    g, o = _pair(nb, oracle_mod, sc)
    sg, _, _ = _step_and_compare(g, o, 50)
    assert sg["n_contacts"] > 2000


def test_warp_and_block_scheduling_agree(nb):
    sc = scenes.loose_pour(seed=6, n=20000)
    sc["vel"] = np.random.default_rng(12).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    sc["params"]["precision"] = "fp32"
    sc["params"]["warm_start"] = "prev"
    out = []
    for flags in (0, 4):
        sc["params"]["sweep_flags"] = flags
        g = nb.Scene(sc)
        for _ in range(3):
            g.step(30)
        out.append((g.get_bodies(), g.get_contacts()))
    assert np.array_equal(out[0][1]["colour"], out[1][1]["colour"])
    _rel_close(out[0][0]["vel"], out[1][0]["vel"], 1e-5)
    _rel_close(out[0][1]["impulse"], out[1][1]["impulse"], 1e-5)
