"""The benchmark workloads at their full sizes, in the launch configuration the
benchmark times, checked where the oracle cannot follow them whole:
properties that hold at any size, and outputs recomputed one by one.

- Dense 1M packing (HCP 100^3, FP32 sweeps, 100 sweeps): the contact count
  is n_x n_y (6 n_z - 1); no colour holds two contacts of one body; every
  impulse lies in its friction cone with p_n >= 0; the gap and normal of
  sampled contacts equal their FP64 definition recomputed here (same
  operation order, so bit for bit).
- Settled 1M-sphere pour (the benchmark's default): colours, cones, sampled
  geometry bit for bit.
- 4,096-scene batch: no contact joins two scenes; every scene's bodies stay
  in its box.
- 30M-sphere gas: the contacts found obey the keep rule of Sect. 4,
  recomputed for a sample, and the contact set of a step is unique.
- Completeness (pour, gas, batch, settled hopper): inside random sub-boxes
  the oracle's brute-force detection on the bodies there finds exactly the
  GPU's contacts among them, walls and cones included, bit for bit.
- Every workload (dense, pour, ramp, gas, batch, hopper): FP32 sweeps
  against FP64 sweeps from the same state, within about ten times the error
  measured on a GB300.
- 1M-body composite pile: no contact inside a body, colours valid over bodies,
  cones, sampled member-pair geometry from the body state bit for bit.
- 1M ramp on a 16 x 16 x 1 subdomain grid: sampled s_c(j) bit for bit, every
  cell used, colours valid."""
import math

import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def _check_colouring(c, n):
    col = c["colour"]
    assert col.min() >= 0
    for k in np.unique(col):
        rows = col == k
        b = np.concatenate([c["j1"][rows], c["j2"][rows][c["j2"][rows] < n]])
        assert len(np.unique(b)) == len(b), f"colour {k} touches a body twice"


def _check_cone(c, mu, rel=1e-5):
    p = c["impulse"]
    scale = max(float(np.abs(p[:, 0]).max()), 1e-300)
    assert p[:, 0].min() >= -rel * scale
    assert np.all(np.hypot(p[:, 1], p[:, 2]) <= mu * p[:, 0] + rel * scale)


def _subbox_complete(oracle_mod, sc, b0, c, n, rng, wall_index, boxes=4, side=8.0, min_inside=40, idx_pool=None,
                     floor=False):
    """Completeness of the full-size detection inside random sub-boxes: the
    oracle's brute-force detection (every pair, every wall) run on the
    bodies whose centres lie in a sub-box, with their start-of-step state
    (hence the same hulls), must find exactly the GPU's contacts between
    those bodies and the walls, with the same gaps and normals bit for bit.
    A dropped neighbour cell or a missed wall anywhere in a box fails.
    wall_index(k) maps the oracle scene's wall k to the GPU's body index;
    idx_pool restricts the bodies (one scene of a batch); floor puts every
    sub-box on the floor of the box (z from box_lo)."""
    from paper_1501_05810_gb300 import workloads
    pos = b0["pos"]
    lo = np.array(sc["params"]["box_lo"], dtype=np.float64)
    hi = np.array(sc["params"]["box_hi"], dtype=np.float64)
    pool = np.arange(len(pos)) if idx_pool is None else idx_pool
    key_gpu = (c["j1"].astype(np.int64) << 32) | c["j2"].astype(np.int64)
    found = 0
    for _ in range(boxes):
        for _attempt in range(50):
            corner = rng.uniform(lo, np.maximum(lo, hi - side))
            if floor:
                corner[2] = lo[2]
            inside = np.all((pos[pool] >= corner) & (pos[pool] < corner + side), axis=1)
            if inside.sum() >= min_inside:
                break
        idx = pool[inside]
        m = len(idx)
        sub = workloads.cut(dict(sc, pos=pos, vel=b0["vel"], angvel=b0["angvel"]), np.isin(np.arange(len(pos)), idx))
        o = oracle_mod.OracleScene(sub)
        o.detect_contacts()
        co = o.get_contacts()
        o.close()
        j2 = co["j2"].astype(np.int64)
        g1 = idx[co["j1"].astype(np.int64)]
        g2 = np.where(j2 < m, idx[np.minimum(j2, m - 1)], np.array([wall_index(k) for k in (j2 - m)], dtype=np.int64)
                      if len(j2) else j2)
        k_or = (g1 << 32) | g2
        order = np.argsort(k_or)
        member = np.zeros(len(pos) + 1, bool)
        member[idx] = True
        jg2 = c["j2"].astype(np.int64)
        mask = member[c["j1"]] & ((jg2 >= n) | member[np.minimum(jg2, len(pos))])
        assert np.array_equal(k_or[order], key_gpu[mask]), (len(k_or), int(mask.sum()))
        assert np.array_equal(co["xi"][order], c["xi"][mask])
        assert np.array_equal(co["normal"][order], c["normal"][mask])
        found += len(k_or)
    assert found > 0
    return found


def test_dense_packing_full_size(nb):
    sc = scenes.dense_packing(1_000_000, seed=0, precision="fp32")
    g = nb.Scene(sc)
    b0 = g.get_bodies()
    st = g.step(100, 1e-6)
    assert st["n_contacts"] == 100 * 100 * (6 * 100 - 1)
    c = g.get_contacts()
    n = len(sc["radius"])
    _check_colouring(c, n)
    _check_cone(c, sc["params"]["mu"])
    # sampled sphere-sphere contacts: the geometry from the start-of-step positions
    rng = np.random.default_rng(1)
    ss = np.nonzero(c["j2"] < n)[0]
    pick = rng.choice(ss, 2000, replace=False)
    a, b = c["j1"][pick].astype(np.int64), c["j2"][pick].astype(np.int64)
    lo, hi = np.array(sc["params"]["box_lo"]), np.array(sc["params"]["box_hi"])
    L = hi - lo
    d3 = b0["pos"][a] - b0["pos"][b]
    for k in range(3):
        if sc["params"]["periodic"][k]:
            d3[:, k] = np.where(d3[:, k] > 0.5 * L[k], d3[:, k] - L[k],
                                np.where(d3[:, k] < -0.5 * L[k], d3[:, k] + L[k], d3[:, k]))
    d = np.sqrt((d3[:, 0] * d3[:, 0] + d3[:, 1] * d3[:, 1]) + d3[:, 2] * d3[:, 2])
    r = sc["radius"]
    assert np.array_equal(c["xi"][pick], (d - r[a]) - r[b])
    assert np.array_equal(c["normal"][pick], d3 / d[:, None])


def test_settled_pour_full_size(nb, oracle_mod):
    """The benchmark's default workload (the settled 1M-sphere pour, FP32
    sweeps, 100 sweeps or residual 1e-6, previous-step warm start) in its
    launch configuration: valid colouring, impulses in their cones, sampled
    gaps and normals equal to their FP64 definition bit for bit, and the
    contact set complete inside sub-boxes against the oracle's brute force
    (walls included)."""
    from paper_1501_05810_gb300 import workloads
    sc = workloads.settled_pour(1_000_000, precision="fp32")
    sc["params"] = dict(sc["params"], warm_start="prev")
    g = nb.Scene(sc)
    for _ in range(3):
        g.step(100, 1e-6)
    b0 = g.get_bodies()
    st = g.step(100, 1e-6)
    n = len(sc["radius"])
    assert st["n_contacts"] > 2_000_000 and st["sweeps_done"] >= 1
    c = g.get_contacts()
    _check_colouring(c, n)
    _check_cone(c, sc["params"]["mu"])
    rng = np.random.default_rng(5)
    ss = np.nonzero(c["j2"] < n)[0]
    pick = rng.choice(ss, 2000, replace=False)
    a, b = c["j1"][pick].astype(np.int64), c["j2"][pick].astype(np.int64)
    d3 = b0["pos"][a] - b0["pos"][b]
    d = np.sqrt((d3[:, 0] * d3[:, 0] + d3[:, 1] * d3[:, 1]) + d3[:, 2] * d3[:, 2])
    r = sc["radius"]
    assert np.array_equal(c["xi"][pick], (d - r[a]) - r[b])
    assert np.array_equal(c["normal"][pick], d3 / d[:, None])
    found = _subbox_complete(oracle_mod, sc, b0, c, n, rng, lambda k: n + k, boxes=5, side=8.0)
    assert found > 1000
    # a sub-box on the floor: wall contacts too
    lo = np.array(sc["params"]["box_lo"])
    floor = dict(sc, params=dict(sc["params"], box_hi=(lo[0] + 60.0, lo[1] + 60.0, lo[2] + 8.0)))
    _subbox_complete(oracle_mod, floor, b0, c, n, rng, lambda k: n + k, boxes=2, side=8.0)


def test_batch_full_size(nb, oracle_mod):
    bs = scenes.batch_scenes(4096, seed=0, precision="fp32", contacts_per_body=4)
    g = nb.BatchScene(bs)
    for _ in range(300):   # 0.15 s: the lowest layers have reached the floor and one another
        g.step(30, 1e-6, stats=False)
    g.step(100, 1e-6)
    c = g.get_contacts()
    off = g.offsets
    scene_of = np.repeat(np.arange(len(bs)), np.diff(off))
    n = int(off[-1])
    ss = c["j2"] < n
    assert np.array_equal(scene_of[c["j1"][ss]], scene_of[c["j2"][ss]])
    pos = g.get_bodies()["pos"]
    lo = np.repeat(np.array([s["params"]["box_lo"] for s in bs]), np.diff(off), axis=0)
    hi = np.repeat(np.array([s["params"]["box_hi"] for s in bs]), np.diff(off), axis=0)
    assert np.all(pos >= lo - 0.1) and np.all(pos <= hi + 0.1)
    _check_colouring(c, n)
    # completeness inside sub-boxes of a few scenes, walls included (the
    # batch numbers each scene's six walls after all bodies: n + 6 s + k)
    b0 = g.get_bodies()
    g.detect_contacts()
    c = g.get_contacts()
    rng = np.random.default_rng(13)
    rad = np.concatenate([x["radius"] for x in bs])
    den = np.concatenate([x["density"] for x in bs])
    for si in rng.choice(len(bs), 4, replace=False):
        one = dict(bs[si], radius=rad, density=den)   # global body numbering, this scene's box and walls
        found = _subbox_complete(oracle_mod, one, b0, c, n, rng, lambda k, si=si: n + 6 * int(si) + int(k),
                                 boxes=2, side=6.0, min_inside=20, idx_pool=np.arange(off[si], off[si + 1]),
                                 floor=True)
        assert found > 0


def test_gas_full_size_keep_rule(nb, oracle_mod):
    sc = scenes.granular_gas(cells=196, seed=0, precision="fp32", contacts_per_body=2)
    g = nb.Scene(sc)
    n = len(sc["radius"])
    dt, tau = sc["params"]["dt"], sc["params"]["tau"]
    for _ in range(200):   # the gas starts without contacts; its first collisions by then
        g.step(50, 0.0, stats=False)
    b0 = g.get_bodies()
    nc = g.detect_contacts()
    assert nc > 0
    c = g.get_contacts()
    key = (c["j1"].astype(np.int64) << 32) | c["j2"].astype(np.int64)
    assert np.all(np.diff(key) > 0)                      # canonical order, no duplicates
    # the velocities are FP32 in the scene: the hull of Sect. 4 from them
    v = b0["vel"].astype(np.float32).astype(np.float64)
    w = b0["angvel"].astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(2)
    pick = rng.choice(len(key), min(5000, len(key)), replace=False)
    a, b = c["j1"][pick].astype(np.int64), c["j2"][pick].astype(np.int64)
    r = sc["radius"]
    h = lambda i: dt * (np.sqrt((v[i, 0] ** 2 + v[i, 1] ** 2) + v[i, 2] ** 2)
                        + np.sqrt((w[i, 0] ** 2 + w[i, 1] ** 2) + w[i, 2] ** 2) * r[i]) + tau
    L = np.array(sc["params"]["box_hi"]) - np.array(sc["params"]["box_lo"])
    d3 = b0["pos"][a] - b0["pos"][b]
    d3 = np.where(d3 > 0.5 * L, d3 - L, np.where(d3 < -0.5 * L, d3 + L, d3))
    d = np.sqrt((d3[:, 0] ** 2 + d3[:, 1] ** 2) + d3[:, 2] ** 2)
    slack = 1e-12 * np.max(L)
    assert np.all((d - r[a]) - r[b] <= h(a) + h(b) + slack)
    # and nothing is missing: brute force inside sub-boxes (no walls here)
    sc_b = dict(sc)
    found = _subbox_complete(oracle_mod, sc_b, b0, c, n, np.random.default_rng(12), lambda k: n + k, boxes=5,
                             side=14.0)
    assert found >= 20


# FP32 sweeps against FP64 sweeps from one state, per workload: the error
# measured on a GB300 (largest difference relative to the largest value after
# one step) and the bound held here, about ten times the measurement.
FP32_BOUND = {            # (impulses, velocities); measured
    "dense": (7e-6, 2e-5),      # 6.7e-7, 1.9e-6
    "hopper": (5e-5, 2e-5),     # 4.2e-6, 1.5e-6
    "pour": (1.1e-5, 2.5e-5),   # 1.1e-6, 2.5e-6
    "ramp": (9e-2, 5e-3),       # 8.8e-3, 4.7e-4: dt = 1e-5 makes the impulses tiny against the bulk velocity
    "gas": (9e-6, 2e-6),        # 8.3e-7, 1.2e-7
    "batch": (2e-5, 1.2e-5),    # 2.0e-6, 1.2e-6
}


def _fp32_case(nb, workload):
    """(scene or scene list, pre-steps, pre-step sweeps, sweeps of the
    compared step, minimum contacts) of a workload at its full size."""
    if workload == "dense":
        return scenes.dense_packing(1_000_000, seed=0), 0, 0, 100, 5_000_000
    if workload == "hopper":   # the settled state the hopper discharge is measured on
        return scenes.hopper(2_000_000, seed=0, warm_start="prev"), 2000, 30, 100, 300_000
    if workload == "pour":
        from paper_1501_05810_gb300 import workloads
        sc = workloads.settled_pour(1_000_000)
        return sc, 0, 0, 100, 2_000_000
    if workload == "ramp":
        return scenes.hcp_packing(100, 100, 100, dt=1e-5, tau=0.005, mu=0.85, tilt_deg=30.0, v0=0.1, omega=0.75,
                                  warm_start="prev"), 0, 0, 100, 5_000_000
    if workload == "gas":   # its first collisions after 200 steps
        return scenes.granular_gas(cells=196, seed=0, contacts_per_body=2), 200, 50, 50, 1_000
    return scenes.batch_scenes(4096, seed=0, contacts_per_body=4, warm_start="prev"), 400, 30, 100, 500_000


@pytest.mark.parametrize("workload", sorted(FP32_BOUND))
def test_fp32_sweeps_against_fp64_at_full_size(nb, oracle_mod, workload):
    """The error of FP32 sweeps (FP64 positions) against FP64 sweeps on the
    same state at full size, after one step: FP64 sweeps match the oracle to
    1e-10 at every size the oracle can run, so this is the FP32 error against
    the FP64 reference for the configuration.  The pre-steps that bring a
    workload into its regime run in FP64; the hopper's settled state is also
    checked for completeness of its contact set (cone walls included)."""
    sc, pre, pre_sweeps, sweeps, min_contacts = _fp32_case(nb, workload)
    batch = isinstance(sc, list)

    def make(prec):
        if batch:
            return nb.BatchScene([dict(x, params=dict(x["params"], precision=prec)) for x in sc])
        return nb.Scene(dict(sc, params=dict(sc["params"], precision=prec)))

    out = {}
    state = None
    for prec in ("fp64", "fp32"):
        g = make(prec)
        if state is None:
            for _ in range(pre):   # FP64 once, then shared
                g.step(pre_sweeps, 0.0, stats=False)
            state = g.get_bodies()
            if workload == "hopper":
                g.detect_contacts()
                n = len(sc["radius"])
                _subbox_complete(oracle_mod, sc, state, g.get_contacts(), n, np.random.default_rng(14),
                                 lambda k: n + k, boxes=4, side=8.0)
        g.set_bodies(state["pos"], state["quat"], state["vel"], state["angvel"])
        g.step(sweeps, 0.0)
        out[prec] = (g.get_bodies(), g.get_contacts())
        g.close()
    (b64, c64), (b32, c32) = out["fp64"], out["fp32"]
    # the FP32 scene holds FP32 velocities, so its hulls differ in the last
    # bits: compare the contacts both found (a borderline pair may differ)
    k64 = (c64["j1"].astype(np.int64) << 32) | c64["j2"]
    k32 = (c32["j1"].astype(np.int64) << 32) | c32["j2"]
    common, i64, i32 = np.intersect1d(k64, k32, assume_unique=True, return_indices=True)
    assert len(k64) > min_contacts
    assert len(common) >= (1.0 - 1e-4) * max(len(k64), len(k32))
    ep = np.abs(c32["impulse"][i32] - c64["impulse"][i64]).max() / np.abs(c64["impulse"]).max()
    ev = np.abs(b32["vel"] - b64["vel"]).max() / max(np.abs(b64["vel"]).max(), 1e-300)
    print(f"{workload}: {len(c64['j1'])} contacts, FP32 vs FP64 after {sweeps} sweeps: impulses {ep:.2e}, "
          f"velocities {ev:.2e} (relative to the largest)")
    bp, bv = FP32_BOUND[workload]
    assert ep < bp and ev < bv


def test_composite_pile_full_size(nb):
    """The 1M-body composite pile of the benchmark: no contact joins two
    members of one body, the colouring is valid over bodies, impulses lie in
    their cones, and sampled member-pair gaps and normals equal their FP64
    definition from the bodies' state (members at X + R(q) d, bit for bit)."""
    sc = scenes.composite_gas(100, 100, 100, seed=0, spacing=1.02, v_max=0.5, dt=2e-2, mu=0.4, omega=1.0,
                              gravity=(0.0, 0.0, -9.81), precision="fp32", contacts_per_body=8, warm_start="prev")
    sc["vel"][:, 2] -= 3.0
    g = nb.Scene(sc)
    for _ in range(3):
        g.step(50, 0.0, stats=False)
    b0 = g.get_bodies()
    st = g.step(50, 0.0)
    assert st["n_contacts"] > 1_000_000
    c = g.get_contacts()
    mb = sc["members"]["body"]
    nm = len(mb)
    mem = c["j2"] < nm
    a, bm = c["j1"].astype(np.int64), c["j2"].astype(np.int64)
    assert np.all(mb[a[mem]] != mb[bm[mem]])
    # colours over bodies
    body1 = mb[a]
    body2 = np.where(mem, mb[np.minimum(bm, nm - 1)], -1)
    for k in np.unique(c["colour"]):
        rows = c["colour"] == k
        bb = np.concatenate([body1[rows], body2[rows][body2[rows] >= 0]])
        assert len(np.unique(bb)) == len(bb), f"colour {k} touches a body twice"
    _check_cone(c, sc["params"]["mu"], rel=1e-4)
    # geometry of sampled member pairs from the start-of-step body state
    rng = np.random.default_rng(3)
    pick = rng.choice(np.nonzero(mem)[0], 2000, replace=False)

    def member_pos(m):
        i = mb[m]
        q = b0["quat"][i]
        w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
        R = np.empty((len(m), 3, 3))
        R[:, 0, 0] = 1.0 - 2.0 * (y * y + z * z); R[:, 0, 1] = 2.0 * (x * y - w * z); R[:, 0, 2] = 2.0 * (x * z + w * y)
        R[:, 1, 0] = 2.0 * (x * y + w * z); R[:, 1, 1] = 1.0 - 2.0 * (x * x + z * z); R[:, 1, 2] = 2.0 * (y * z - w * x)
        R[:, 2, 0] = 2.0 * (x * z - w * y); R[:, 2, 1] = 2.0 * (y * z + w * x); R[:, 2, 2] = 1.0 - 2.0 * (x * x + y * y)
        d = _member_offsets(sc)[m]
        rd = (R[:, :, 0] * d[:, 0:1] + R[:, :, 1] * d[:, 1:2]) + R[:, :, 2] * d[:, 2:3]
        return b0["pos"][i] + rd

    pa, pb = member_pos(a[pick]), member_pos(bm[pick])
    d3 = pa - pb
    d = np.sqrt((d3[:, 0] * d3[:, 0] + d3[:, 1] * d3[:, 1]) + d3[:, 2] * d3[:, 2])
    r = sc["members"]["radius"]
    assert np.array_equal(c["xi"][pick], (d - r[a[pick]]) - r[bm[pick]])
    assert np.array_equal(c["normal"][pick], d3 / d[:, None])


def _member_offsets(sc):
    """Members' offsets from their body's centre of mass (the masses of the
    members add up; the body's centre of mass is their weighted mean)."""
    mb, off, r = sc["members"]["body"], sc["members"]["offset"], sc["members"]["radius"]
    rho = sc["density"][mb]
    mm = rho * (4.0 / 3.0) * np.pi * r * r * r
    n = len(sc["density"])
    M = np.zeros(n)
    X = np.zeros((n, 3))
    # sequential sums in member order, as the definition writes them
    for m in range(len(mb)):
        M[mb[m]] += mm[m]
        X[mb[m]] += mm[m] * off[m]
    X /= M[:, None]
    return off - X[mb]


def test_subdomain_ramp_full_size(nb):
    """The 1M ramp on the 16 x 16 x 1 grid of the benchmark: sampled s_c(j)
    equal the cell of body j1's centre recomputed here, every cell of the
    grid holds contacts, and the colouring is valid."""
    sc = scenes.hcp_packing(100, 100, 100, dt=1e-5, tau=0.005, mu=0.85, tilt_deg=30.0, v0=0.1, omega=0.5,
                            precision="fp32", warm_start="prev", subdomains=(16, 16, 1))
    g = nb.Scene(sc)
    b0 = g.get_bodies()
    st = g.step(100, 0.0)
    assert st["n_contacts"] == 100 * 100 * (6 * 100 - 1)
    c = g.get_contacts()
    sub = g.get_subdomains()
    n = len(sc["radius"])
    _check_colouring(c, n)
    lo, hi = np.array(sc["params"]["box_lo"]), np.array(sc["params"]["box_hi"])
    gd = np.array([16, 16, 1])
    rng = np.random.default_rng(4)
    pick = rng.choice(len(sub), 20000, replace=False)
    x = b0["pos"][c["j1"][pick].astype(np.int64)]
    k = np.clip(np.floor(((x - lo) * gd) / (hi - lo)), 0, gd - 1).astype(np.int64)
    want = (k[:, 2] * gd[1] + k[:, 1]) * gd[0] + k[:, 0]
    assert np.array_equal(sub[pick].astype(np.int64), want)
    assert len(np.unique(sub)) == 256
