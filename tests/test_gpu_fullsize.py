"""The benchmark workloads at their full sizes, in the launch configuration the
benchmark times, checked where the oracle cannot follow them whole:
properties that hold at any size, and outputs recomputed one by one.

- Dense 1M packing (HCP 100^3, FP32 sweeps, 100 sweeps): the contact count
  is n_x n_y (6 n_z - 1); no colour holds two contacts of one body; every
  impulse lies in its friction cone with p_n >= 0; the gap and normal of
  sampled contacts equal their FP64 definition recomputed here (same
  operation order, so bit for bit).
- 4,096-scene batch: no contact joins two scenes; every scene's bodies stay
  in its box.
- 30M-sphere gas: the contacts found obey the keep rule of Sect. 4,
  recomputed for a sample, and the contact set of a step is unique.
- Dense packing and settled 2M hopper: FP32 sweeps against FP64 sweeps from
  the same state, impulses and velocities within 1e-2 of the largest.
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


def test_batch_full_size(nb):
    bs = scenes.batch_scenes(4096, seed=0, precision="fp32", contacts_per_body=4)
    g = nb.BatchScene(bs)
    for _ in range(3):
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


def test_gas_full_size_keep_rule(nb):
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


@pytest.mark.parametrize("workload", ["dense", "hopper"])
def test_fp32_sweeps_against_fp64_at_full_size(nb, workload):
    """The error of FP32 sweeps (FP64 positions) against FP64 sweeps on the
    same state at full size (the hopper after its 2,000 settling steps of 30
    sweeps), after one step of 100 sweeps: FP64 sweeps match the oracle to
    1e-10 at every size the oracle can run, so this is the FP32 error
    against the FP64 reference for the configuration."""
    if workload == "dense":
        sc = scenes.dense_packing(1_000_000, seed=0)
        pre = 0
    else:
        sc = scenes.hopper(2_000_000, seed=0, warm_start="prev")
        pre = 2000   # the settled state the hopper discharge is measured on
    out = {}
    state = None
    for prec in ("fp64", "fp32"):
        s = dict(sc, params=dict(sc["params"], precision=prec))
        g = nb.Scene(s)
        if state is None:
            for _ in range(pre):   # bring the hopper into contact (FP64 once, then shared)
                g.step(30, 0.0, stats=False)
            state = g.get_bodies()
        else:
            g.set_bodies(state["pos"], state["quat"], state["vel"], state["angvel"])
        if pre:
            g.set_bodies(state["pos"], state["quat"], state["vel"], state["angvel"])
        g.step(100, 0.0)
        out[prec] = (g.get_bodies(), g.get_contacts())
        g.close()
    (b64, c64), (b32, c32) = out["fp64"], out["fp32"]
    # the FP32 scene holds FP32 velocities, so its hulls differ in the last
    # bits: compare the contacts both found (a borderline pair may differ)
    k64 = (c64["j1"].astype(np.int64) << 32) | c64["j2"]
    k32 = (c32["j1"].astype(np.int64) << 32) | c32["j2"]
    common, i64, i32 = np.intersect1d(k64, k32, assume_unique=True, return_indices=True)
    assert len(k64) > (300_000 if pre else 5_000_000)   # the hopper: ~478k contacts after 1 s
    assert len(common) >= (1.0 - 1e-5) * max(len(k64), len(k32))
    ep = np.abs(c32["impulse"][i32] - c64["impulse"][i64]).max() / np.abs(c64["impulse"]).max()
    ev = np.abs(b32["vel"] - b64["vel"]).max() / max(np.abs(b64["vel"]).max(), 1e-300)
    print(f"{workload}: {len(c64['j1'])} contacts, FP32 vs FP64 after 100 sweeps: impulses {ep:.2e}, "
          f"velocities {ev:.2e} (relative to the largest)")
    assert ep < 1e-2 and ev < 1e-2


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
