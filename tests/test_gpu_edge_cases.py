"""GPU counterparts of the oracle's edge-case pins, each against the oracle:
a periodic box away from the origin (minimum image and wrap), coincident
centres, a zero-sweep solve, planes of general normal (spheres and
composite members), and the general one-contact solver where several
sliding states qualify and where it falls back."""
import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu

ORIGINS = [(0.0, 0.0, 0.0), (-7.5, 3.25, -2.0)]


@pytest.fixture(scope="module")
def nb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def _pair(gap, origin, ra=0.5, rb=0.3, va=(0.0, 0.0, 0.0), dt=1e-3):
    """Two spheres closing a periodic box origin + [0, 10]^3 across x = lo."""
    lo = np.asarray(origin, float)
    prm = scenes.default_params(dt=dt, tau=0.01, gravity=(0, 0, 0), box_lo=tuple(lo), box_hi=tuple(lo + 10.0),
                                periodic=(1, 1, 1))
    pos = np.array([[0.2, 5.0, 5.0], [10.0 + 0.2 - (ra + rb + gap), 5.0, 5.0]]) + lo
    return scenes._scene("pair", prm, pos, np.array([va, (0, 0, 0)], float), np.zeros((2, 3)), [ra, rb],
                         [1.0, 1.0], [])


def _same_contacts(g, o):
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    assert np.array_equal(cg["xi"], co["xi"]) and np.array_equal(cg["normal"], co["normal"])
    return cg, co


@pytest.mark.parametrize("origin", ORIGINS)
def test_periodic_box_off_the_origin(nb, oracle_mod, origin):
    """Minimum image across x = lo and the wrap of a sphere leaving through
    it, bit for bit with the oracle; a sphere that stays inside moves by
    exactly dt v (the wrap leaves it alone)."""
    sc = _pair(0.001, origin)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    assert g.detect_contacts() == o.detect_contacts() == 1
    cg, _ = _same_contacts(g, o)
    assert np.allclose(cg["normal"][0], [1, 0, 0])
    sc = _pair(1.0, origin, va=(-30.0, 0.0, 0.0), dt=0.01)
    sc["vel"][1] = [0.37, -0.11, 0.23]
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    g.step(1)
    o.step(1)
    bg, bo = g.get_bodies(), o.get_bodies()
    assert np.array_equal(bg["pos"], bo["pos"])
    lo = origin[0]
    assert lo <= bg["pos"][0, 0] < lo + 10.0 and abs(bg["pos"][0, 0] - (lo + 10.0 + 0.2 - 0.3)) < 1e-12
    assert np.array_equal(bg["pos"][1], sc["pos"][1] + 0.01 * sc["vel"][1])


@pytest.mark.parametrize("origin", ORIGINS)
def test_periodic_cloud_off_the_origin_matches_oracle(nb, oracle_mod, origin):
    """A periodic cloud shifted away from the origin: three steps, each from
    the oracle's state, contacts and geometry bit for bit, velocities to 1e-10."""
    sc = scenes.periodic_cloud(seed=11, per_side=7, dt=2e-2)
    off = np.asarray(origin)
    sc["pos"] = sc["pos"] + off
    sc["params"]["box_lo"] = tuple(np.asarray(sc["params"]["box_lo"]) + off)
    sc["params"]["box_hi"] = tuple(np.asarray(sc["params"]["box_hi"]) + off)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for _ in range(3):
        sg, so = g.step(25), o.step(25)
        assert sg["n_contacts"] == so["n_contacts"] > 20
        _same_contacts(g, o)
        bg, bo = g.get_bodies(), o.get_bodies()
        assert np.abs(bg["vel"] - bo["vel"]).max() <= 1e-10 * np.abs(bo["vel"]).max()
        assert np.abs(bg["pos"] - bo["pos"]).max() <= 1e-12 * max(1.0, np.abs(bo["pos"]).max())
        g.set_bodies(bo["pos"], bo["quat"], bo["vel"], bo["angvel"])


@pytest.mark.parametrize("composite", [False, True])
def test_coincident_centres(nb, oracle_mod, composite):
    prm = scenes.default_params(dt=1e-3, gravity=(0, 0, 0), box_lo=(-5, -5, -5), box_hi=(5, 5, 5))
    sc = scenes._scene("same", prm, np.array([[0.5, -1.0, 2.0]] * 2), np.zeros((2, 3)), np.zeros((2, 3)),
                       [0.5, 0.3], [1.0, 1.0], [])
    if composite:
        sc = scenes.as_composites(sc)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    assert g.detect_contacts() == o.detect_contacts() == 1
    cg, _ = _same_contacts(g, o)
    assert np.array_equal(cg["normal"][0], [0.0, 0.0, 1.0]) and cg["xi"][0] == -0.8


def test_zero_sweep_solve(nb, oracle_mod):
    """max_sweeps = 0: zero impulses, v' = v + dt g and x' = x + dt v', as in
    the oracle, bit for bit."""
    sc = scenes.column(3, dt=1e-3)
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    sg, so = g.step(0), o.step(0)
    assert sg["n_contacts"] == so["n_contacts"] == 3 and sg["sweeps_done"] == 0
    assert np.all(g.get_contacts()["impulse"] == 0.0)
    bg, bo = g.get_bodies(), o.get_bodies()
    for k in ("pos", "vel", "angvel"):
        assert np.array_equal(bg[k], bo[k]), k


def test_sphere_gaps_under_a_tilted_plane(nb, oracle_mod):
    rng = np.random.default_rng(31)
    n = 6
    nrm = np.array([0.48, -0.6, 0.64])
    pos = rng.uniform(-3.0, 3.0, (n, 3))
    r = rng.uniform(0.3, 0.6, n)
    prm = scenes.default_params(dt=1e-3, gravity=(0, 0, 0), tau=2.0, box_lo=(-20, -20, -20), box_hi=(20, 20, 20))
    pos[:, 0] = np.clip(pos[:, 0] + np.arange(n) * 10.0 - 25.0, -19.0, 19.0)
    c = float((pos @ nrm - r).min() - 0.2)
    sc = scenes._scene("tilted", prm, pos, np.zeros((n, 3)), np.zeros((n, 3)), r, np.ones(n), [(tuple(nrm), c)])
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    assert g.detect_contacts() == o.detect_contacts() >= 2
    _same_contacts(g, o)


def test_composite_member_gaps_under_a_tilted_plane(nb, oracle_mod):
    """A rotated asymmetric composite over a plane of general normal: the
    member-wall contacts, gaps and normals bit for bit with the oracle, and
    one step's velocities to 1e-10."""
    nrm = np.array([0.48, 0.6, 0.64])
    sc = scenes.spinning_body(angvel=(0.2, -0.4, 0.9), tau=1.0)
    rng = np.random.default_rng(8)
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    X = np.array([1.5, -2.0, 0.75])
    sc["planes"] = [(tuple(nrm), float(X @ nrm - 1.2))]
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for obj in (g, o):
        obj.set_bodies(X[None], q[None], np.array([[0.1, 0.2, -1.0]]), np.array([[0.2, -0.4, 0.9]]))
    assert g.detect_contacts() == o.detect_contacts() >= 2
    _same_contacts(g, o)
    g.step(30)
    o.step(30)
    bg, bo = g.get_bodies(), o.get_bodies()
    assert np.abs(bg["vel"] - bo["vel"]).max() <= 1e-10 * max(1.0, np.abs(bo["vel"]).max())
    assert np.abs(bg["angvel"] - bo["angvel"]).max() <= 1e-10 * max(1.0, np.abs(bo["angvel"]).max())


def _skew(v):
    return np.array([[0.0, -v[2], v[1]], [v[2], 0.0, -v[0]], [-v[1], v[0], 0.0]])


def _coupled_case(rng):
    """The strongly coupled family of the oracle's pins: one or two bodies
    with long levers and small anisotropic inertia, mu up to 3, approaching."""
    W = np.zeros((3, 3))
    for _ in range(rng.integers(1, 3)):
        m = rng.uniform(0.5, 2.0)
        A = rng.normal(size=(3, 3))
        I = A @ A.T * rng.uniform(0.01, 1.0) + 0.01 * np.eye(3)
        lev = rng.normal(size=3) * rng.uniform(0.5, 3.0)
        W += np.eye(3) / m - _skew(lev) @ np.linalg.inv(I) @ _skew(lev)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    W = Q.T @ W @ Q
    mu = rng.uniform(0.5, 3.0)
    b = rng.normal(size=3)
    b[0] = -abs(b[0])
    return W, mu, b


def test_one_contact_solver_matches_oracle(nb, oracle_mod):
    """nbgs_one_contact (the device solver of the composite sweep) against
    the oracle's on 40,000 problems of the strongly coupled family, among
    them the four with several valid sliding states (the least-energy one
    must be chosen) and the ones that fall back to the diagonal form."""
    import torch
    rng = np.random.default_rng(5)
    cases = [_coupled_case(rng) for _ in range(40000)]
    W6 = np.array([[W[0, 0], W[1, 1], W[2, 2], W[0, 1], W[0, 2], W[1, 2]] for W, _, _ in cases])
    mu = np.array([m for _, m, _ in cases])
    b = np.array([bb for _, _, bb in cases])
    dev = torch.device("cuda:0")
    tW, tm, tb = (torch.as_tensor(a, dtype=torch.float64, device=dev) for a in (W6, mu, b))
    tp = torch.empty((len(cases), 3), dtype=torch.float64, device=dev)
    assert nb.library().nbgs_one_contact(len(cases), tW.data_ptr(), tm.data_ptr(), tb.data_ptr(), tp.data_ptr(),
                                         torch.cuda.current_stream().cuda_stream) == nb.NBGS_OK
    torch.cuda.synchronize()
    pg = tp.cpu().numpy()
    po = np.array([oracle_mod.one_contact_general(W6[i], mu[i], b[i])[0] for i in range(len(cases))])
    scale = np.maximum(1.0, np.abs(po).max(1))
    err = np.abs(pg - po).max(1) / scale
    for i in (3864, 23274, 31903, 37769):   # several valid slides: the least-energy one
        assert err[i] <= 1e-9, (i, pg[i], po[i])
    print("one-contact solver, GPU against oracle: largest relative difference", float(err.max()))
    assert err.max() <= 1e-10   # measured on a GB300: 1.8e-12


def test_pair_normals_are_correctly_rounded(nb):
    """nbgs_pair_normals (the detection's sphere geometry): d and the three
    quotients (x_i - x_j) / d bit for bit equal to IEEE division and square
    root in FP64 (numpy), on 2M random differences over 80 binades, exact
    powers of two, distances whose significand is all ones, signed zeros,
    tiny numerators and coincident centres."""
    import torch
    rng = np.random.default_rng(17)
    m = 2_000_000
    dv = rng.normal(size=(m, 3)) * np.exp2(rng.integers(-40, 40, (m, 1)))
    dv[:1000] = rng.uniform(0.0, 100.0, (1000, 3)) - rng.uniform(0.0, 100.0, (1000, 3))
    k = 1000
    for e in range(-20, 21):                    # axis-aligned: d an exact power of two
        dv[k] = [0.0, -np.ldexp(1.0, e), 0.0]
        dv[k + 1] = [np.ldexp(1.0, e), 0.0, -0.0]
        k += 2
    ones = np.nextafter(2.0, 0.0)               # significand all ones
    for e in range(-10, 11):
        dv[k] = [np.ldexp(ones, e), 0.0, 0.0]
        dv[k + 1] = [np.ldexp(ones, e) * 0.6, np.ldexp(ones, e) * 0.8, 0.0]
        k += 2
    dv[k] = [0.0, 0.0, 0.0]                     # coincident centres
    dv[k + 1] = [-0.0, 0.0, -0.0]
    dv[k + 2] = [1e-300, 1.0, 0.0]              # tiny numerator
    dv[k + 3] = [5e-324, -2.0, 3.0]             # subnormal numerator
    dev = torch.device("cuda:0")
    td = torch.as_tensor(dv, device=dev)
    to = torch.empty((m, 4), dtype=torch.float64, device=dev)
    assert nb.library().nbgs_pair_normals(m, td.data_ptr(), to.data_ptr(),
                                          torch.cuda.current_stream().cuda_stream) == nb.NBGS_OK
    torch.cuda.synchronize()
    out = to.cpu().numpy()
    x, y, z = dv[:, 0], dv[:, 1], dv[:, 2]
    d = np.sqrt((x * x + y * y) + z * z)
    with np.errstate(invalid="ignore", divide="ignore"):
        ref = np.stack([x / d, y / d, z / d, d], axis=1)
    zero = d == 0.0
    ref[zero, :3] = [0.0, 0.0, 1.0]
    same = out.view(np.uint64) == ref.view(np.uint64)
    bad = np.nonzero(~same.all(1))[0]
    assert len(bad) == 0, (len(bad), dv[bad[:5]], out[bad[:5]], ref[bad[:5]])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_update_bodies_round_trip_keeps_the_history(nb, precision):
    """Reading the state back and writing it again with nbgs_update_bodies
    between steps leaves every step as it was (the warm start still finds
    the previous impulses), bit for bit; nbgs_set_bodies starts a new
    history instead (cold start: different impulses after a few sweeps)."""
    sc = scenes.loose_pour(seed=3, n=6000, precision=precision, warm_start="prev")
    sc["vel"] = np.random.default_rng(4).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.02
    a, b, c = nb.Scene(sc), nb.Scene(sc), nb.Scene(sc)
    for g in (a, b, c):
        g.step(20)
    for _ in range(3):
        for g, how in ((b, "update"), (c, "set")):
            st = g.get_bodies()
            getattr(g, how + "_bodies")(st["pos"], st["quat"], st["vel"], st["angvel"])
        for g in (a, b, c):
            g.step(5)
    ba, bb = a.get_bodies(), b.get_bodies()
    ca, cb, cc = a.get_contacts(), b.get_contacts(), c.get_contacts()
    assert len(ca["j1"]) > 1000
    for k in ("pos", "quat", "vel", "angvel"):
        assert np.array_equal(ba[k], bb[k]), k
    assert np.array_equal(ca["impulse"], cb["impulse"])
    assert not np.array_equal(ca["impulse"], cc["impulse"])
