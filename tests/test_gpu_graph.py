"""nbgs_graph_step: time steps captured as CUDA graphs and replayed without
host synchronisation (device-sized launches, colouring rounds in one
cooperative launch).  Each graph step must do exactly what nbgs_step does:
the same contacts, colours, impulses and body states, bit for bit, on single
scenes and on batches; and through the graph path the oracle is matched as
for ordinary steps."""
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


def _state(g):
    b, c = g.get_bodies(), g.get_contacts()
    return b, c


def _same(x, y):
    (bx, cx), (by, cy) = x, y
    for k in ("pos", "quat", "vel", "angvel"):
        assert np.array_equal(bx[k], by[k]), k
    for k in ("j1", "j2", "colour", "normal", "xi", "impulse"):
        assert np.array_equal(cx[k], cy[k]), k


def _pour(precision, n=9001, seed=2):
    sc = scenes.loose_pour(seed=seed, n=n, precision=precision, warm_start="prev")
    sc["vel"] = np.random.default_rng(7).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.02
    return sc


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_graph_steps_equal_ordinary_steps(nb, precision):
    sc = _pour(precision)
    a, b = nb.Scene(sc), nb.Scene(sc)
    for g in (a, b):
        g.step(30, 1e-6)
    for _ in range(5):
        a.step(30, 1e-6)
    b.graph_step(30, 1e-6, 5)
    _same(_state(a), _state(b))
    # more replays after a read-out, then ordinary steps again on the graph scene
    for _ in range(3):
        a.step(30, 1e-6)
    b.graph_step(30, 1e-6, 3)
    _same(_state(a), _state(b))
    sa, sb = a.step(30, 1e-6), b.step(30, 1e-6)
    assert sa == sb
    _same(_state(a), _state(b))


def test_graph_steps_of_a_batch_equal_ordinary_steps(nb):
    bs = scenes.batch_scenes(64, seed=3, n_lo=200, n_hi=3000, precision="fp32", contacts_per_body=8,
                             warm_start="prev")
    for x in bs:
        x["vel"][:, 2] -= 2.0   # contacts from the first steps on
        x["params"]["dt"] = 5e-3
    a, b = nb.BatchScene(bs), nb.BatchScene(bs)
    for g in (a, b):
        g.step(50, 1e-6)
    for _ in range(4):
        a.step(50, 1e-6)
    b.graph_step(50, 1e-6, 4)
    _same(_state(a), _state(b))
    ka, ra = a.scene_stats()
    kb, rb = b.scene_stats()
    assert np.array_equal(ka, kb) and np.array_equal(ra, rb)
    assert len(b.get_contacts()["j1"]) > 1000


def test_graph_steps_match_oracle(nb, oracle_mod):
    """Two steps from the same state: one ordinary and one replayed graph step
    on the GPU, two oracle steps; FP64, 1e-10 as for ordinary steps."""
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc["params"]["dt"] = 2e-2
    sc["params"]["warm_start"] = "prev"
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    g.step(50)
    o.step(50)
    g.graph_step(50, 0.0, 1)
    so = o.step(50)
    cg, co = g.get_contacts(), o.get_contacts()
    assert len(cg["j1"]) == so["n_contacts"] > 2000
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    assert np.array_equal(cg["colour"], co["colour"])
    bg, bo = g.get_bodies(), o.get_bodies()
    scale = float(np.abs(bo["vel"]).max())
    assert np.abs(bg["vel"] - bo["vel"]).max() <= 1e-10 * scale
    assert np.abs(cg["impulse"] - co["impulse"]).max() <= 1e-10 * float(np.abs(co["impulse"]).max())


def test_graph_step_capacity_is_reported(nb):
    """Contacts beyond the buffers a graph was captured with: the replays stay
    inside the buffers and the next synchronising call returns
    NBGS_ECAPACITY."""
    sc = _pour("fp32", n=4000)
    sc["params"]["contacts_per_body"] = 1
    sc["vel"] = np.zeros_like(sc["vel"])
    sc["params"]["dt"] = 5e-3
    g = nb.Scene(sc)
    g.step(10)                       # few contacts: small buffers
    g.graph_step(10, 0.0, 400)       # the column collapses: far more contacts
    with pytest.raises(nb.NBGSError) as e:
        g.sync()
    assert e.value.status == nb.NBGS_ECAPACITY


def test_graph_step_refusals(nb):
    sc = _pour("fp64", n=2000)
    g = nb.Scene(sc)
    with pytest.raises(nb.NBGSError):
        g.graph_step(10, 0.0, 1)     # no ordinary step yet
    sc2 = dict(sc, params=dict(sc["params"], subdomains="jacobi"))
    g2 = nb.Scene(sc2)
    g2.step(5)
    with pytest.raises(nb.NBGSError):
        g2.graph_step(5, 0.0, 1)
