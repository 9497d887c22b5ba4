"""Batched scenes (nbgs_create_batch): every scene of a batch must end
exactly where the oracle puts that scene when it is stepped alone --
contacts and colours bit-exact in scene-local numbering, velocities and
impulses within 1e-10 (FP64), and each scene stopping at its own
tolerance."""
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


def _small_batch(seed=3, sizes=(60, 151, 300, 97, 420, 33)):
    rng = np.random.default_rng(seed)
    out = []
    for k, n in enumerate(sizes):
        sc = scenes.batch_scene(seed * 100 + k, n, mu=float(rng.uniform(0.2, 0.8)))
        sc["vel"] = rng.normal(0.0, 2.0, sc["vel"].shape)
        sc["angvel"] = rng.normal(0.0, 2.0, sc["vel"].shape)
        sc["params"]["dt"] = 0.03
        out.append(sc)
    return scenes.layout_batch(out)


def _local(c, off, n_s, n_total, s):
    j1 = c["j1"].astype(np.int64) - off
    j2 = c["j2"].astype(np.int64)
    wall = j2 >= n_total
    j2 = np.where(wall, n_s + (j2 - n_total - 6 * s), j2 - off)
    return j1, j2


def _close(a, b, rel):
    scale = max(float(np.abs(b).max()) if b.size else 0.0, 1e-300)
    assert (float(np.abs(a - b).max()) if b.size else 0.0) <= rel * scale


def test_batch_matches_each_scene_alone(nb, oracle_mod):
    batch = _small_batch()
    g = nb.BatchScene(batch)
    g.step(25)
    cg = g.get_contacts()
    bg = g.get_bodies()
    owner = np.searchsorted(g.offsets, cg["j1"].astype(np.int64), side="right") - 1
    total = 0
    for s, sc in enumerate(batch):
        o = oracle_mod.OracleScene(sc)
        o.step(25)
        co, bo = o.get_contacts(), o.get_bodies()
        sel = owner == s
        off, n_s = int(g.offsets[s]), len(sc["radius"])
        j1, j2 = _local({k: v[sel] for k, v in cg.items()}, off, n_s, g.n, s)
        assert np.array_equal(j1, co["j1"]) and np.array_equal(j2, co["j2"])
        assert np.array_equal(cg["colour"][sel], co["colour"])
        assert np.array_equal(cg["xi"][sel], co["xi"]) and np.array_equal(cg["normal"][sel], co["normal"])
        _close(cg["impulse"][sel], co["impulse"], 1e-10)
        _close(bg["vel"][off:off + n_s], bo["vel"], 1e-10)
        _close(bg["angvel"][off:off + n_s], bo["angvel"], 1e-10)
        assert np.abs(bg["pos"][off:off + n_s] - bo["pos"]).max() <= 1e-12 * np.abs(bo["pos"]).max()
        total += len(co["j1"])
    assert total == len(cg["j1"]) and total > 500


def test_batch_warm_start_matches_each_scene_alone(nb, oracle_mod):
    """Previous-step warm starts in a batch: each scene's previous contacts
    and impulses are matched within the scene, as when it steps alone."""
    batch = _small_batch(seed=7, sizes=(90, 240, 55))
    for sc in batch:
        sc["params"]["warm_start"] = "prev"
    g = nb.BatchScene(batch)
    oracles = [oracle_mod.OracleScene(sc) for sc in batch]
    for _ in range(3):
        g.step(25)
        for o in oracles:
            o.step(25)
    cg = g.get_contacts()
    owner = np.searchsorted(g.offsets, cg["j1"].astype(np.int64), side="right") - 1
    for s, (sc, o) in enumerate(zip(batch, oracles)):
        co = o.get_contacts()
        sel = owner == s
        off, n_s = int(g.offsets[s]), len(sc["radius"])
        j1, j2 = _local({k: v[sel] for k, v in cg.items()}, off, n_s, g.n, s)
        assert np.array_equal(j1, co["j1"]) and np.array_equal(j2, co["j2"])
        _close(cg["impulse"][sel], co["impulse"], 1e-8)


def test_batch_per_scene_tolerance(nb, oracle_mod):
    batch = _small_batch(seed=5, sizes=(80, 200, 50, 260))
    g = nb.BatchScene(batch)
    kg, rg = g.step_scenes(400, 1e-6)
    bg = g.get_bodies()
    for s, sc in enumerate(batch):
        o = oracle_mod.OracleScene(sc)
        st = o.step(400, 1e-6)
        assert abs(int(kg[s]) - st["sweeps_done"]) <= 1, (s, kg[s], st["sweeps_done"])
        if kg[s] == st["sweeps_done"]:
            assert abs(rg[s] - st["residual"]) <= 1e-6 * max(1.0, st["residual"]) + 1e-12
            off, n_s = int(g.offsets[s]), len(sc["radius"])
            _close(bg["vel"][off:off + n_s], o.get_bodies()["vel"], 1e-9)
    assert len(set(kg.tolist())) > 1   # the scenes really stopped at different sweeps


def test_autotune_keeps_results(nb):
    sc = scenes.loose_pour(seed=6, n=6000)
    sc["vel"] = np.random.default_rng(1).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    ref = nb.Scene(sc)
    ref.step(20)
    g = nb.Scene(sc)
    g.detect_contacts()
    g.colour_contacts()
    flags, bps = nb.autotune(g, 20, 0.0)
    assert flags in (0, 1, 2, 3, 4, 8) and bps >= 1
    g.solve_nbgs(20)
    g.integrate()
    a, b = g.get_bodies(), ref.get_bodies()
    _close(a["vel"], b["vel"], 1e-12)
