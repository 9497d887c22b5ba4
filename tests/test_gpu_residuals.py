"""FP64 final residuals (eq. nonpenetration and eq. coulomb, Sect. 3) of the
CUDA path against the oracle, on states far from convergence.

After 2, 5 or 8 sweeps the constraints are still violated by amounts
between 1e-4 and 1e3 (in units of the reference speed), so the four
maxima are large and distinct and a kernel that returns zeros, swaps two
slots or drops a term fails.  The cone residual is zero to roundoff after
every sweep (the one-contact solve projects onto the cone), so it is
tested on impulses set directly on both sides: random values in and out of
the cone.  Both sides evaluate the same FP64 expressions on velocities that
agree to ~1e-15, hence a relative tolerance of 1e-10."""
import math

import numpy as np
import pytest

from paper_1501_05810_gb300 import scenes

pytestmark = pytest.mark.gpu

RTOL = 1e-10
TEETH = 1e-6
KEYS = ("non_penetration", "cone", "complementarity", "dissipation")


@pytest.fixture(scope="module")
def nb():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1501_05810_gb300 import build
    build.build()
    from paper_1501_05810_gb300 import nbgs
    return nbgs


def _config1_dense():
    sc = scenes.config1(1)
    sc["vel"][:, 2] -= 3.0
    sc["params"]["dt"] = 2e-2
    return sc


def _pour_9001():
    sc = scenes.loose_pour(seed=2, n=9001)
    sc["vel"] = np.random.default_rng(7).normal(0.0, 2.0, sc["vel"].shape)
    sc["params"]["dt"] = 0.05
    return sc


def _cone_rim():
    """Twelve spheres pressed from below against the orifice rim of a small
    hopper (upward gravity), the rest on the cone face above."""
    sc = scenes.hopper(400, seed=4, dt=2e-3)
    z_o = 2.0 / math.tan(math.radians(30.0))
    rng = np.random.default_rng(11)
    k = 12
    phi = np.linspace(0.0, 2.0 * math.pi, k, endpoint=False)
    ring = np.stack([1.9 * np.cos(phi), 1.9 * np.sin(phi), np.full(k, z_o - 0.45)], -1) + rng.uniform(-0.01, 0.01,
                                                                                                     (k, 3))
    sc["pos"] = np.concatenate([ring, sc["pos"][k:]])
    sc["params"]["gravity"] = (0.0, 0.0, 9.81)
    return sc


CASES = {"config1_dense": _config1_dense, "pour_9001": _pour_9001, "cone_rim": _cone_rim}


def _solve_both(nb, oracle_mod, sc, sweeps):
    g, o = nb.Scene(sc), oracle_mod.OracleScene(sc)
    for obj in (g, o):
        obj.detect_contacts()
        obj.colour_contacts()
        obj.solve_nbgs(sweeps, 0.0)
    cg, co = g.get_contacts(), o.get_contacts()
    assert np.array_equal(cg["j1"], co["j1"]) and np.array_equal(cg["j2"], co["j2"])
    vg, vo = g.get_bodies()["vel"], o.get_bodies()["vel"]
    assert np.abs(vg - vo).max() <= 1e-12 * max(1.0, float(np.abs(vo).max()))
    return g, o, co


def _close(rg, ro, keys):
    for k in keys:
        assert abs(rg[k] - ro[k]) <= RTOL * ro[k], (k, rg[k], ro[k])


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("sweeps", [2, 5, 8])
def test_unconverged_residuals_match_oracle(nb, oracle_mod, case, sweeps):
    g, o, _ = _solve_both(nb, oracle_mod, CASES[case](), sweeps)
    rg, ro = g.final_residuals(), o.final_residuals()
    live = ("non_penetration", "complementarity", "dissipation")
    for k in live:
        assert ro[k] >= TEETH, (k, ro[k])   # the state is far from solved
    _close(rg, ro, live)
    # projected onto the cone after every sweep: roundoff on both sides
    assert rg["cone"] <= 1e-9 and ro["cone"] <= 1e-9


@pytest.mark.parametrize("case", sorted(CASES))
def test_residuals_of_set_impulses_match_oracle(nb, oracle_mod, case):
    """Impulses outside the cone (|p_t| > mu p_n, negative p_n) on both
    sides: all four residuals large, distinct and equal to 1e-10."""
    g, o, co = _solve_both(nb, oracle_mod, CASES[case](), 5)
    m = len(co["j1"])
    s = float(np.abs(co["impulse"]).max())
    rng = np.random.default_rng(5)
    imp = np.stack([rng.uniform(-0.2, 1.0, m) * s, rng.normal(0.0, 0.5 * s, m), rng.normal(0.0, 0.5 * s, m)], -1)
    g.set_impulses(imp)
    o.set_impulses(imp)
    assert np.array_equal(g.get_contacts()["impulse"], imp)
    rg, ro = g.final_residuals(), o.final_residuals()
    for k in KEYS:
        assert ro[k] >= TEETH, (k, ro[k])
    assert len({ro[k] for k in KEYS}) == 4   # a swap of two slots shows
    _close(rg, ro, KEYS)


def test_set_impulses_refused_before_a_solve(nb):
    g = nb.Scene(scenes.config1(0))
    g.detect_contacts()
    with pytest.raises(nb.NBGSError):
        g.set_impulses(np.zeros((1, 3)))
