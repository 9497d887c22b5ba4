"""The synthetic scene generators against the setup figures the paper prints
for its test problems (Sect. 7.2.1 granular gas of composites, Sect. 7.2.2
hexagonal close packing on a ramp), read from tests/golden/workload_setups.txt.

These pin the inputs, not the method: the members of a gas particle, the
grid, the speeds and the solid volume fraction the member radii produce; the
packing density, the tilt of gravity and the downhill start of the ramp."""
import math
import os

import numpy as np

from paper_1501_05810_gb300 import scenes

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    out = {}
    for line in open(os.path.join(HERE, "golden", "workload_setups.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            out[k] = float(v)
    return out


G = _golden()


def test_golden_closed_forms():
    """The fixture's derived values against their closed forms."""
    assert G["gas_speed_max"] == 2.0 * math.sqrt(3.0) / 10.0
    assert abs(G["hcp_density"] - math.pi / (3.0 * math.sqrt(2.0))) <= 1e-15
    assert round(G["hcp_density"], 3) == G["hcp_density_printed"]


def test_composite_gas_members_grid_and_speeds():
    sc = scenes.composite_gas(6, 5, 4, seed=3)
    m = sc["members"]
    counts = np.bincount(m["body"], minlength=len(sc["pos"]))
    assert counts.min() == G["gas_members_min"] and counts.max() == G["gas_members_max"]
    # every member touches the inside of the bounding sphere
    reach = np.linalg.norm(m["offset"], axis=1) + m["radius"]
    assert np.abs(reach - 0.5 * G["gas_bounding_diameter"]).max() <= 1e-12
    # diameters 0.6..0.8 (reading of the printed range as diameters)
    assert m["radius"].min() >= 0.3 and m["radius"].max() <= 0.4
    # reference points on a Cartesian grid of the printed spacing
    p = sc["pos"]
    for a in range(3):
        steps = np.diff(np.unique(p[:, a]))
        assert np.allclose(steps, G["gas_spacing"], rtol=0, atol=1e-12)
    speed = np.linalg.norm(sc["vel"], axis=1)
    assert speed.max() <= G["gas_speed_max"]
    assert sc["params"]["mu"] == G["gas_mu"] and sc["params"]["omega"] == G["gas_omega"]
    assert tuple(sc["params"]["gravity"]) == (0.0, 0.0, 0.0)


def test_composite_gas_solid_volume_fraction():
    """The union volume of a particle's members (overlaps counted once),
    estimated by seeded Monte Carlo over the bounding cube, over the cell
    volume 1.1^3: 23 % on average as printed.  Standard error ~0.0025 here."""
    sc = scenes.composite_gas(6, 6, 6, seed=0)
    m = sc["members"]
    rng = np.random.default_rng(11)
    n = len(sc["pos"])
    half = 0.5 * G["gas_bounding_diameter"]
    samples = 4000
    vol = np.empty(n)
    starts = np.searchsorted(m["body"], np.arange(n + 1))
    for b in range(n):
        pts = rng.uniform(-half, half, (samples, 3))
        inside = np.zeros(samples, bool)
        for k in range(starts[b], starts[b + 1]):
            inside |= np.sum((pts - m["offset"][k]) ** 2, axis=1) <= m["radius"][k] ** 2
        vol[b] = inside.mean() * (2.0 * half) ** 3
    phi = vol.mean() / G["gas_spacing"] ** 3
    assert abs(phi - G["gas_volume_fraction"]) <= 0.01, phi
    # counting overlaps twice would give far more: the reading needs the union
    summed = np.bincount(m["body"], 4.0 / 3.0 * math.pi * m["radius"] ** 3).mean() / G["gas_spacing"] ** 3
    assert summed > 0.35


def test_hcp_packing_density_and_contacts():
    """Sphere volume over the periodic cell per layer (slab of the layer
    spacing 2 sqrt(2/3) r) is the HCP density; every interior sphere has 12
    touching neighbours at distance 2r."""
    nx, ny, nz, r = 6, 4, 5, 0.5
    sc = scenes.hcp_packing(nx, ny, nz, radius=r)
    lo, hi = np.array(sc["params"]["box_lo"]), np.array(sc["params"]["box_hi"])
    slab = 2.0 * math.sqrt(2.0 / 3.0) * r
    dens = len(sc["pos"]) * 4.0 / 3.0 * math.pi * r ** 3 / ((hi[0] - lo[0]) * (hi[1] - lo[1]) * nz * slab)
    assert abs(dens - G["hcp_density"]) <= 1e-12
    # periodic minimum-image distances in x, y
    p = sc["pos"]
    d = p[:, None, :] - p[None, :, :]
    for a in range(2):
        L = hi[a] - lo[a]
        d[..., a] -= L * np.round(d[..., a] / L)
    dist = np.linalg.norm(d, axis=-1)
    touching = np.isclose(dist, 2.0 * r, rtol=0, atol=1e-9)
    layer = np.round((p[:, 2] - r) / slab).astype(int)
    interior = (layer > 0) & (layer < nz - 1)
    assert np.all(touching[interior].sum(axis=1) == 12)
    assert np.all(dist[~np.eye(len(p), dtype=bool)] >= 2.0 * r - 1e-9)


def test_ramp_gravity_and_downhill_start():
    import bench
    sc, _ = bench.workload("ramp")
    gx, gy, gz = sc["params"]["gravity"]
    assert abs(math.hypot(gx, gz) - G["hcp_gravity"]) <= 1e-12 and gy == 0.0
    assert abs(math.degrees(math.atan2(gx, -gz)) - G["hcp_tilt_deg"]) <= 1e-12
    v = sc["vel"]
    assert np.all(v[:, 0] > 0.0) and np.all(v[:, 1:] == 0.0)   # downhill: along gravity's x part
    assert sc["params"]["mu"] == G["hcp_mu"]
    assert sc["params"]["omega"] == G["gas_omega"]   # the same under-relaxation in both setups
