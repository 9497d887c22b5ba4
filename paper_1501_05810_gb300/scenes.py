"""Seeded synthetic scenes (inputs only).

This module is the one place that both the CUDA path and the CPU oracle take
their inputs from.  It holds no arithmetic of the method itself: it draws
positions, velocities, radii and densities with ``numpy.random.default_rng``
and lays out lattices and walls.  Masses, hulls, contacts and everything
else are computed by each side on its own.

A scene is a dict::

    {"name": str,
     "params": {dt, gravity, mu, omega, tau, beta, box_lo, box_hi, periodic,
                warm_start, colour_seed, precision},
     "pos": (n, 3) f64, "vel": (n, 3) f64, "angvel": (n, 3) f64,
     "radius": (n,) f64, "density": (n,) f64,
     "planes": [((nx, ny, nz), c), ...],   # wall solid {y : n . y <= c}
     "cones": [{apex, axis, half_angle, r_orifice, r_top}, ...]}   # hopper walls

Workload shapes follow the paper's setups (granular gas, Sect. 7.2.1;
hexagonal close packing, Sect. 7.2.2) scaled to one GPU, plus a conical
hopper discharge.
"""
from __future__ import annotations

import math

import numpy as np


def default_params(**kw) -> dict:
    p = {
        "dt": 1e-3,
        "gravity": (0.0, 0.0, -9.81),
        "mu": 0.5,
        "omega": 1.0,
        "tau": 0.005,
        "beta": 1.0,
        "box_lo": (0.0, 0.0, 0.0),
        "box_hi": (1.0, 1.0, 1.0),
        "periodic": (0, 0, 0),
        "warm_start": "none",
        "colour_seed": 0x5EED,
        "precision": "fp64",
    }
    p.update(kw)
    return p


def box_walls(lo, hi, axes=(0, 1, 2)) -> list:
    """Six (or fewer) half-space walls enclosing [lo, hi]; each wall solid is
    {y : n . y <= c} with n the unit normal pointing into the box."""
    planes = []
    for a in axes:
        n = [0.0, 0.0, 0.0]
        n[a] = 1.0
        planes.append((tuple(n), float(lo[a])))
        n = [0.0, 0.0, 0.0]
        n[a] = -1.0
        planes.append((tuple(n), -float(hi[a])))
    return planes


def _scene(name, params, pos, vel, angvel, radius, density, planes, cones=()):
    n = len(radius)
    return {
        "name": name,
        "params": params,
        "pos": np.ascontiguousarray(pos, dtype=np.float64).reshape(n, 3),
        "vel": np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3),
        "angvel": np.ascontiguousarray(angvel, dtype=np.float64).reshape(n, 3),
        "radius": np.ascontiguousarray(radius, dtype=np.float64).reshape(n),
        "density": np.ascontiguousarray(density, dtype=np.float64).reshape(n),
        "planes": list(planes),
        "cones": [dict(c) for c in cones],
    }


def cone(apex, axis, half_angle_deg: float, r_orifice: float, r_top: float) -> dict:
    """A conical hopper wall (frustum of the cone with the given apex, axis
    and half-angle between the orifice radius and the top radius)."""
    return {"apex": tuple(float(a) for a in apex), "axis": tuple(float(a) for a in axis),
            "half_angle": math.radians(half_angle_deg), "r_orifice": float(r_orifice), "r_top": float(r_top)}


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def lattice_box(seed: int = 0, per_side: int = 10, spacing: float = 1.05, radius: float = 0.5,
                jitter: float = 0.02, vel_sigma: float = 0.1, **params) -> dict:
    """Monodisperse spheres on a jittered simple-cubic lattice inside a box of
    side per_side * spacing with six walls; velocities N(0, vel_sigma^2).

    per_side=10 is the 1,000-sphere FP64 workload: r = 0.5, density 1,
    spacing 1.05, jitter U(-0.02, 0.02), gravity -9.81 z, mu = 0.5, dt = 1e-3,
    50 sweeps per step.  The box side is 10 * 1.05 = 10.5 so that the
    lattice fits without initial overlap."""
    rng = np.random.default_rng(seed)
    side = per_side * spacing
    k = np.arange(per_side)
    gx, gy, gz = np.meshgrid(k, k, k, indexing="ij")
    base = (np.stack([gx, gy, gz], -1).reshape(-1, 3) + 0.5) * spacing
    pos = base + rng.uniform(-jitter, jitter, base.shape)
    n = len(pos)
    vel = rng.normal(0.0, vel_sigma, (n, 3))
    prm = default_params(box_lo=(0.0, 0.0, 0.0), box_hi=(side, side, side), **params)
    return _scene(f"lattice_box_{n}", prm, pos, vel, np.zeros((n, 3)), np.full(n, radius),
                  np.ones(n), box_walls((0, 0, 0), (side, side, side)))


def config1(seed: int = 0) -> dict:
    """1,000 spheres, FP64: the small parity workload."""
    return lattice_box(seed, per_side=10, dt=1e-3, mu=0.5, tau=0.005, precision="fp64")


def loose_pour(seed: int = 0, n: int = 1_000_000, r_lo: float = 0.4, r_hi: float = 0.6,
               base: float = 100.0, height: float = 200.0, phi: float = 0.3, **params) -> dict:
    """Polydisperse spheres r ~ U(r_lo, r_hi), density 1, on a jittered cubic
    lattice at volume fraction phi filling a walled box from the floor up,
    under gravity.  n = 1e6 with base 100 x 100 x 200 is the 1M-sphere pour;
    smaller n shrink the base so the column keeps its shape."""
    rng = np.random.default_rng(seed)
    radius = rng.uniform(r_lo, r_hi, n)
    mean_vol = 4.0 / 3.0 * math.pi * np.mean(radius ** 3)
    s = max((mean_vol / phi) ** (1.0 / 3.0), 2.0 * r_hi * 1.0001)
    if n != 1_000_000:
        base = base * (n / 1_000_000) ** (1.0 / 3.0)
        height = height * (n / 1_000_000) ** (1.0 / 3.0)
    nx = max(1, int(base // s))
    nz = int(math.ceil(n / (nx * nx)))
    idx = np.arange(n)
    ix, iy, iz = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    pos = (np.stack([ix, iy, iz], -1) + 0.5) * s
    j = (s - 2.0 * r_hi) / 2.0
    pos = pos + rng.uniform(-j, j, pos.shape)
    height = max(height, (nz + 1) * s)
    lo, hi = (0.0, 0.0, 0.0), (nx * s, nx * s, height)
    prm = default_params(**{**dict(dt=5e-4, mu=0.5, tau=0.01 * r_lo, box_lo=lo, box_hi=hi), **params})
    return _scene(f"loose_pour_{n}", prm, pos, np.zeros((n, 3)), np.zeros((n, 3)), radius,
                  np.ones(n), box_walls(lo, hi))


def hcp_packing(nx: int, ny: int, nz: int, radius: float = 0.5, density: float = 1.0,
                tilt_deg: float = 0.0, g: float = 9.81, v0: float = 0.0, **params) -> dict:
    """Hexagonal close packing of equal spheres (Sect. 7.2.2): periodic in x
    and y, confined in z by two walls touching the first and last layer.
    ny must be even.  Gravity of magnitude g is tilted by tilt_deg in the
    x-z plane (a ramp); every sphere starts with velocity v0 along +x."""
    if ny % 2:
        raise ValueError("hcp_packing needs an even ny")
    r = radius
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    x = (2.0 * i + ((j + k) % 2)) * r
    y = math.sqrt(3.0) * (j + (k % 2) / 3.0) * r
    z = r + 2.0 * math.sqrt(6.0) / 3.0 * k * r
    pos = np.stack([x, y, z], -1)
    n = len(pos)
    Lx, Ly = 2.0 * r * nx, math.sqrt(3.0) * r * ny
    top = 2.0 * r + 2.0 * math.sqrt(6.0) / 3.0 * (nz - 1) * r
    th = math.radians(tilt_deg)
    grav = (g * math.sin(th), 0.0, -g * math.cos(th))
    vel = np.zeros((n, 3))
    vel[:, 0] = v0
    lo, hi = (0.0, 0.0, 0.0), (Lx, Ly, top)
    prm = default_params(gravity=grav, box_lo=lo, box_hi=hi, periodic=(1, 1, 0), **params)
    return _scene(f"hcp_{nx}x{ny}x{nz}", prm, pos, vel, np.zeros((n, 3)), np.full(n, r),
                  np.full(n, density), box_walls(lo, hi, axes=(2,)))


def dense_packing(n_target: int = 1_000_000, seed: int = 0, **params) -> dict:
    """A dense packing of ~n_target spheres in contact: the hexagonal close
    packing above with r = 0.5 (the mean radius of the 1M pour), x, y
    periodic and walls on both z faces, n_x = n_y (even) and n_z chosen for
    the count.  It carries n_x n_y (6 n_z - 1) contacts, so the sweeps
    dominate the step: the regime the settled 1M-sphere packing is
    measured in.  Gravity -9.81 z, mu = 0.5, dt = 5e-4."""
    side = int(round(n_target ** (1.0 / 3.0)))
    side += side % 2
    nz = max(1, int(round(n_target / (side * side))))
    params.setdefault("dt", 5e-4)
    params.setdefault("mu", 0.5)
    params.setdefault("tau", 0.005)
    sc = hcp_packing(side, side, nz, radius=0.5, **params)
    rng = np.random.default_rng(seed)
    sc["vel"] = sc["vel"] + rng.normal(0.0, 1e-3, sc["vel"].shape)
    sc["name"] = f"dense_hcp_{len(sc['radius'])}"
    return sc


def granular_gas(cells: int = 196, seed: int = 0, r_lo: float = 0.45, r_hi: float = 0.55,
                 phi: float = 0.5, jitter: float = 0.01, **params) -> dict:
    """Dense granular gas: FCC lattice of cells^3 * 4 spheres with
    r ~ U(r_lo, r_hi) in a triply periodic cube sized so that the volume
    fraction is exactly phi for the drawn radii; velocities N(0, 1) per
    component, no gravity, mu = 0.3, dt = 1e-4.  cells = 196 gives
    30,118,144 spheres."""
    rng = np.random.default_rng(seed)
    n = 4 * cells ** 3
    radius = rng.uniform(r_lo, r_hi, n)
    vol = 4.0 / 3.0 * math.pi * float(np.sum(radius ** 3))
    side = (vol / phi) ** (1.0 / 3.0)
    a = side / cells
    c = np.arange(cells)
    gx, gy, gz = np.meshgrid(c, c, c, indexing="ij")
    corner = np.stack([gx, gy, gz], -1).reshape(-1, 1, 3).astype(np.float64)
    basis = np.array([[0.25, 0.25, 0.25], [0.75, 0.75, 0.25], [0.75, 0.25, 0.75], [0.25, 0.75, 0.75]])
    pos = ((corner + basis[None]) * a).reshape(-1, 3)
    pos = pos + rng.uniform(-jitter, jitter, pos.shape)
    pos = np.mod(pos, side)
    vel = rng.normal(0.0, 1.0, (n, 3))
    prm = default_params(dt=1e-4, gravity=(0.0, 0.0, 0.0), mu=0.3, tau=0.01 * r_lo,
                         box_lo=(0.0, 0.0, 0.0), box_hi=(side, side, side), periodic=(1, 1, 1),
                         **params)
    return _scene(f"granular_gas_{n}", prm, pos, vel, np.zeros((n, 3)), radius, np.ones(n), [])


# ---------------------------------------------------------------------------
# Known-answer scenes
# ---------------------------------------------------------------------------

def sphere_on_plane(radius: float = 0.5, density: float = 1.0, gap: float = 0.0, **params) -> dict:
    prm = default_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 5), **params)
    pos = np.array([[0.0, 0.0, radius + gap]])
    return _scene("sphere_on_plane", prm, pos, np.zeros((1, 3)), np.zeros((1, 3)), [radius], [density],
                  [((0.0, 0.0, 1.0), 0.0)])


def sphere_in_cone(radius: float = 0.5, half_angle_deg: float = 30.0, height: float = None,
                   **params) -> dict:
    """One sphere on the axis of an upward-opening cone (apex at the origin,
    orifice radius 0.2 r so that the sphere cannot pass); at rest it touches
    the cone along a circle with its centre r / sin(a) above the apex."""
    a = math.radians(half_angle_deg)
    z = radius / math.sin(a) if height is None else height
    prm = default_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 10), **params)
    pos = np.array([[0.0, 0.0, z]])
    return _scene("sphere_in_cone", prm, pos, np.zeros((1, 3)), np.zeros((1, 3)), [radius], [1.0], [],
                  [cone((0, 0, 0), (0, 0, 1), half_angle_deg, 0.2 * radius, 4.0)])


def hopper(n: int = 2_000_000, seed: int = 0, half_angle_deg: float = 30.0, r_lo: float = 0.4, r_hi: float = 0.6,
           orifice_diameter: float = None, spacing: float = None, jitter: float = 0.004, **params) -> dict:
    """Conical hopper discharge: n spheres r ~ U(r_lo, r_hi) on a jittered
    cubic lattice (gaps of 0.02 between the largest spheres) filling an
    upward-opening cone of the given half-angle from just above its orifice
    (diameter 8 r_mean unless given), falling under gravity through the
    orifice onto a floor 20 r_mean below it.  mu = 0.5, dt = 5e-4."""
    rng = np.random.default_rng(seed)
    a = math.radians(half_angle_deg)
    r_mean = 0.5 * (r_lo + r_hi)
    d_o = 8.0 * r_mean if orifice_diameter is None else orifice_diameter
    r_o = 0.5 * d_o
    sp = 2.0 * r_hi + 0.02 if spacing is None else spacing
    ta = math.tan(a)
    z_o = r_o / ta   # orifice height above the apex
    # cone volume above the orifice level that holds n lattice sites
    def sites(z_top):
        zs = np.arange(z_o + r_hi + 0.05, z_top, sp)
        tot = 0
        for z in zs:
            rad = z * ta - (r_hi + 0.01) / math.cos(a)
            if rad <= 0:
                continue
            m = int(rad // sp)
            tot += int(np.count_nonzero((np.add.outer(np.arange(-m, m + 1) ** 2, np.arange(-m, m + 1) ** 2)) * sp * sp
                                        <= rad * rad))
        return tot
    z_top = z_o + 4.0 * sp
    while sites(z_top) < n:
        z_top *= 1.15
    pts = []
    for z in np.arange(z_o + r_hi + 0.05, z_top, sp):
        rad = z * ta - (r_hi + 0.01) / math.cos(a)
        if rad <= 0:
            continue
        m = int(rad // sp)
        g = np.arange(-m, m + 1) * sp
        gx, gy = np.meshgrid(g, g, indexing="ij")
        keep = gx * gx + gy * gy <= rad * rad
        pts.append(np.stack([gx[keep], gy[keep], np.full(int(keep.sum()), z)], -1))
        if sum(len(q) for q in pts) >= n:
            break
    pos = np.concatenate(pts)[:n]
    pos = pos + rng.uniform(-jitter, jitter, pos.shape)
    radius = rng.uniform(r_lo, r_hi, n)
    r_top = (pos[:, 2].max() + sp) * ta + 2.0 * r_hi
    floor = -20.0 * r_mean
    half = r_top + 2.0
    kw = dict(dt=5e-4, mu=0.5, tau=0.01 * r_lo)
    kw.update(params)
    prm = default_params(box_lo=(-half, -half, floor - 1.0), box_hi=(half, half, r_top / ta + 2.0), **kw)
    planes = [((0.0, 0.0, 1.0), floor)]
    return _scene(f"hopper_{n}", prm, pos, np.zeros((n, 3)), np.zeros((n, 3)), radius, np.ones(n), planes,
                  [cone((0, 0, 0), (0, 0, 1), half_angle_deg, r_o, r_top)])


def head_on(ra: float = 0.5, rb: float = 0.4, rho_a: float = 1.0, rho_b: float = 2.0, gap: float = 0.01,
            va: float = 1.0, vb: float = -0.5, **params) -> dict:
    """Two spheres on the x axis approaching each other, gravity off."""
    params.setdefault("gravity", (0.0, 0.0, 0.0))
    prm = default_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 5), **params)
    pos = np.array([[-(ra + gap / 2), 0.0, 0.0], [rb + gap / 2, 0.0, 0.0]])
    vel = np.array([[va, 0.0, 0.0], [vb, 0.0, 0.0]])
    return _scene("head_on", prm, pos, vel, np.zeros((2, 3)), [ra, rb], [rho_a, rho_b], [])


def sliding(v0: float = 1.0, radius: float = 0.5, **params) -> dict:
    """A sphere resting on the floor z = 0 and moving along +x at v0."""
    prm = default_params(box_lo=(-50, -5, -5), box_hi=(50, 5, 5), **params)
    pos = np.array([[0.0, 0.0, radius]])
    vel = np.array([[v0, 0.0, 0.0]])
    return _scene("sliding", prm, pos, vel, np.zeros((1, 3)), [radius], [1.0], [((0.0, 0.0, 1.0), 0.0)])


def column(k: int = 5, radius: float = 0.5, **params) -> dict:
    """k equal spheres stacked in touching contact on the floor z = 0."""
    prm = default_params(box_lo=(-5, -5, -1), box_hi=(5, 5, 2 * radius * k + 5), **params)
    z = radius + 2.0 * radius * np.arange(k)
    pos = np.stack([np.zeros(k), np.zeros(k), z], -1)
    return _scene(f"column_{k}", prm, pos, np.zeros((k, 3)), np.zeros((k, 3)), np.full(k, radius),
                  np.ones(k), [((0.0, 0.0, 1.0), 0.0)])


def periodic_cloud(seed: int = 0, per_side: int = 6, spacing: float = 1.02, r_lo: float = 0.4,
                   r_hi: float = 0.5, vel_sigma: float = 1.0, **params) -> dict:
    """Triply periodic box of polydisperse spheres on a jittered cubic lattice
    with random linear and angular velocities; gravity off, no walls."""
    rng = np.random.default_rng(seed)
    side = per_side * spacing
    k = np.arange(per_side)
    gx, gy, gz = np.meshgrid(k, k, k, indexing="ij")
    pos = (np.stack([gx, gy, gz], -1).reshape(-1, 3) + 0.5) * spacing
    n = len(pos)
    radius = rng.uniform(r_lo, r_hi, n)
    j = (spacing - 2 * r_hi) / 2.0 * 0.9
    pos = pos + rng.uniform(-j, j, pos.shape)
    vel = rng.normal(0.0, vel_sigma, (n, 3))
    ang = rng.normal(0.0, vel_sigma, (n, 3))
    params.setdefault("gravity", (0.0, 0.0, 0.0))
    params.setdefault("dt", 1e-2)
    params.setdefault("periodic", (1, 1, 1))
    prm = default_params(box_lo=(0, 0, 0), box_hi=(side, side, side), **params)
    return _scene(f"periodic_cloud_{n}", prm, pos, vel, ang, radius, rng.uniform(0.5, 2.0, n), [])


# ---------------------------------------------------------------------------
# Batched scenes
# ---------------------------------------------------------------------------

def batch_scene(seed: int, n: int, mu: float, r_lo: float = 0.4, r_hi: float = 0.6, phi: float = 0.3,
                **params) -> dict:
    """One walled-box scene of n polydisperse spheres on a jittered cubic
    lattice at volume fraction phi, base side B = ceil((n V / phi / 2)^(1/3))
    and height 2B, settling under gravity."""
    rng = np.random.default_rng(seed)
    radius = rng.uniform(r_lo, r_hi, n)
    mean_vol = 4.0 / 3.0 * math.pi * np.mean(radius ** 3)
    base = math.ceil((n * mean_vol / phi / 2.0) ** (1.0 / 3.0))
    s = max((mean_vol / phi) ** (1.0 / 3.0), 2.0 * r_hi * 1.0001)
    nx = max(1, int(base // s))
    nz = int(math.ceil(n / (nx * nx)))
    height = max(2.0 * base, (nz + 1) * s)
    idx = np.arange(n)
    ix, iy, iz = idx % nx, (idx // nx) % nx, idx // (nx * nx)
    pos = (np.stack([ix, iy, iz], -1) + 0.5) * s
    j = (s - 2.0 * r_hi) / 2.0
    pos = pos + rng.uniform(-j, j, pos.shape)
    lo, hi = (0.0, 0.0, 0.0), (nx * s, nx * s, height)
    prm = default_params(dt=5e-4, mu=mu, tau=0.01 * r_lo, box_lo=lo, box_hi=hi, **params)
    return _scene(f"batch_scene_{seed}_{n}", prm, pos, np.zeros((n, 3)), np.zeros((n, 3)), radius, np.ones(n),
                  box_walls(lo, hi))


def batch_scenes(n_scenes: int = 4096, seed: int = 0, n_lo: int = 200, n_hi: int = 20000, mu_lo: float = 0.2,
                 mu_hi: float = 0.8, **params) -> list:
    """n_scenes independent scenes with log-uniform sphere counts in
    [n_lo, n_hi] and mu ~ U(mu_lo, mu_hi), laid out side by side."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), n_scenes))).astype(int)
    mus = rng.uniform(mu_lo, mu_hi, n_scenes)
    scenes = [batch_scene(int(seed) * 1_000_003 + k, int(sizes[k]), float(mus[k]), **params) for k in range(n_scenes)]
    return layout_batch(scenes)


def layout_batch(scenes: list, gap: float = 4.0) -> list:
    """Translate the scenes (positions, boxes, walls) onto a square grid in
    the x-y plane with `gap` between boxes, so that no two boxes overlap."""
    k = len(scenes)
    cols = max(1, int(math.ceil(math.sqrt(k))))
    size = max(max(sc["params"]["box_hi"][a] - sc["params"]["box_lo"][a] for a in (0, 1)) for sc in scenes)
    out = []
    for i, sc in enumerate(scenes):
        shift = np.array([(i % cols) * (size + gap), (i // cols) * (size + gap), 0.0]) - np.array(sc["params"]["box_lo"])
        prm = dict(sc["params"])
        lo = tuple(np.array(prm["box_lo"]) + shift)
        hi = tuple(np.array(prm["box_hi"]) + shift)
        prm["box_lo"], prm["box_hi"] = lo, hi
        t = dict(sc)
        t["params"] = prm
        t["pos"] = sc["pos"] + shift
        t["planes"] = box_walls(lo, hi)
        out.append(t)
    return out


# ---------------------------------------------------------------------------
# composite particles: rigid unions of 1-4 member spheres
# ---------------------------------------------------------------------------
def _composite_scene(name, params, pos, vel, angvel, density, member_body, member_offset, member_radius, planes):
    """A scene of composite bodies: pos is each body's reference point, the
    members' offsets are measured from it (observational axes)."""
    n = len(density)
    m = len(member_body)
    return {
        "name": name,
        "params": params,
        "pos": np.ascontiguousarray(pos, dtype=np.float64).reshape(n, 3),
        "vel": np.ascontiguousarray(vel, dtype=np.float64).reshape(n, 3),
        "angvel": np.ascontiguousarray(angvel, dtype=np.float64).reshape(n, 3),
        "density": np.ascontiguousarray(density, dtype=np.float64).reshape(n),
        "members": {
            "body": np.ascontiguousarray(member_body, dtype=np.int32).reshape(m),
            "offset": np.ascontiguousarray(member_offset, dtype=np.float64).reshape(m, 3),
            "radius": np.ascontiguousarray(member_radius, dtype=np.float64).reshape(m),
        },
        "planes": list(planes),
        "cones": [],
    }


def as_composites(sc: dict) -> dict:
    """A sphere scene as composites of one member each (offset 0)."""
    n = len(sc["radius"])
    return _composite_scene(sc["name"] + "_as_composites", dict(sc["params"]), sc["pos"], sc["vel"], sc["angvel"],
                            sc["density"], np.arange(n), np.zeros((n, 3)), sc["radius"], sc["planes"])


def dumbbell_on_plane(radius: float = 0.5, half_sep: float = 0.6, gap: float = 0.0, **params) -> dict:
    """Two equal spheres glued at (+-half_sep, 0, 0) resting on the floor z = 0."""
    prm = default_params(box_lo=(-5, -5, -5), box_hi=(5, 5, 5), **params)
    return _composite_scene("dumbbell_on_plane", prm, [[0.0, 0.0, radius + gap]], np.zeros((1, 3)),
                            np.zeros((1, 3)), [1.0], [0, 0], [[-half_sep, 0, 0], [half_sep, 0, 0]],
                            [radius, radius], [((0.0, 0.0, 1.0), 0.0)])


def spinning_body(angvel=(0.3, 2.0, 0.1), offsets=None, radii=None, **params) -> dict:
    """One free composite (gravity off, no walls) spinning with angvel; the
    default is an asymmetric three-member body."""
    if offsets is None:
        offsets = [[0.0, 0.0, 0.0], [0.9, 0.1, 0.0], [0.1, 0.0, 0.6]]
        radii = [0.5, 0.35, 0.3]
    prm = default_params(gravity=(0.0, 0.0, 0.0), box_lo=(-50, -50, -50), box_hi=(50, 50, 50), **params)
    k = len(offsets)
    return _composite_scene("spinning_body", prm, np.zeros((1, 3)), np.zeros((1, 3)), [list(angvel)], [1.0],
                            [0] * k, offsets, radii, [])


def composite_gas(nx: int = 10, ny: int = 10, nz: int = 10, seed: int = 0, spacing: float = 1.1,
                  bound_radius: float = 0.5, r_lo: float = 0.3, r_hi: float = 0.4, v_max: float = 0.2,
                  walls: bool = True, **params) -> dict:
    """The granular gas of Sect. 7.2.1 as the paper ran it: composites of two
    to four spheres of diameters U(0.6, 0.8) (radii r_lo..r_hi) touching the
    inside of a bounding sphere of diameter 1, on a Cartesian grid of spacing
    1.1, velocities U(-v_max, v_max) per component (|v| <= 0.2 sqrt 3),
    confined by walls, no gravity, mu = 0.1, omega = 0.75."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    lo = np.zeros(3)
    hi = np.array([nx, ny, nz], dtype=np.float64) * spacing
    pos = (np.stack([i.ravel(), j.ravel(), k.ravel()], -1) + 0.5) * spacing
    counts = rng.integers(2, 5, n)
    mb = np.repeat(np.arange(n), counts)
    m = len(mb)
    r = rng.uniform(r_lo, r_hi, m)
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    off = d * (bound_radius - r)[:, None]
    vel = rng.uniform(-v_max, v_max, (n, 3))
    kw = dict(gravity=(0.0, 0.0, 0.0), mu=0.1, omega=0.75, dt=1e-4, tau=0.005, box_lo=tuple(lo), box_hi=tuple(hi))
    kw.update(params)
    prm = default_params(**kw)
    planes = box_walls(lo, hi) if walls else []
    return _composite_scene(f"composite_gas_{n}", prm, pos, vel, np.zeros((n, 3)), np.ones(n), mb, off, r, planes)
