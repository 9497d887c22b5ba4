"""Pins of the FP64 reference MLP against mathematics: central finite
differences of the loss, a hand-computed one-neuron case, SiLU's closed
form, and Adam's first step."""
import math

import numpy as np

from oracle import mlp


def test_parameter_count():
    assert mlp.N_PARAMS == 9347


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    theta = mlp.init(1) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.normal(size=(7, 12))
    T = rng.normal(size=(7, 3))
    L, g = mlp.loss_and_grad(theta, X, T)
    assert abs(L - mlp.loss(theta, X, T)) < 1e-15
    idx = np.concatenate([rng.choice(mlp.N_PARAMS, 60, replace=False),
                          [0, 767, 768, 831, 832, 9151, 9152, 9346]])   # layer edges
    h = 1e-6
    for k in idx:
        e = np.zeros(mlp.N_PARAMS)
        e[k] = h
        fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)), (k, fd, g[k])


def test_silu_closed_form_and_derivative():
    z = np.linspace(-8, 8, 33)
    assert np.allclose(mlp.silu(z), z / (1 + np.exp(-z)))
    h = 1e-6
    fd = (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h)
    assert np.allclose(mlp.silu_grad(z), fd, atol=1e-8)
    assert mlp.silu(0.0) == 0.0 and abs(mlp.silu_grad(0.0) - 0.5) < 1e-15


def test_single_path_by_hand():
    # only input 0 -> hidden unit 0 of each layer -> output 0 carries weight
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(mlp.SIZES[:-1], mlp.SIZES[1:])]
    w = [0.5, -1.5, 2.0, 0.25]
    for (W, _), wk in zip(layers, w):
        W[0, 0] = wk
    layers[3][1][1] = 0.75                          # bias of output 1
    theta = mlp.flatten(layers)
    x = np.zeros((1, 12))
    x[0, 0] = 1.2
    s = lambda z: z / (1 + math.exp(-z))
    a = s(0.5 * 1.2)
    a = s(-1.5 * a)
    a = s(2.0 * a)
    y, _, _ = mlp.forward(theta, x)
    assert abs(y[0, 0] - 0.25 * a) < 1e-15 and y[0, 1] == 0.75 and y[0, 2] == 0.0


def test_adam_first_step_moves_by_lr_times_sign():
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = mlp.adam(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, -0.01 * np.sign(g))


def test_bf16_rounding():
    """bfloat16 keeps 7 fraction bits: near 1 the spacing is 2^-7."""
    assert mlp.bf16_round(1.0) == 1.0
    assert mlp.bf16_round(1.0 + 2 ** -9) == 1.0                        # a quarter ulp: down
    assert mlp.bf16_round(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7           # three quarters: up
    assert mlp.bf16_round(1.0 + 2 ** -8) == 1.0                        # tie: to the even 1.0
    assert mlp.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6           # tie: up to the even neighbour
    assert mlp.bf16_round(-(1.0 + 3 * 2 ** -8)) == -(1.0 + 2 ** -6)
    x = np.random.default_rng(2).normal(size=1000)
    assert np.all(np.abs(mlp.bf16_round(x) - x) <= np.abs(x) * 2 ** -8)


def test_skip_connection_carries_previous_impulse():
    # all parameters zero: the output is inputs 3..5 exactly
    X = np.random.default_rng(3).normal(size=(5, 12))
    Y, _, _ = mlp.forward(np.zeros(mlp.N_PARAMS), X)
    assert np.array_equal(Y, X[:, 3:6])
    # and the gradient still matches finite differences with the skip active
    theta = mlp.init(2)
    T = np.zeros((5, 3))
    L, g = mlp.loss_and_grad(theta, X, T)
    k, h = 9344, 1e-6                                   # output bias 0
    e = np.zeros(mlp.N_PARAMS)
    e[k] = h
    fd = (mlp.loss(theta + e, X, T) - mlp.loss(theta - e, X, T)) / (2 * h)
    assert abs(fd - g[k]) < 1e-8


# ---------------------------------------------------------------------------
# the 12 contact features, on configurations worked out by hand
# ---------------------------------------------------------------------------
def _features(c, vel, angvel, radius, invm, invI, params, v_ref, prev=None):
    c = {k: np.asarray(v) for k, v in c.items()}
    c["j1"], c["j2"] = c["j1"].astype(np.uint32), c["j2"].astype(np.uint32)
    bodies = {"vel": np.asarray(vel, float), "angvel": np.asarray(angvel, float)}
    return mlp.contact_features(c, bodies, np.asarray(radius, float), np.asarray(invm, float),
                                np.asarray(invI, float), params, v_ref, prev)


def test_features_of_a_sliding_spinning_sphere_over_a_floor():
    """Sphere r = 0.5, m = 2 (1/m = 0.5, I = 2/5 m r^2 = 0.2), 0.01 above the
    floor z = 0 (normal +z, contact frame t = x, o = y), v = (0.3, -0.4, -0.2),
    w = (1, 2, 3), g = -9.81 z, dt = 0.01, v_ref = 2.  The contact point sits
    at -l_a n with l_a = r + xi = 0.51, so after the gravity kick
    u = v + dt g + w x (-0.51 z) = (0.3 - 1.02, -0.4 + 0.51, -0.2 - 0.0981)."""
    params = {"dt": 0.01, "gravity": (0.0, 0.0, -9.81), "mu": 0.4}
    c = {"j1": [0], "j2": [1], "normal": [[0.0, 0.0, 1.0]], "xi": [0.01]}
    F = _features(c, [[0.3, -0.4, -0.2]], [[1.0, 2.0, 3.0]], [0.5], [0.5], [5.0], params, 2.0)[0]
    ut, uo, un = -0.72, 0.11, -0.2981
    utl = math.hypot(ut, uo)
    want = [un / 2.0, utl / 2.0, (0.01 / 0.01) / 2.0, 0.0, 0.0, 0.0,
            math.log(0.5), (0.5 + 5.0 * 0.51 ** 2) / 0.5, 0.5, 0.0, 0.4, 1.0 / 12.0,
            -ut / utl, -uo / utl, 0.5, 2.0]
    assert np.allclose(F, want, rtol=0, atol=1e-14), np.c_[F, want]


def test_features_of_a_pair_with_an_immovable_partner_and_degrees():
    """Body 0 (r 0.5, 1/m 0.5, 1/I 5) rests 0.02 above body 1 (r 0.3, infinite
    mass: no kick, no degree); body 0 also touches the wall 2.  Normal +z
    from 1 to 0: l_a = xi + r_a = 0.52 below 0's centre, l_b = r_b = 0.3 above
    1's.  With v_0 = (0.1, 0, 0), w_0 = (0, 0.5, 0), v_1 = (0, 0.2, 0),
    w_1 = (1, 0, 0) (an immovable body still moves with its given velocity):
    u = v_0 + dt g + w_0 x (-0.52 z) - v_1 - w_1 x (0.3 z)
      = (0.1 - 0.26, 0 - 0.2 + 0.3, -0.0981)."""
    params = {"dt": 0.01, "gravity": (0.0, 0.0, -9.81), "mu": 0.7}
    c = {"j1": [0, 0], "j2": [1, 2], "normal": [[0.0, 0.0, 1.0], [1.0, 0.0, 0.0]], "xi": [0.02, 0.0]}
    vel = [[0.1, 0.0, 0.0], [0.0, 0.2, 0.0]]
    ang = [[0.0, 0.5, 0.0], [1.0, 0.0, 0.0]]
    F = _features(c, vel, ang, [0.5, 0.3], [0.5, 0.0], [5.0, 0.0], params, 1.0)
    ut, uo = -0.16, 0.1
    utl = math.hypot(ut, uo)
    assert np.allclose(F[0, :3], [-0.0981, utl, 2.0], rtol=0, atol=1e-14)
    assert abs(F[0, 7] - (0.5 + 5.0 * 0.52 ** 2) / 0.5) < 1e-14          # w_t / w_n, partner immovable
    assert F[0, 8] == 0.5 and F[0, 9] == 0.3 and F[0, 10] == 0.7
    assert np.allclose(F[:, 11], [2.0 / 12.0, 2.0 / 12.0])             # body 0 in two contacts, 1 counts none
    assert np.allclose(F[0, 12:14], [-ut / utl, -uo / utl], rtol=0, atol=1e-14)
    # second contact: wall along +x, frame of n = x (Duff et al.: t = (0, 0, -1), o = (0, 1, 0));
    # u = v_0 + dt g + w_0 x (-0.5 x) = (0.1, 0, -0.0981 + 0.25)
    u2 = np.array([0.1, 0.0, -0.0981 + 0.25])
    t2, o2 = np.array([0.0, 0.0, -1.0]), np.array([0.0, 1.0, 0.0])
    ut2, uo2 = u2 @ t2, u2 @ o2
    assert np.allclose(F[1, :2], [0.1, math.hypot(ut2, uo2)], rtol=0, atol=1e-14)
    assert np.allclose(F[1, 12:14], [-ut2 / abs(ut2), 0.0], rtol=0, atol=1e-14)


def test_features_carry_the_previous_impulse_projected_onto_the_cone():
    """Two floor contacts of two spheres; the previous step saw contact
    (0, 2) with impulse (p_n, p_t, p_o) = (1, 0.3, 0.4) in the frame of +z
    (t = x, o = y), so |p_t| = 0.5 > mu p_n = 0.4: the warm start scales the
    tangential part by 0.8 to (0.24, 0.32, 1) in world axes, then expresses
    it along n, e2 = -u_t/|u_t|, e3 = n x e2, times w_n / v_ref.  Contact
    (1, 2) has no previous key (and sorts after every previous key): zero.
    Sphere 1 rests, so its e2 falls back to t (cos 1, sin 0)."""
    params = {"dt": 0.01, "gravity": (0.0, 0.0, 0.0), "mu": 0.4}
    c = {"j1": [0, 1], "j2": [2, 2], "normal": [[0.0, 0.0, 1.0]] * 2, "xi": [0.0, 0.0]}
    prev = {"j1": np.array([0], np.uint32), "j2": np.array([2], np.uint32),
            "normal": np.array([[0.0, 0.0, 1.0]]), "impulse": np.array([[1.0, 0.3, 0.4]])}
    vel = [[0.6, -0.8, 0.0], [0.0, 0.0, 0.0]]
    F = _features(c, vel, np.zeros((2, 3)), [0.5, 0.5], [0.5, 0.5], [5.0, 5.0], params, 4.0, prev)
    cth, sth = -0.6, 0.8                                   # e2 = -(0.6, -0.8) / 1
    P = np.array([0.24, 0.32, 1.0])
    e2, e3 = np.array([cth, sth, 0.0]), np.array([-sth, cth, 0.0])
    sc = 0.5 / 4.0
    assert np.allclose(F[0, 3:6], [P[2] * sc, (P @ e2) * sc, (P @ e3) * sc], rtol=0, atol=1e-15)
    assert np.allclose(F[0, 12:14], [cth, sth], rtol=0, atol=1e-15)
    assert np.all(F[1, 3:6] == 0.0) and F[1, 12] == 1.0 and F[1, 13] == 0.0
    # a previous impulse pulling (p_n < 0) projects to nothing
    prev["impulse"] = np.array([[-1.0, 0.3, 0.4]])
    F = _features(c, vel, np.zeros((2, 3)), [0.5, 0.5], [0.5, 0.5], [5.0, 5.0], params, 4.0, prev)
    assert np.all(F[:, 3:6] == 0.0)
    # inside the cone it is kept as it is
    prev["impulse"] = np.array([[2.0, 0.3, 0.4]])
    F = _features(c, vel, np.zeros((2, 3)), [0.5, 0.5], [0.5, 0.5], [5.0, 5.0], params, 4.0, prev)
    P = np.array([0.3, 0.4, 2.0])
    assert np.allclose(F[0, 3:6], [P[2] * sc, (P @ e2) * sc, (P @ e3) * sc], rtol=0, atol=1e-15)


def test_features_of_two_movable_bodies():
    """Body 0 (r 0.5, 1/m 0.5, 1/I 5) on body 1 (r 0.25, 1/m 2, 1/I 40),
    which also touches wall 2: w_n = 0.5 + 2 = 2.5, w_t = 2.5 + 5 (0.5)^2 +
    40 (0.25)^2 = 6.25, degrees 1 + 2 over 12.  Both bodies take the
    gravity kick, so it cancels from u = (0.2, 0, 0); tangential speed 0.2
    along t = x, so e2 = -x."""
    params = {"dt": 0.01, "gravity": (0.0, 0.0, -9.81), "mu": 0.5}
    c = {"j1": [0, 1], "j2": [1, 2], "normal": [[0.0, 0.0, 1.0]] * 2, "xi": [0.0, 0.0]}
    F = _features(c, [[0.2, 0.0, 0.0], [0.0, 0.0, 0.0]], np.zeros((2, 3)), [0.5, 0.25], [0.5, 2.0],
                  [5.0, 40.0], params, 1.0)
    assert np.allclose(F[0, :3], [0.0, 0.2, 0.0], rtol=0, atol=1e-15)
    assert abs(F[0, 6] - math.log(2.5)) < 1e-15 and abs(F[0, 7] - 2.5) < 1e-14
    assert F[0, 8] == 0.5 and F[0, 9] == 0.25
    assert np.allclose(F[:, 11], [3.0 / 12.0, 2.0 / 12.0])
    assert np.allclose(F[0, 12:14], [-1.0, 0.0], rtol=0, atol=1e-15) and F[0, 14] == 2.5


def test_features_treat_a_tiny_tangential_speed_as_none():
    """Below 1e-12 v_ref the tangential velocity has no direction: e2 falls
    back to the frame's t (cos 1, sin 0); just above it, e2 = -u_t / |u_t|."""
    params = {"dt": 0.01, "gravity": (0.0, 0.0, 0.0), "mu": 0.5}
    c = {"j1": [0], "j2": [1], "normal": [[0.0, 0.0, 1.0]], "xi": [0.0]}
    for speed, want in ((1e-10, (1.0, 0.0)), (3e-9, (-1.0, 0.0))):
        F = _features(c, [[speed, 0.0, 0.0]], np.zeros((1, 3)), [0.5], [0.5], [5.0], params, 1e3)
        assert tuple(F[0, 12:14]) == want, (speed, F[0, 12:14])


def test_rounded_gradient_reference():
    """The reference of the tensor-core training (operands of the products
    rounded, sums exact): with the identity as rounding it is the exact
    gradient (so it has every term of the chain rule and no transposed
    operand); with bfloat16 it stays within bfloat16's relative precision of
    the exact gradient; each rounding point matters (rounding only the
    deltas, or only the weights, moves the result)."""
    rng = np.random.default_rng(3)
    theta = mlp.init(2) + rng.normal(0, 0.05, mlp.N_PARAMS)
    X = rng.normal(size=(257, 12))
    T = rng.normal(size=(257, 3))
    L, g = mlp.loss_and_grad(theta, X, T)
    Li, gi = mlp.loss_and_grad_rounded(theta, X, T, rnd=lambda a: a)
    assert abs(Li - L) <= 1e-14 * L and np.abs(gi - g).max() <= 1e-12 * np.abs(g).max()
    Lb, gb = mlp.loss_and_grad_rounded(theta, X, T)
    cos = np.dot(gb, g) / (np.linalg.norm(gb) * np.linalg.norm(g))
    assert abs(Lb - L) <= 2e-2 * L and cos > 1 - 1e-3 and np.abs(gb - g).max() > 1e-6 * np.abs(g).max()
    # a product operand that escapes the rounding changes the result
    calls = []

    def spy(a):
        calls.append(np.shape(a))
        return mlp.bf16_round(a)
    mlp.loss_and_grad_rounded(theta, X, T, rnd=spy)
    # forward: X, 4 weights, 3 activations; backward: 4 deltas, 3 weights
    assert len(calls) == 1 + 4 + 3 + 4 + 3
