"""Pins of the oracle's lagged IPC friction on point-triangle pairs (§6.4
friction potential, with lagged contact point, tangent basis and contact
force).

Fixed by: the profile's closed forms (stick value mu fn yh dt / 3, sliding
force magnitude mu fn -- Coulomb's law -- and stick stiffness
mu fn 2 / (yh dt)), its C^2 continuity at y = yh; central differences of
E -> g and g -> H in both regimes; invariance to the choice of tangent
basis; zero cost of normal motion and of rigid translation; PSD Hessians;
the lag data against closed forms (barycentrics of a face point, an edge
point, a vertex; fn = -b'(d) against a finite difference of b); and one
Newton step of a point sliding over a fixed triangle, whose tangential
velocity drops by exactly mu fn dt / m (Coulomb) in the sliding regime.
"""
import numpy as np
import pytest

from oracle import oracle as orc

MU, YH, DT, DHAT, KAPPA = 0.4, 1e-3, 0.01, 1e-3, 1e4


def _tri(seed=0):
    rng = np.random.default_rng(seed)
    a = np.array([0.0, 0.0, 0.0]) + rng.uniform(-0.01, 0.01, 3)
    b = np.array([1.0, 0.1, 0.0]) + rng.uniform(-0.01, 0.01, 3)
    c = np.array([0.2, 1.0, 0.05]) + rng.uniform(-0.01, 0.01, 3)
    return a, b, c


def _normal(a, b, c):
    n = np.cross(b - a, c - a)
    return n / np.linalg.norm(n)


def _lag(xe):
    lag = orc.friction_lag(xe.reshape(4, 3), np.array([[0, 1, 2, 3]]), DHAT, KAPPA)
    return {k: v[0] for k, v in lag.items()}


def _face_stencil(seed=0, d=4e-4, bary=(0.3, 0.3, 0.4)):
    a, b, c = _tri(seed)
    n = _normal(a, b, c)
    p = bary[0] * a + bary[1] * b + bary[2] * c + d * n
    return np.concatenate([p, a, b, c]), n


def _el(xe, lag, mu=MU, yh=YH, dt=DT):
    return orc.friction_element(xe, lag["beta"], lag["T"], lag["fn"], lag["dxt"], mu, yh, dt)


def test_lag_data_closed_forms():
    xe, n = _face_stencil(1, d=4e-4, bary=(0.2, 0.5, 0.3))
    lag = _lag(xe)
    assert np.allclose(lag["beta"], [0.2, 0.5, 0.3], atol=1e-12)
    assert np.allclose(lag["dxt"], 4e-4 * n, atol=1e-15)
    T = lag["T"]
    # n from p - c at |p - c| = 4e-4 carries ~1e-16 / 4e-4 relative rounding
    assert np.allclose(T @ T.T, np.eye(2), atol=1e-14) and np.abs(T @ n).max() <= 2e-12
    # fn = -b'(d): central difference of b(d) = -kappa (d - dhat)^2 ln(d/dhat)
    b = lambda d: -KAPPA * (d - DHAT) ** 2 * np.log(d / DHAT)
    h = 1e-9
    assert lag["fn"] == pytest.approx(-(b(4e-4 + h) - b(4e-4 - h)) / (2 * h), rel=1e-6)
    assert lag["fn"] > 0
    # outside dhat: no contact force
    xe2, _ = _face_stencil(1, d=2e-3)
    assert _lag(xe2)["fn"] == 0.0
    # edge region: beyond edge (a, b), the closest point on that edge
    a, b, c = _tri(2)
    n = _normal(a, b, c)
    m = 0.7 * a + 0.3 * b
    out = np.cross(n, b - a); out /= np.linalg.norm(out)
    if np.dot(out, c - a) > 0:
        out = -out
    p = m + 2e-4 * out + 1e-4 * n
    lag = _lag(np.concatenate([p, a, b, c]))
    assert np.allclose(lag["beta"], [0.7, 0.3, 0.0], atol=1e-12)
    # vertex region
    p = a + 1e-4 * (a - (b + c) / 2) / np.linalg.norm(a - (b + c) / 2) + 1e-4 * n
    assert np.allclose(_lag(np.concatenate([p, a, b, c]))["beta"], [1, 0, 0])


def _slide(xe, lag, s, direction):
    """Move the point by s along a unit tangent direction (triangle fixed)."""
    x = xe.copy()
    x[:3] += s * direction
    return x


def test_profile_closed_forms_and_coulomb_force():
    xe, n = _face_stencil(3)
    lag = _lag(xe)
    fn = lag["fn"]
    t = lag["T"][0] * 0.6 + lag["T"][1] * 0.8
    # stick value at zero slide
    E0, g0, H0 = _el(xe, lag)
    assert E0 == pytest.approx(MU * fn * YH * DT / 3, rel=1e-14)
    # (the lag state's separation is re-formed in another rounding order)
    assert np.abs(g0).max() <= 1e-9 * MU * fn
    # stick stiffness along the slide direction: mu fn 2 / (yh dt)
    assert t @ H0[:3, :3] @ t == pytest.approx(MU * fn * 2 / (YH * DT), rel=1e-9)
    # sliding (y = 3 yh): E = mu fn s, force on the point = mu fn along -t (Coulomb)
    s = 3 * YH * DT
    E, g, H = _el(_slide(xe, lag, s, t), lag)
    assert E == pytest.approx(MU * fn * s, rel=1e-12)
    assert np.allclose(g[:3], MU * fn * t, rtol=1e-12, atol=1e-12 * MU * fn)
    assert np.allclose(g[3:].reshape(3, 3).sum(0), -MU * fn * t, rtol=1e-12,
                       atol=1e-12 * MU * fn)


def test_profile_c2_at_threshold():
    xe, n = _face_stencil(4)
    lag = _lag(xe)
    t = lag["T"][0]
    s = YH * DT
    eps = 1e-9 * s
    Em, gm, Hm = _el(_slide(xe, lag, s - eps, t), lag)
    Ep, gp, Hp = _el(_slide(xe, lag, s + eps, t), lag)
    assert Ep == pytest.approx(Em, rel=1e-8)
    assert np.allclose(gp, gm, rtol=1e-7, atol=1e-7 * np.abs(gm).max())
    # second derivative along t vanishes on both sides at the threshold
    assert abs(t @ Hm[:3, :3] @ t) <= 1e-6 * MU * lag["fn"] / s
    assert abs(t @ Hp[:3, :3] @ t) <= 1e-6 * MU * lag["fn"] / s


@pytest.mark.parametrize("seed,slide", [(0, 0.3), (1, 0.8), (2, 2.5), (3, 10.0)])
def test_derivatives_match_central_differences(seed, slide):
    xe, n = _face_stencil(seed)
    lag = _lag(xe)
    rng = np.random.default_rng(seed)
    x = xe + rng.normal(size=12) * slide * YH * DT
    E, g, H = _el(x, lag)
    h = 1e-4 * YH * DT   # the cubic profile: truncation h^2/6 mu fn 2/(yh dt)^2
    gfd = np.zeros(12); Hfd = np.zeros((12, 12))
    for k in range(12):
        d = np.zeros(12); d[k] = h
        Ep, gp, _ = _el(x + d, lag)
        Em, gm, _ = _el(x - d, lag)
        gfd[k] = (Ep - Em) / (2 * h)
        Hfd[:, k] = (gp - gm) / (2 * h)
    assert np.linalg.norm(g - gfd) <= 1e-6 * np.linalg.norm(g)
    assert np.linalg.norm(H - Hfd) <= 1e-5 * np.linalg.norm(H)
    assert np.linalg.eigvalsh(H).min() >= -1e-10 * np.abs(H).max()


def test_tangent_basis_invariance_normal_motion_and_translation():
    xe, n = _face_stencil(5)
    lag = _lag(xe)
    x = xe + np.random.default_rng(2).normal(size=12) * YH * DT
    E, g, H = _el(x, lag)
    th = 0.7
    Q = np.array([[np.cos(th), -np.sin(th)], [np.sin(th), np.cos(th)]])
    lag2 = dict(lag, T=Q @ lag["T"])
    E2, g2, H2 = _el(x, lag2)
    assert E2 == pytest.approx(E, rel=1e-13)
    assert np.allclose(g2, g, rtol=1e-12, atol=1e-12 * np.abs(g).max())
    assert np.allclose(H2, H, rtol=1e-12, atol=1e-12 * np.abs(H).max())
    # normal motion of the point and rigid translation cost nothing
    E0 = _el(xe, lag)[0]
    assert _el(_slide(xe, lag, 3e-4, n), lag)[0] == pytest.approx(E0, rel=1e-12)
    assert _el(xe + np.tile([0.3, -0.2, 0.1], 4), lag)[0] == pytest.approx(E0, rel=1e-9)


def test_newton_step_sliding_point_loses_coulomb_impulse():
    """A free point of mass m over a pinned triangle, moving tangentially
    at v0 well above the slide threshold: barrier + friction, no gravity.
    The barrier force is normal (face region), so the tangential velocity
    after one step is v0 - mu fn dt / m with fn the lagged contact force."""
    a, b, c = _tri(6)
    n = _normal(a, b, c)
    p = 0.3 * a + 0.3 * b + 0.4 * c + 5e-4 * n
    X = np.array([p, a, b, c])
    t = np.cross(n, b - a); t /= np.linalg.norm(t)
    m = 1.0   # mu fn dt / m ~ 0.08 m/s < v0: stays in the sliding regime
    v0 = 0.5 * t
    pairs = np.array([[0, 1, 2, 3]], np.int32)
    sc = orc.Scene(4, mass=np.array([m, 1.0, 1.0, 1.0]),
                   pt={"pairs": pairs, "dhat": DHAT, "kappa": KAPPA},
                   fr={"pairs": pairs, "mu": MU, "yhat": YH, "dhat": DHAT, "kappa": KAPPA},
                   pinned=[1, 2, 3])
    v = np.zeros((4, 3)); v[0] = v0
    x1, v1, st, rep = sc.newton_step(X, v, DT, gravity=(0.0, 0.0, 0.0), newton_tol=1e-10,
                                     pcg_tol=1e-14)
    assert st == 0, rep
    fn = sc.fr["fn"][0]
    assert fn > 0
    vt = v1[0] @ t
    assert vt == pytest.approx(0.5 - MU * fn * DT / m, rel=1e-8)
    # no tangential motion across the slide direction
    assert abs(v1[0] @ np.cross(n, t)) <= 1e-10


def test_exact_zero_slide_takes_the_limits():
    """Exactly representable configuration: the lag state's separation is
    re-formed exactly, so s = 0 and the limits apply: E = mu fn yh dt / 3,
    g = 0, H = mu fn 2/(yh dt) J^T J; and they agree with a tiny slide."""
    xe = np.array([0.25, 0.25, 5e-4, 0, 0, 0, 1, 0, 0, 0, 1, 0], float)
    lag = _lag(xe)
    assert np.array_equal(lag["beta"], [0.5, 0.25, 0.25])
    E0, g0, H0 = _el(xe, lag)
    fn = lag["fn"]
    assert E0 == MU * fn * DT * YH / 3.0 and not g0.any()
    c = np.array([1.0, -0.5, -0.25, -0.25])
    P = np.eye(3) - np.outer([0, 0, 1.0], [0, 0, 1.0])     # T^T T
    Hexp = MU * fn * 2 / (YH * DT) * np.kron(np.outer(c, c), P)
    assert np.allclose(H0, Hexp, rtol=1e-12, atol=1e-12 * np.abs(Hexp).max())
    x = xe.copy(); x[0] += 1e-8 * YH * DT
    E1, g1, H1 = _el(x, lag)
    assert E1 == pytest.approx(E0, rel=1e-12)
    assert np.allclose(H1, H0, rtol=1e-6, atol=1e-6 * np.abs(H0).max())
