"""Pins of the oracle's other tet4 densities (§6.1 "Non-Linear Material
Models", App. B): Neo-Hookean, St. Venant-Kirchhoff, fixed co-rotational
and ARAP with a volume term, the last two with a lagged rotation R.

Fixed by: the small-strain limit of linear elasticity (textbook stiffness,
numpy), exactly for NH and StVK and on symmetric strains for the lagged
co-rotational models (whose lagged R makes an infinitesimal rotation cost
2 mu |W|^2 resp. mu |W|^2 per unit volume, in closed form); central
differences of E -> g and g -> H; rotation invariance (of x, and of x with
R for the lagged models); E = g = 0 at rest; the second-order accuracy of
the energy at strains of 1e-6 (which fails without the cancellation-free
forms); the densities' plain definitions at large strain (numpy); the
polar rotation in closed form for F = Q S and for an inverted F; and the
invalid state of NH (J <= 0).
"""
import numpy as np
import pytest

from oracle import oracle as orc

MODELS = [orc.MODEL_NH, orc.MODEL_STVK, orc.MODEL_COROT, orc.MODEL_ARAP]
MU, LAM = 3.0e4, 8.0e4


def _tet(seed, jitter=0.2):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    X += rng.uniform(-jitter, jitter, X.shape)
    if np.linalg.det((X[1:] - X[0]).T) < 0:
        X = X[[0, 2, 1, 3]]
    return X


def _elem(X):
    Dminv, V, bad = orc.tet_rest(X, np.array([[0, 1, 2, 3]], np.int32))
    assert bad == 0
    return Dminv[0], V[0]


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


def _F(X, x):
    return (x[1:] - x[0]).T @ np.linalg.inv((X[1:] - X[0]).T)


def _linear_elastic_K(X, mu, lam):
    """u^T K u = V (2 mu |eps|^2 + lam tr(eps)^2), eps = sym(grad u) (numpy)."""
    Dmi = np.linalg.inv((X[1:] - X[0]).T)
    V = np.linalg.det((X[1:] - X[0]).T) / 6.0
    basis = np.eye(12)

    def eps_of(u):
        u = u.reshape(4, 3)
        Gu = (u[1:] - u[0]).T @ Dmi
        return 0.5 * (Gu + Gu.T)

    E = [eps_of(basis[k]) for k in range(12)]
    K = np.zeros((12, 12))
    for a in range(12):
        for b in range(12):
            K[a, b] = V * (2 * mu * np.sum(E[a] * E[b]) + lam * np.trace(E[a]) * np.trace(E[b]))
    return K


def _el(model, X, x, R=None, mu=MU, lam=LAM):
    Dminv, V = _elem(X)
    bad, E, g, H = orc.tet_element(model, x.ravel(), Dminv, V, mu, lam, R)
    assert bad == 0
    return E, g, H


@pytest.mark.parametrize("model", [orc.MODEL_NH, orc.MODEL_STVK])
@pytest.mark.parametrize("seed", range(3))
def test_rest_hessian_is_linear_elasticity(model, seed):
    X = _tet(seed)
    E, g, H = _el(model, X, X)
    assert abs(E) <= 1e-20 * MU and np.abs(g).max() <= 1e-9 * MU
    K = _linear_elastic_K(X, MU, LAM)
    assert np.linalg.norm(H - K) <= 1e-12 * np.linalg.norm(K)


@pytest.mark.parametrize("model,scale", [(orc.MODEL_COROT, 1.0), (orc.MODEL_ARAP, 0.5)])
def test_lagged_models_small_strain(model, scale):
    """With R = I at rest: a symmetric strain u = S X costs the
    linear-elastic energy with (scale mu, lambda); an infinitesimal
    rotation u = W X (W skew) is not followed by the lagged R, so
    psi = scale mu |W|^2 eps^2 + O(eps^3) and u^T H u = 2 V scale mu |W|^2."""
    X = _tet(4)
    E, g, H = _el(model, X, X, np.eye(3))
    assert abs(E) <= 1e-20 * MU and np.abs(g).max() <= 1e-9 * MU
    K = _linear_elastic_K(X, scale * MU, LAM)
    rng = np.random.default_rng(9)
    Dminv, V = _elem(X)
    for _ in range(4):
        S = rng.normal(size=(3, 3)); S = S + S.T
        u = (X @ S.T).ravel()
        assert u @ H @ u == pytest.approx(u @ K @ u, rel=1e-12)
        W = rng.normal(size=(3, 3)); W = W - W.T
        u = (X @ W.T).ravel()
        # psi = scale mu |W|^2 eps^2 (J - 1 = O(eps^2)): u^T H u = 2 V scale mu |W|^2
        assert u @ H @ u == pytest.approx(2 * V * scale * MU * np.sum(W * W), rel=1e-12)


def test_arap_is_corot_with_half_mu():
    X = _tet(5)
    x = X + np.random.default_rng(1).uniform(-0.2, 0.2, X.shape)
    R = _rot(2)
    Ea, ga, Ha = _el(orc.MODEL_ARAP, X, x, R, MU, LAM)
    Ec, gc, Hc = _el(orc.MODEL_COROT, X, x, R, MU / 2, LAM)
    assert Ea == pytest.approx(Ec, rel=1e-14)
    assert np.allclose(ga, gc, rtol=1e-13, atol=1e-13 * np.abs(gc).max())
    assert np.allclose(Ha, Hc, rtol=1e-13, atol=1e-13 * np.abs(Hc).max())


def _state(seed, amp=0.25):
    X = _tet(seed)
    x = X + np.random.default_rng(50 + seed).uniform(-amp, amp, X.shape)
    if np.linalg.det(_F(X, x)) <= 0.2:
        x = X + 0.3 * (x - X)
    return X, x


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("seed", range(3))
def test_gradient_and_hessian_match_central_differences(model, seed):
    X, x = _state(seed)
    R = _rot(seed + 20)
    E, g, H = _el(model, X, x, R)
    h = 1e-6
    gfd = np.zeros(12); Hfd = np.zeros((12, 12))
    for k in range(12):
        d = np.zeros(12); d[k] = h
        Ep, gp, _ = _el(model, X, (x.ravel() + d).reshape(4, 3), R)
        Em, gm, _ = _el(model, X, (x.ravel() - d).reshape(4, 3), R)
        gfd[k] = (Ep - Em) / (2 * h)
        Hfd[:, k] = (gp - gm) / (2 * h)
    assert np.linalg.norm(g - gfd) <= 1e-6 * np.linalg.norm(g)
    assert np.linalg.norm(H - Hfd) <= 1e-6 * np.linalg.norm(H)
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("model", MODELS)
def test_rotation_invariance(model):
    X, x = _state(7)
    R = _rot(8)
    q = _rot(11)
    Rq = q @ R if model in (orc.MODEL_COROT, orc.MODEL_ARAP) else R
    E, g, H = _el(model, X, x, R)
    Er, gr, Hr = _el(model, X, x @ q.T, Rq)
    Q = np.kron(np.eye(4), q)
    assert Er == pytest.approx(E, rel=1e-12)
    assert np.linalg.norm(gr - Q @ g) <= 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(Hr - Q @ H @ Q.T) <= 1e-12 * np.linalg.norm(H)


@pytest.mark.parametrize("model", MODELS)
def test_energy_second_order_accurate_at_tiny_strain(model):
    """E(X + eps u) = eps^2/2 u^T H(X) u + O(eps^3): at eps = 1e-6 the
    relative difference is ~1e-6. A density evaluated with O(1) terms
    subtracted from each other would be off by ~1e-4 here."""
    X = _tet(3)
    R = np.eye(3)
    _, _, H0 = _el(model, X, X, R)
    u = np.random.default_rng(2).normal(size=12)
    eps = 1e-6
    E, _, _ = _el(model, X, X + eps * u.reshape(4, 3), R)
    ref = 0.5 * eps * eps * (u @ H0 @ u)
    assert abs(E - ref) <= 1e-5 * abs(ref)


def _plain_psi(model, F, R, mu, lam):
    """The densities' definitions, evaluated directly (valid away from rest)."""
    J = np.linalg.det(F)
    Ic = np.sum(F * F)
    if model == orc.MODEL_NH:
        return 0.5 * mu * (Ic - 3) - mu * np.log(J) + 0.5 * lam * np.log(J) ** 2
    if model == orc.MODEL_STVK:
        E = 0.5 * (F.T @ F - np.eye(3))
        return mu * np.sum(E * E) + 0.5 * lam * np.trace(E) ** 2
    if model == orc.MODEL_COROT:
        return mu * np.sum((F - R) ** 2) + 0.5 * lam * (J - 1) ** 2
    return 0.5 * mu * (Ic - 2 * np.trace(F.T @ R) + 3) + 0.5 * lam * (J - 1) ** 2


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("seed", range(3))
def test_energy_equals_plain_definition_at_large_strain(model, seed):
    X, x = _state(seed, amp=0.35)
    R = _rot(seed + 30)
    Dminv, V = _elem(X)
    E, _, _ = _el(model, X, x, R)
    ref = V * _plain_psi(model, _F(X, x), R, MU, LAM)
    assert E == pytest.approx(ref, rel=1e-11)


def test_nh_inverted_tet_is_invalid():
    X = _tet(1)
    x = X.copy()
    x[3] = X[0] - (X[3] - X[0])     # reflect one vertex through the base: J < 0
    Dminv, V = _elem(X)
    bad, E, g, H = orc.tet_element(orc.MODEL_NH, x.ravel(), Dminv, V, MU, LAM)
    assert bad == 1 and E == 0.0 and not g.any()
    for m in (orc.MODEL_STVK, orc.MODEL_COROT, orc.MODEL_ARAP):
        bad, E, _, _ = orc.tet_element(m, x.ravel(), Dminv, V, MU, LAM, np.eye(3))
        assert bad == 0 and E > 0


def test_lagged_rotation_closed_forms():
    X = _tet(2)
    tets = np.array([[0, 1, 2, 3]], np.int32)
    Dminv, V = _elem(X)
    q = _rot(3)
    rng = np.random.default_rng(4)
    # F = Q S with S symmetric positive definite: R = Q
    A = rng.normal(size=(3, 3)); S = A @ A.T + 0.5 * np.eye(3)
    for F, Rexp in [(q @ S, q), (q @ np.diag([2.0, 1.5, -0.5]), q), (np.eye(3), np.eye(3))]:
        x = X[0] + (X - X[0]) @ F.T
        R = orc.lagged_rotations(x, tets, Dminv[None]).reshape(3, 3)
        assert np.abs(R - Rexp).max() <= 1e-12
        assert np.abs(R @ R.T - np.eye(3)).max() <= 1e-13 and np.linalg.det(R) > 0


def test_scene_newton_step_lagged_rotations_and_validity():
    """Newton steps of a small cube for each model converge; the lagged
    rotations are those of the start-of-step state."""
    from paper_2303_02156_gb300 import scenes
    m = scenes.kuhn_box(3, 3, 3, h=0.1, seed=1)
    T = m["tets"].shape[0]
    for model in MODELS:
        inp, mass, bad = orc.tet_scene_inputs(model, m["X"], m["tets"], np.full(T, 1e5),
                                              np.full(T, 0.3), 1000.0)
        assert bad == 0
        sc = orc.Scene(m["X"].shape[0], mass=mass, snh=inp, pinned=m["pinned"])
        x, v = m["X"].copy(), np.zeros_like(m["X"])
        for _ in range(3):
            x, v, st, rep = sc.newton_step(x, v, 0.01)
            assert st == 0, (model, rep)
        if model in (orc.MODEL_COROT, orc.MODEL_ARAP):
            # the rotations held in the last step are those of its start
            assert np.abs(sc.R.reshape(-1, 3, 3) @ sc.R.reshape(-1, 3, 3).transpose(0, 2, 1)
                          - np.eye(3)).max() <= 1e-12
        E, g, _, bad = sc.eval(x, level=1)
        assert bad == 0
