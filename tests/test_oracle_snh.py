"""Pins of the oracle's Stable Neo-Hookean tet4 element (§3.1 Eq. 7; App. B).

Each check is fixed by something other than the oracle's own formula:
finite differences, the small-strain limit of linear elasticity (textbook),
rest stationarity (App. B chooses alpha for it), rotation and translation
invariance, the rank of the rest Hessian and the paper's function arity.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes


def _tet(seed=0, jitter=0.2):
    rng = np.random.default_rng(seed)
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    X += rng.uniform(-jitter, jitter, X.shape)
    d = np.linalg.det((X[1:] - X[0]).T)
    if d < 0:
        X = X[[0, 2, 1, 3]]
    return X


def _elem(X, mu, lam):
    Dminv, V, bad = orc.tet_rest(X, np.array([[0, 1, 2, 3]], np.int32))
    assert bad == 0
    return Dminv[0], V[0]


def _linear_elastic_K(X, mu, lam):
    """Textbook linear-FEM stiffness of a tet: u^T K u = V (2 mu |eps|^2 +
    lam tr(eps)^2), eps = sym(grad u), grad u = Du Dm^-1 (computed here
    with numpy, independently of the oracle)."""
    Dm = (X[1:] - X[0]).T
    Dmi = np.linalg.inv(Dm)
    V = np.linalg.det(Dm) / 6.0
    K = np.zeros((12, 12))
    basis = np.eye(12)

    def eps_of(u):
        u = u.reshape(4, 3)
        Du = (u[1:] - u[0]).T
        Gu = Du @ Dmi
        return 0.5 * (Gu + Gu.T)

    E = [eps_of(basis[k]) for k in range(12)]
    for a in range(12):
        for b in range(12):
            K[a, b] = V * (2 * mu * np.sum(E[a] * E[b]) + lam * np.trace(E[a]) * np.trace(E[b]))
    return K


@pytest.mark.parametrize("young,nu", [(1e5, 0.3), (3e4, 0.45), (1e6, 0.2)])
def test_small_strain_limit_is_linear_elasticity(young, nu):
    # Rest Hessian of SNH with mu' = 4mu/3, lambda' = lambda + 5mu/6 equals the
    # linear-elastic stiffness with (mu, lambda): pins the App. B reading.
    X = _tet(1)
    mu = young / (2 * (1 + nu)); lam = young * nu / ((1 + nu) * (1 - 2 * nu))
    mus, lams = orc.snh_lame(young, nu)
    assert mus[0] == pytest.approx(4 * mu / 3, rel=1e-15)
    assert lams[0] == pytest.approx(lam + 5 * mu / 6, rel=1e-15)
    Dminv, V = _elem(X, mus[0], lams[0])
    E, g, H = orc.snh_element(X, Dminv, V, mus[0], lams[0])
    K = _linear_elastic_K(X, mu, lam)
    assert np.linalg.norm(H - K) <= 1e-12 * np.linalg.norm(K)


def test_literal_parameters_do_not_match_linear_elasticity():
    # the literal listing (mu' = mu) must NOT reproduce linear elasticity
    X = _tet(2)
    mu = 1e5 / 2.6; lam = 1e5 * 0.3 / (1.3 * 0.4)
    mus, lams = orc.snh_lame(1e5, 0.3, literal=True)
    assert mus[0] == pytest.approx(mu) and lams[0] == pytest.approx(lam)
    Dminv, V = _elem(X, mus[0], lams[0])
    _, _, H = orc.snh_element(X, Dminv, V, mus[0], lams[0])
    K = _linear_elastic_K(X, mu, lam)
    assert np.linalg.norm(H - K) > 1e-3 * np.linalg.norm(K)


@pytest.mark.parametrize("seed", range(4))
def test_rest_energy_and_gradient_zero(seed):
    rng = np.random.default_rng(seed)
    X = _tet(seed)
    mu, lam = rng.uniform(1e3, 1e6), rng.uniform(1e3, 1e6)
    Dminv, V = _elem(X, mu, lam)
    E, g, H = orc.snh_element(X, Dminv, V, mu, lam)
    scale = V * mu
    assert abs(E) <= 1e-12 * scale
    assert np.linalg.norm(g) <= 1e-12 * scale


def _deformed(X, seed, amp=0.15):
    rng = np.random.default_rng(100 + seed)
    return X + rng.uniform(-amp, amp, X.shape)


@pytest.mark.parametrize("seed", range(4))
def test_gradient_matches_central_differences(seed):
    X = _tet(seed); x = _deformed(X, seed)
    mu, lam = 4e4, 9e4
    Dminv, V = _elem(X, mu, lam)
    E, g, H = orc.snh_element(x, Dminv, V, mu, lam)
    h = 1e-6
    gfd = np.zeros(12)
    xf = x.ravel()
    for k in range(12):
        xp = xf.copy(); xp[k] += h
        xm = xf.copy(); xm[k] -= h
        gfd[k] = (orc.snh_element(xp, Dminv, V, mu, lam)[0]
                  - orc.snh_element(xm, Dminv, V, mu, lam)[0]) / (2 * h)
    assert np.linalg.norm(gfd - g) <= 1e-6 * np.linalg.norm(g)


@pytest.mark.parametrize("seed", range(4))
def test_hessian_matches_central_differences(seed):
    X = _tet(seed); x = _deformed(X, seed)
    mu, lam = 4e4, 9e4
    Dminv, V = _elem(X, mu, lam)
    E, g, H = orc.snh_element(x, Dminv, V, mu, lam)
    h = 1e-6
    Hfd = np.zeros((12, 12))
    xf = x.ravel()
    for k in range(12):
        xp = xf.copy(); xp[k] += h
        xm = xf.copy(); xm[k] -= h
        Hfd[:, k] = (orc.snh_element(xp, Dminv, V, mu, lam)[1]
                     - orc.snh_element(xm, Dminv, V, mu, lam)[1]) / (2 * h)
    assert np.linalg.norm(Hfd - H) <= 1e-6 * np.linalg.norm(H)
    assert np.array_equal(H, H.T) or np.linalg.norm(H - H.T) <= 1e-14 * np.linalg.norm(H)


def _rot(seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    return q


@pytest.mark.parametrize("seed", range(3))
def test_rotation_invariance(seed):
    X = _tet(seed); x = _deformed(X, seed)
    mu, lam = 4e4, 9e4
    Dminv, V = _elem(X, mu, lam)
    E, g, H = orc.snh_element(x, Dminv, V, mu, lam)
    R = _rot(seed)
    Er, gr, Hr = orc.snh_element(x @ R.T, Dminv, V, mu, lam)
    RR = np.kron(np.eye(4), R)
    assert Er == pytest.approx(E, rel=1e-12)
    assert np.linalg.norm(gr - RR @ g) <= 1e-12 * np.linalg.norm(g)
    assert np.linalg.norm(Hr - RR @ H @ RR.T) <= 1e-12 * np.linalg.norm(H)


@pytest.mark.parametrize("seed", range(3))
def test_translation_invariance(seed):
    X = _tet(seed); x = _deformed(X, seed)
    mu, lam = 4e4, 9e4
    Dminv, V = _elem(X, mu, lam)
    E, g, H = orc.snh_element(x, Dminv, V, mu, lam)
    assert np.linalg.norm(g.reshape(4, 3).sum(0)) <= 1e-12 * np.linalg.norm(g)
    for t in np.eye(3):
        assert np.linalg.norm(H @ np.tile(t, 4)) <= 1e-12 * np.linalg.norm(H)
    Et, gt, _ = orc.snh_element(x + np.array([0.3, -2.0, 1.1]), Dminv, V, mu, lam)
    assert Et == pytest.approx(E, rel=1e-12)


def test_rest_hessian_rank_six():
    X = _tet(3)
    mu, lam = 5e4, 2e5
    Dminv, V = _elem(X, mu, lam)
    _, _, H = orc.snh_element(X, Dminv, V, mu, lam)
    w = np.linalg.eigvalsh(H)
    tol = 1e-10 * np.abs(w).max()
    assert np.sum(np.abs(w) <= tol) == 6
    assert np.sum(w > tol) == 6


def test_function_arity_matches_paper():
    # §5.2 "Code Generation": the NH tet4 E+grad+Hess function has 26 inputs
    # (12 xe, 12 Xe, mu, lambda) and 157 outputs (1 + 12 + 144).
    X = _tet(0)
    Dminv, V = _elem(X, 1.0, 1.0)
    E, g, H = orc.snh_element(X, Dminv, V, 1.0, 1.0)
    assert 1 + g.size + H.size == 157
    assert X.size + X.size + 2 == 26


def test_inverted_tet_reported_degenerate():
    X = _tet(0)[[0, 2, 1, 3]]
    _, V, bad = orc.tet_rest(X, np.array([[0, 1, 2, 3]], np.int32))
    assert bad == 1 and V[0] < 0


def test_generator_tets_positive_and_mass_sums_to_total():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    Dminv, V, bad = orc.tet_rest(m["X"], m["tets"])
    assert bad == 0 and V.min() > 0
    assert m["tets"].shape == (384, 4) and m["X"].shape == (125, 3)
    mass = orc.lumped_mass(125, m["tets"], V, 1000.0)
    assert mass.sum() == pytest.approx(1000.0 * V.sum(), rel=1e-13)
    # the jittered cube keeps the volume of the unit cube (only boundary
    # nodes change it, and only slightly)
    assert V.sum() == pytest.approx(1.0, rel=0.05)


def _snh_psi_plain(F, mu, lam):
    """App. B's Stable Neo-Hookean density written as printed (with the
    re-parameterized mu', lambda' passed in): psi = mu/2 (Ic - 3)
    + lambda/2 (J - alpha)^2 - mu/2 ln(Ic + 1), alpha = 1 + mu/lambda
    - mu/(4 lambda). Plain numpy, no cancellation-free rewriting."""
    Ic = np.sum(F * F)
    J = np.linalg.det(F)
    alpha = 1.0 + mu / lam - mu / (4.0 * lam)
    return 0.5 * mu * (Ic - 3.0) + 0.5 * lam * (J - alpha) ** 2 - 0.5 * mu * np.log(Ic + 1.0)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("inverted", [False, True])
def test_energy_equals_plain_definition_at_large_strain(seed, inverted):
    # E = V (psi(F) - psi(I)) at strains of order one, including inverted
    # tets (J < 0). At large strain the plain form of App. B has no
    # cancellation, so it checks the value of the oracle's rewritten energy
    # independently of that rewriting.
    rng = np.random.default_rng(100 + seed)
    X = _tet(seed)
    F = np.eye(3) + rng.uniform(-0.6, 0.6, (3, 3))
    if (np.linalg.det(F) < 0) != inverted:
        F[:, 0] *= -1.0
    assert (np.linalg.det(F) < 0) == inverted
    assert abs(np.linalg.det(F)) > 0.05
    young = 10 ** rng.uniform(4, 6); nu = rng.uniform(0.2, 0.45)
    mus, lams = orc.snh_lame(young, nu)
    mu, lam = mus[0], lams[0]
    x = X @ F.T   # x_a = F X_a, so the deformation gradient is F
    Dminv, V = _elem(X, mu, lam)
    E, _, _ = orc.snh_element(x, Dminv, V, mu, lam)
    Eplain = V * (_snh_psi_plain(F, mu, lam) - _snh_psi_plain(np.eye(3), mu, lam))
    assert abs(E - Eplain) <= 1e-12 * V * mu
    # and it is not trivially small: a dropped term would show
    assert abs(Eplain) > 1e-2 * V * mu
