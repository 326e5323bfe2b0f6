"""Pins of the oracle's high-order Lagrange tets (§6.2 Eq. 12; App. A
shape functions): 10-node quadratic and 20-node cubic SNH elements with a
quadrature sum.

Fixed by: the shape functions' Kronecker property at the nodes, partition
of unity and exact reproduction of every polynomial up to the element's
order (random polynomials, numpy); reference gradients against central
differences; the quadrature rules' exactness on monomials (the closed form
a! b! c! / (a+b+c+3)!); the affine patch test (under an affine map a
straight-sided element has F = A at every point, so E equals the linear
tet's V psi(A), the virtual work of an affine variation is V P:dA, and so is
the Hessian form); E = g = 0 at rest also for a curved element; central
differences of E -> g and g -> H at curved states; rotation invariance;
the per-point F-space projection giving a PSD Hessian; and the rest Hessian
against the linear-elastic energy of quadratic / cubic displacement fields
integrated from their analytic strain.
"""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes

MU, LAM = 3.0e4, 8.0e4
EDGES = [(0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3)]
FACES = [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)]
VERT = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)


def _ref_nodes(K):
    """Reference positions of the local nodes (the documented order)."""
    pts = [v for v in VERT]
    if K == 10:
        pts += [(VERT[i] + VERT[j]) / 2 for i, j in EDGES]
    elif K == 20:
        for i, j in EDGES:
            pts += [(2 * VERT[i] + VERT[j]) / 3, (VERT[i] + 2 * VERT[j]) / 3]
        pts += [(VERT[i] + VERT[j] + VERT[k]) / 3 for i, j, k in FACES]
    return np.array(pts)


def _order(K):
    return {4: 1, 10: 2, 20: 3}[K]


@pytest.mark.parametrize("K", [4, 10, 20])
def test_shape_functions(K):
    nodes = _ref_nodes(K)
    for b in range(K):
        N, _ = orc.tetho_shape(K, nodes[b])
        assert np.allclose(N, np.eye(K)[b], atol=1e-14)
    rng = np.random.default_rng(K)
    p = _order(K)
    mons = [(a, b, c) for a in range(p + 1) for b in range(p + 1) for c in range(p + 1)
            if a + b + c <= p]
    for _ in range(5):
        xi = rng.dirichlet(np.ones(4))[1:]
        N, dN = orc.tetho_shape(K, xi)
        assert N.sum() == pytest.approx(1.0, abs=1e-14)
        assert np.abs(dN.sum(0)).max() <= 1e-13
        # reproduction of a random polynomial of degree <= order
        coef = rng.normal(size=len(mons))
        f = lambda z: sum(cc * z[0] ** a * z[1] ** b * z[2] ** c
                          for cc, (a, b, c) in zip(coef, mons))
        assert N @ np.array([f(nd) for nd in nodes]) == pytest.approx(f(xi), abs=1e-12)
        h = 1e-6
        for m in range(3):
            d = np.zeros(3); d[m] = h
            Np, _ = orc.tetho_shape(K, xi + d)
            Nm, _ = orc.tetho_shape(K, xi - d)
            assert np.allclose((Np - Nm) / (2 * h), dN[:, m], atol=1e-8)


@pytest.mark.parametrize("rule,deg", [(scenes.tet_rule_4point(), 2), (scenes.tet_rule_conical(2), 1),
                                      (scenes.tet_rule_conical(3), 3),
                                      (scenes.tet_rule_conical(4), 5)])
def test_quadrature_rules_exact(rule, deg):
    assert rule[:, 0].sum() == pytest.approx(1 / 6, rel=1e-14)
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            for c in range(deg + 1 - a - b):
                q = np.sum(rule[:, 0] * rule[:, 1] ** a * rule[:, 2] ** b * rule[:, 3] ** c)
                exact = math.factorial(a) * math.factorial(b) * math.factorial(c) / \
                    math.factorial(a + b + c + 3)
                assert q == pytest.approx(exact, rel=1e-12, abs=1e-16)


def _element(K, seed=0):
    """A straight-sided element on a random tet (nodes at their Lagrange
    positions) and its 4-node corner tet."""
    rng = np.random.default_rng(seed)
    X4 = VERT + rng.uniform(-0.2, 0.2, (4, 3))
    if np.linalg.det((X4[1:] - X4[0]).T) < 0:
        X4 = X4[[0, 2, 1, 3]]
    lam = np.column_stack([1 - _ref_nodes(K).sum(1), _ref_nodes(K)])   # barycentric
    return lam @ X4, X4


def _rule(K):
    return scenes.tet_rule_4point() if K == 10 else scenes.tet_rule_conical(3)


@pytest.mark.parametrize("K", [10, 20])
def test_affine_patch_equals_linear_tet(K):
    Xe, X4 = _element(K, 1)
    rng = np.random.default_rng(5)
    A = np.eye(3) + rng.uniform(-0.25, 0.25, (3, 3))
    b = rng.normal(size=3)
    xe = Xe @ A.T + b
    bad, E, g, H = orc.tetho_element(K, _rule(K), Xe, xe, MU, LAM)
    assert bad == 0
    Dminv, V, _ = orc.tet_rest(X4, np.array([[0, 1, 2, 3]], np.int32))
    E4, g4, H4 = orc.snh_element((X4 @ A.T + b).ravel(), Dminv[0], V[0], MU, LAM)
    assert E == pytest.approx(E4, rel=1e-12)
    # virtual work of an affine variation dx = dA X, and the Hessian form
    for _ in range(3):
        dA = rng.normal(size=(3, 3))
        dx = (Xe @ dA.T).ravel()
        dx4 = (X4 @ dA.T).ravel()
        assert dx @ g == pytest.approx(dx4 @ g4, rel=1e-11)
        assert dx @ H @ dx == pytest.approx(dx4 @ H4 @ dx4, rel=1e-11)


def _curved(K, seed, amp_rest=0.03, amp=0.08):
    Xe, _ = _element(K, seed)
    rng = np.random.default_rng(100 + seed)
    Xc = Xe.copy()
    Xc[4:] += rng.uniform(-amp_rest, amp_rest, Xc[4:].shape)   # curved rest element
    xe = Xc + rng.uniform(-amp, amp, Xc.shape)
    return Xc, xe


@pytest.mark.parametrize("K", [10, 20])
def test_rest_energy_zero_for_curved_element(K):
    Xc, _ = _curved(K, 2)
    bad, E, g, H = orc.tetho_element(K, _rule(K), Xc, Xc, MU, LAM)
    assert bad == 0 and abs(E) <= 1e-20 * MU and np.abs(g).max() <= 1e-9 * MU
    assert np.abs(H - H.T).max() <= 1e-12 * np.abs(H).max()


@pytest.mark.parametrize("K", [10, 20])
def test_derivatives_match_central_differences(K):
    Xc, xe = _curved(K, 3)
    rule = _rule(K)
    bad, E, g, H = orc.tetho_element(K, rule, Xc, xe, MU, LAM)
    h = 1e-6
    n3 = 3 * K
    gfd = np.zeros(n3); Hfd = np.zeros((n3, n3))
    for k in range(n3):
        d = np.zeros(n3); d[k] = h
        _, Ep, gp, _ = orc.tetho_element(K, rule, Xc, (xe.ravel() + d).reshape(K, 3), MU, LAM)
        _, Em, gm, _ = orc.tetho_element(K, rule, Xc, (xe.ravel() - d).reshape(K, 3), MU, LAM)
        gfd[k] = (Ep - Em) / (2 * h)
        Hfd[:, k] = (gp - gm) / (2 * h)
    assert np.linalg.norm(g - gfd) <= 1e-6 * np.linalg.norm(g)
    assert np.linalg.norm(H - Hfd) <= 1e-6 * np.linalg.norm(H)


@pytest.mark.parametrize("K", [10, 20])
def test_rotation_invariance_and_projection(K):
    Xc, xe = _curved(K, 4, amp=0.2)
    q, _ = np.linalg.qr(np.random.default_rng(7).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    rule = _rule(K)
    _, E, g, H = orc.tetho_element(K, rule, Xc, xe, MU, LAM)
    _, Er, gr, Hr = orc.tetho_element(K, rule, Xc, xe @ q.T, MU, LAM)
    Q = np.kron(np.eye(K), q)
    assert Er == pytest.approx(E, rel=1e-12)
    assert np.linalg.norm(gr - Q @ g) <= 1e-11 * np.linalg.norm(g)
    assert np.linalg.norm(Hr - Q @ H @ Q.T) <= 1e-11 * np.linalg.norm(H)
    _, Ep, gp, Hp = orc.tetho_element(K, rule, Xc, xe, MU, LAM, project=True)
    assert Ep == E and np.array_equal(gp, g)
    w = np.linalg.eigvalsh(Hp)
    assert w.min() >= -1e-10 * np.abs(w).max()
    assert np.linalg.eigvalsh(Hp - H).min() >= -1e-10 * np.abs(w).max()


def test_mesh_generator_shares_nodes():
    for order in (2, 3):
        m = scenes.kuhn_box_ho(2, 2, 2, order, h=0.5, jitter=0.0)
        K = m["tets"].shape[1]
        rule = _rule(K)
        # rest: every element has positive Jacobians, and E = 0
        T = m["tets"].shape[0]
        E, g, H, bad = orc.tetho_batch(K, m["X"], m["X"], m["tets"], rule, np.full(T, MU),
                                       np.full(T, LAM), level=1)
        assert bad == 0 and np.abs(E).max() <= 1e-20
        # conformity: the assembled rest gradient is zero and a global affine
        # field has the affine virtual work of the whole box
        gg, _ = orc.tetho_assemble(m["X"].shape[0], m["tets"], g, None)
        assert np.abs(gg).max() <= 1e-9
        # node count of a conforming mesh: (2 order + 1)^3 grid points
        # for order 2; order 3 adds face nodes (not on a grid)
        if order == 2:
            assert m["X"].shape[0] == 5 ** 3


@pytest.mark.parametrize("K,deg", [(10, 2), (20, 3)])
def test_rest_hessian_is_linear_elasticity_for_polynomial_fields(K, deg):
    """At rest the SNH Hessian (mu' = 4mu/3, lambda' = lambda + 5mu/6) is the
    linear-elastic stiffness with (mu, lambda). For a displacement field u(X)
    that is a polynomial of the element's order (reproduced exactly by a
    straight-sided element), u^T H u equals the integral of
    2 mu |eps(u)|^2 + lambda tr(eps(u))^2, computed here from the analytic
    strain of u on a conical rule exact for the integrand's degree."""
    Xe, X4 = _element(K, 11)
    rng = np.random.default_rng(K)
    young, nu = 1e5, 0.3
    mu = young / (2 * (1 + nu)); lam = young * nu / ((1 + nu) * (1 - 2 * nu))
    mus, lams = orc.snh_lame(young, nu)
    mons = [(a, b, c) for a in range(deg + 1) for b in range(deg + 1) for c in range(deg + 1)
            if 1 <= a + b + c <= deg]
    coef = rng.normal(size=(3, len(mons))) * 0.1

    def u_of(X):
        return np.array([sum(coef[i, k] * X[0] ** a * X[1] ** b * X[2] ** c
                             for k, (a, b, c) in enumerate(mons)) for i in range(3)])

    def grad_u(X):
        G = np.zeros((3, 3))
        for i in range(3):
            for k, (a, b, c) in enumerate(mons):
                e = (a, b, c)
                for j in range(3):
                    if e[j] == 0:
                        continue
                    p = list(e); p[j] -= 1
                    G[i, j] += coef[i, k] * e[j] * X[0] ** p[0] * X[1] ** p[1] * X[2] ** p[2]
        return G

    # the oracle's rest Hessian with a rule exact for the integrand
    # (products of two gradients: degree 2 (deg - 1))
    rule = scenes.tet_rule_conical(4)
    bad, E, g, H = orc.tetho_element(K, rule, Xe, Xe, mus[0], lams[0])
    assert bad == 0
    uvec = np.concatenate([u_of(x) for x in Xe])
    # the reference integral over the physical tet: X(xi) = X0 + Dm xi
    Dm = (X4[1:] - X4[0]).T
    det = np.linalg.det(Dm)
    ref = 0.0
    for w, *xi in rule:
        X = X4[0] + Dm @ np.array(xi)
        Gu = grad_u(X)
        eps = 0.5 * (Gu + Gu.T)
        ref += w * det * (2 * mu * np.sum(eps * eps) + lam * np.trace(eps) ** 2)
    assert uvec @ H @ uvec == pytest.approx(ref, rel=1e-10)
