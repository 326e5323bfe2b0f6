"""Pins of the oracle's PSD clamp (§5.2; Algorithm 1 ProjectToPD), hinge
bending (§6.3, Eq. 13) and point-triangle barrier (§6.4, Eq. 15)."""
import math

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes


# ------------------------------------------------------------------ clamp
def _rand_orth(n, rng):
    q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    return q


@pytest.mark.parametrize("seed", range(5))
def test_clamp_known_spectrum(seed):
    rng = np.random.default_rng(seed)
    Q = _rand_orth(12, rng)
    lam = rng.normal(size=12) * 10.0 ** rng.uniform(-3, 3, 12)
    A = Q @ np.diag(lam) @ Q.T
    A = 0.5 * (A + A.T)
    P, sweeps = orc.clamp_psd(A)
    ref = Q @ np.diag(np.maximum(lam, 0)) @ Q.T
    assert sweeps >= 0
    assert np.linalg.norm(P - ref) <= 1e-12 * np.linalg.norm(A)


@pytest.mark.parametrize("seed", range(5))
def test_clamp_matches_library_eigh(seed):
    rng = np.random.default_rng(10 + seed)
    A = rng.normal(size=(12, 12)); A = A + A.T
    w, V = np.linalg.eigh(A)
    ref = (V * np.maximum(w, 0)) @ V.T
    P, _ = orc.clamp_psd(A)
    assert np.linalg.norm(P - ref) <= 1e-12 * np.linalg.norm(A)
    # output PSD, idempotent, symmetric
    assert np.linalg.eigvalsh(P).min() >= -1e-14 * np.linalg.norm(A)
    P2, _ = orc.clamp_psd(P)
    assert np.linalg.norm(P2 - P) <= 1e-13 * np.linalg.norm(A)
    assert np.linalg.norm(P - P.T) <= 1e-14 * np.linalg.norm(A)


def test_clamp_psd_input_unchanged_and_diagonal():
    rng = np.random.default_rng(3)
    B = rng.normal(size=(12, 12)); A = B @ B.T
    P, _ = orc.clamp_psd(A)
    assert np.linalg.norm(P - A) <= 1e-13 * np.linalg.norm(A)
    d = rng.normal(size=12)
    P, sweeps = orc.clamp_psd(np.diag(d))
    assert sweeps == 0
    assert np.array_equal(P, np.diag(np.maximum(d, 0)))


def test_clamp_repeated_eigenvalues():
    rng = np.random.default_rng(4)
    Q = _rand_orth(12, rng)
    lam = np.array([-2, -2, -2, 0, 0, 0, 1, 1, 3, 3, 3, 5.0])
    A = Q @ np.diag(lam) @ Q.T
    P, _ = orc.clamp_psd(0.5 * (A + A.T))
    ref = Q @ np.diag(np.maximum(lam, 0)) @ Q.T
    assert np.linalg.norm(P - ref) <= 1e-12 * np.linalg.norm(A)


def test_clamp_of_deformed_snh_hessian_is_psd():
    X = scenes.two_tet()["X"][:4]
    Dminv, V, _ = orc.tet_rest(X, np.array([[0, 1, 2, 3]], np.int32))
    x = X + np.random.default_rng(5).uniform(-0.3, 0.3, X.shape)
    _, _, H = orc.snh_element(x, Dminv[0], V[0], 1e4, 1e5)
    assert np.linalg.eigvalsh(H).min() < 0  # this state is indefinite
    P, _ = orc.clamp_psd(H)
    w, Vv = np.linalg.eigh(H)
    assert np.linalg.norm(P - (Vv * np.maximum(w, 0)) @ Vv.T) <= 1e-12 * np.linalg.norm(H)


# ------------------------------------------------------------------ hinge
def _sheet():
    return scenes.shell_sheet(4, length=1.0, noise=0.0, seed=0)


def test_hinge_weights_annihilate_flat_and_affine_images():
    sh = _sheet()
    rng = np.random.default_rng(0)
    A = rng.normal(size=(3, 3)); b = rng.normal(size=3)
    for k in range(sh["hinges"].shape[0]):
        st = sh["hinges"][k]
        xe = sh["X"][st]
        E, g, H = orc.hinge_element(xe, sh["q"][k], sh["c"][k], 1e-3)
        scale = 1e-3 * sh["c"][k] * np.sum(sh["q"][k] ** 2)
        assert abs(E) <= 1e-14 * scale and np.linalg.norm(g) <= 1e-13 * scale
        E2, g2, _ = orc.hinge_element(xe @ A.T + b, sh["q"][k], sh["c"][k], 1e-3)
        assert abs(E2) <= 1e-12 * scale and np.linalg.norm(g2) <= 1e-12 * scale


def test_hinge_Q_symmetric_psd_rank3_and_quadratic():
    sh = _sheet()
    k = 7
    st = sh["hinges"][k]
    xe = sh["X"][st].copy()
    xe[2, 2] += 0.01; xe[3, 2] += 0.02
    E, g, H = orc.hinge_element(xe, sh["q"][k], sh["c"][k], 1e-3)
    w = np.linalg.eigvalsh(H)
    assert np.allclose(H, H.T, rtol=0, atol=0)
    assert w.min() >= -1e-15 * w.max() and np.sum(w > 1e-12 * w.max()) == 3
    # exact quadratic: E = 1/2 x^T H x, g = H x
    assert E == pytest.approx(0.5 * xe.ravel() @ H @ xe.ravel(), rel=1e-12)
    assert np.allclose(g, H @ xe.ravel(), rtol=1e-12, atol=0)
    # folding energy grows as the square of the (small) fold height
    xe2 = sh["X"][st].copy(); xe2[2, 2] += 0.002
    xe4 = sh["X"][st].copy(); xe4[2, 2] += 0.004
    E2 = orc.hinge_element(xe2, sh["q"][k], sh["c"][k], 1e-3)[0]
    E4 = orc.hinge_element(xe4, sh["q"][k], sh["c"][k], 1e-3)[0]
    assert E2 > 0 and E4 / E2 == pytest.approx(4.0, rel=1e-10)


def test_sheet_counts():
    sh = scenes.shell_sheet(10, noise=0.0)
    assert sh["n_tri"] == 200
    assert sh["hinges"].shape[0] == 3 * 100 + 2 * 10 - 4 * 10  # 280 interior edges


# ------------------------------------------------------------------ barrier
DHAT, KAPPA = 1e-3, 1e4


def test_barrier_1d_closed_form():
    b, b1, b2 = orc.barrier_1d(DHAT, DHAT, KAPPA)
    assert b == 0.0 and b1 == 0.0
    for d in [1e-4, 3e-4, 7e-4, 9.9e-4]:
        b, b1, b2 = orc.barrier_1d(d, DHAT, KAPPA)
        assert b > 0 and b1 < 0 and b2 > 0
        h = 1e-9
        fd1 = (orc.barrier_1d(d + h, DHAT, KAPPA)[0] - orc.barrier_1d(d - h, DHAT, KAPPA)[0]) / (2 * h)
        fd2 = (orc.barrier_1d(d + h, DHAT, KAPPA)[1] - orc.barrier_1d(d - h, DHAT, KAPPA)[1]) / (2 * h)
        assert fd1 == pytest.approx(b1, rel=1e-6)
        assert fd2 == pytest.approx(b2, rel=1e-6)


def _tri(seed=0):
    rng = np.random.default_rng(seed)
    T = np.array([[0, 0, 0], [1e-2, 0, 0], [0, 1e-2, 0]], float)
    T += rng.uniform(-2e-3, 2e-3, T.shape)
    return T


def _fd_check(xe, rel=1e-5):
    st, E, g, H = orc.barrier_element(xe, DHAT, KAPPA)
    assert st == 1
    xf = xe.ravel()
    h = 1e-9
    gfd = np.zeros(12); Hfd = np.zeros((12, 12))
    for k in range(12):
        xp = xf.copy(); xp[k] += h
        xm = xf.copy(); xm[k] -= h
        sp = orc.barrier_element(xp, DHAT, KAPPA)
        sm = orc.barrier_element(xm, DHAT, KAPPA)
        gfd[k] = (sp[1] - sm[1]) / (2 * h)
        Hfd[:, k] = (sp[2] - sm[2]) / (2 * h)
    assert np.linalg.norm(gfd - g) <= rel * np.linalg.norm(g)
    assert np.linalg.norm(Hfd - H) <= rel * np.linalg.norm(H)
    assert np.linalg.norm(H - H.T) <= 1e-12 * np.linalg.norm(H)
    return E, g, H


@pytest.mark.parametrize("seed", range(3))
def test_barrier_face_region_reduces_to_1d(seed):
    T = _tri(seed)
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    beta = np.array([0.3, 0.3, 0.4])
    d = 4e-4
    p = beta @ T + d * n
    xe = np.vstack([p, T])
    assert orc.pt_region(xe) == 6
    assert orc.pt_distance(xe) == pytest.approx(d, rel=1e-12)
    E, g, H = _fd_check(xe)
    b, b1, b2 = orc.barrier_1d(d, DHAT, KAPPA)
    assert E == pytest.approx(b, rel=1e-12)
    assert np.allclose(g[:3], b1 * n, rtol=1e-10, atol=1e-10 * abs(b1))
    assert np.linalg.norm(g.reshape(4, 3).sum(0)) <= 1e-10 * np.linalg.norm(g)
    # second derivative along the normal for the point is b''
    assert n @ H[:3, :3] @ n == pytest.approx(b2, rel=1e-8)


def test_barrier_edge_and_vertex_regions():
    T = _tri(1)
    # beyond vertex 0, away from the triangle
    c = T.mean(0)
    p = T[0] + 3e-4 * (T[0] - c) / np.linalg.norm(T[0] - c) + np.array([0, 0, 2e-4])
    xe = np.vstack([p, T])
    assert orc.pt_region(xe) == 0
    assert orc.pt_distance(xe) == pytest.approx(np.linalg.norm(p - T[0]), rel=1e-12)
    _fd_check(xe)
    # beyond edge (t0, t1): offset outward in-plane plus a normal offset
    e = T[1] - T[0]; mid = T[0] + 0.4 * e
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    out = np.cross(e, n); out /= np.linalg.norm(out)
    if np.dot(out, T[2] - mid) > 0:
        out = -out
    p = mid + 3e-4 * out + 4e-4 * n
    xe = np.vstack([p, T])
    assert orc.pt_region(xe) == 3
    dline = np.linalg.norm(np.cross(p - T[0], e)) / np.linalg.norm(e)
    assert orc.pt_distance(xe) == pytest.approx(dline, rel=1e-12)
    _fd_check(xe)


def test_barrier_distance_brute_force_and_continuity():
    T = _tri(2)
    rng = np.random.default_rng(0)
    for _ in range(20):
        p = T.mean(0) + rng.uniform(-1.5e-2, 1.5e-2, 3)
        xe = np.vstack([p, T])
        d = orc.pt_distance(xe)
        k = 200
        u, v = np.meshgrid(np.linspace(0, 1, k + 1), np.linspace(0, 1, k + 1))
        m = (u + v) <= 1
        pts = T[0] + np.outer(u[m], T[1] - T[0]) + np.outer(v[m], T[2] - T[0])
        dbf = np.linalg.norm(pts - p, axis=1).min()
        assert d <= dbf * (1 + 1e-12)
        assert dbf - d <= 1.5e-2 / k
    # E and g continuous across the face/edge boundary
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    e = T[1] - T[0]
    out = np.cross(e, n); out /= np.linalg.norm(out)
    if np.dot(out, T[2] - T[0]) > 0:
        out = -out
    base = T[0] + 0.5 * e + 5e-4 * n
    xa = np.vstack([base - 1e-10 * out, T]); xb = np.vstack([base + 1e-10 * out, T])
    assert orc.pt_region(xa) == 6 and orc.pt_region(xb) == 3
    sa, sb = orc.barrier_element(xa, DHAT, KAPPA), orc.barrier_element(xb, DHAT, KAPPA)
    assert sa[1] == pytest.approx(sb[1], rel=1e-6)
    assert np.linalg.norm(sa[2] - sb[2]) <= 1e-5 * np.linalg.norm(sa[2])


def test_barrier_inactive_and_invalid():
    T = _tri(0)
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    far = np.vstack([T.mean(0) + 2e-3 * n, T])
    st, E, g, H = orc.barrier_element(far, DHAT, KAPPA)
    assert st == 0 and E == 0 and not g.any() and not H.any()
    touching = np.vstack([T[1], T])  # on a vertex: distance exactly 0
    st, *_ = orc.barrier_element(touching, DHAT, KAPPA)
    assert st == -1


def test_barrier_rigid_invariance():
    T = _tri(0)
    n = np.cross(T[1] - T[0], T[2] - T[0]); n /= np.linalg.norm(n)
    xe = np.vstack([T.mean(0) + 2e-4 * T[1] / np.linalg.norm(T[1]) + 3e-4 * n, T])
    st, E, g, H = orc.barrier_element(xe, DHAT, KAPPA)
    q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    st2, E2, g2, H2 = orc.barrier_element(xe @ q.T + 0.01, DHAT, KAPPA)
    RR = np.kron(np.eye(4), q)
    assert E2 == pytest.approx(E, rel=1e-10)
    assert np.linalg.norm(g2 - RR @ g) <= 1e-9 * np.linalg.norm(g)
    assert np.linalg.norm(H2 - RR @ H @ RR.T) <= 1e-8 * np.linalg.norm(H)


def test_generator_pairs_distance():
    sh = scenes.shell_sheet(8, length=0.1, noise=0.05, seed=3)
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], 50, 1e-4, 1e-3, seed=3,
                              tri_node_offset=0, point_node_offset=sh["x"].shape[0])
    allx = np.vstack([sh["x"], bp["points"]])
    for k in range(50):
        xe = allx[bp["pairs"][k]]
        assert orc.pt_region(xe) == 6
        assert orc.pt_distance(xe) == pytest.approx(bp["d"][k], rel=1e-9)
