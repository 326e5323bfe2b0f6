"""Pins of the oracle's BSR pattern, slot maps and assembly (§5.3, Eq. 11,
Algorithm 1), inertia (§3, Eq. 2), block-Jacobi PCG (§7.2) and the
backward-Euler Newton step (§3, Eqs. 2-3)."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes


def kuhn_edges(nx, ny, nz):
    """Closed-form edge count of the Kuhn grid: directions e1, e2, e3,
    e1+e2, e1+e3, e2+e3, e1+e2+e3."""
    n = np.array([nx, ny, nz])
    tot = 0
    for d in [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]:
        tot += int(np.prod(n + 1 - np.array(d)))
    return tot


@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 5, 2), (1, 1, 1)])
def test_pattern_block_count_closed_form(dims):
    m = scenes.kuhn_box(*dims, h=0.1, seed=1)
    N = m["X"].shape[0]
    rp, col = orc.bsr_pattern(N, m["tets"])
    assert col.size == N + 2 * kuhn_edges(*dims)
    if dims == (4, 4, 4):
        assert col.size == 1333
    for r in range(N):
        row = col[rp[r]:rp[r + 1]]
        assert np.all(np.diff(row) > 0) and r in row


def test_pattern_block_count_64_cube():
    assert 65 ** 3 + 2 * kuhn_edges(64, 64, 64) == 4_018_753


def _dense_from_bsr(rp, col, vals, N):
    D = np.zeros((3 * N, 3 * N))
    for r in range(N):
        for k in range(rp[r], rp[r + 1]):
            D[3 * r:3 * r + 3, 3 * col[k]:3 * col[k] + 3] = vals[k]
    return D


def _snh_scene(m, young=1e5, nu=0.3, rho=1000.0, hinge=None, pt=None, N=None):
    E, nuv = scenes.material_uniform(m["tets"].shape[0], young, nu)
    snh, mass, bad = orc.snh_scene_inputs(m["X"], m["tets"], E, nuv, rho)
    assert bad == 0
    N = N or m["X"].shape[0]
    if mass.size < N:
        mass = np.concatenate([mass, np.full(N - mass.size, 1e-3)])
    return orc.Scene(N, mass=mass, snh=snh, hinge=hinge, pt=pt, pinned=m["pinned"]), snh


def test_two_tet_brute_force_dense_assembly():
    m = scenes.two_tet()
    sc, snh = _snh_scene(m)
    N = 5
    assert sc.nnzb == 23  # all pairs but (0,4) and (4,0)
    x = m["X"] + np.random.default_rng(0).uniform(-0.2, 0.2, m["X"].shape)
    E, grad, vals, _ = sc.eval(x, level=2, project=True)
    Ee, ge, He = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"],
                               snh["lam"], 2, True)
    Hd = np.zeros((15, 15)); gd = np.zeros(15)
    for e, t in enumerate(m["tets"]):
        R = np.zeros((12, 15))
        for a in range(4):
            R[3 * a:3 * a + 3, 3 * t[a]:3 * t[a] + 3] = np.eye(3)
        Hd += R.T @ He[e] @ R
        gd += R.T @ ge[e]
    assert E == pytest.approx(Ee.sum(), rel=1e-15)
    assert np.allclose(grad, gd, rtol=0, atol=1e-12 * np.abs(gd).max())
    assert np.allclose(_dense_from_bsr(sc.row_ptr, sc.col, vals, N), Hd, rtol=0,
                       atol=1e-12 * np.abs(Hd).max())


def test_c1_dense_assembly_symmetry_and_zero_net_force():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    sc, snh = _snh_scene(m)
    N = m["X"].shape[0]
    x = scenes.jitter_state(m["X"], 0.02, seed=7)
    E, grad, vals, _ = sc.eval(x, level=2, project=True)
    Ee, ge, He = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"],
                               snh["lam"], 2, True)
    Hd = np.zeros((3 * N, 3 * N))
    for e, t in enumerate(m["tets"]):
        idx = (3 * t[:, None] + np.arange(3)).ravel()
        Hd[np.ix_(idx, idx)] += He[e]
    D = _dense_from_bsr(sc.row_ptr, sc.col, vals, N)
    assert np.allclose(D, Hd, rtol=0, atol=1e-11 * np.abs(Hd).max())
    assert np.allclose(D, D.T, rtol=0, atol=1e-12 * np.abs(D).max())
    assert np.linalg.eigvalsh(D).min() >= -1e-9 * np.abs(D).max()
    # net elastic force vanishes (translation invariance of every element)
    assert np.linalg.norm(grad.reshape(-1, 3).sum(0)) <= 1e-10 * np.linalg.norm(grad)
    # slot maps point at the right (row, col)
    for e in range(0, 384, 37):
        t = m["tets"][e]
        for a in range(4):
            for b in range(4):
                s = sc.slots[e, 4 * a + b]
                assert sc.row_ptr[t[a]] <= s < sc.row_ptr[t[a] + 1]
                assert sc.col[s] == t[b]


def test_inertia_closed_form():
    rng = np.random.default_rng(0)
    m = rng.uniform(0.1, 1, 10); x = rng.normal(size=(10, 3)); xt = rng.normal(size=(10, 3))
    grad = np.zeros(30)
    E = orc.inertia(m, 0.01, x, xt, grad=grad)
    assert E == pytest.approx(np.sum(m[:, None] * (x - xt) ** 2) / (2 * 1e-4), rel=1e-14)
    assert np.allclose(grad, (m[:, None] * (x - xt) / 1e-4).ravel(), rtol=1e-14)


def test_pcg_matches_library_solve_c1():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    sc, snh = _snh_scene(m)
    N = m["X"].shape[0]
    x = scenes.jitter_state(m["X"], 0.02, seed=3, fixed=m["pinned"])
    xt = m["X"] + np.array([0, 0, -9.81e-4])
    E, g, vals, _ = sc.eval(x, xt=xt, dt=0.01, level=2, project=True)
    pm = sc.pinned_mask
    b = np.where(np.repeat(pm, 3) == 1, 0.0, -g)
    dx, st, it, rr = orc.pcg(sc.row_ptr, sc.col, vals, sc.diag_slot, pm, b, 1e-13)
    assert st == 0 and rr <= 1e-13
    D = _dense_from_bsr(sc.row_ptr, sc.col, vals, N)
    free = np.repeat(pm == 0, 3)
    ref = np.zeros(3 * N)
    ref[free] = np.linalg.solve(D[np.ix_(free, free)], b[free])
    assert np.linalg.norm(dx - ref) <= 1e-10 * np.linalg.norm(ref)
    assert not dx[~free].any()


def test_newton_free_fall_is_exact():
    # zero stiffness and no pins: E_BE is the inertia alone, so one Newton
    # step lands on xtilde = x + dt v + dt^2 g (Eq. 2)
    m = scenes.kuhn_box(2, 2, 2, h=0.5, seed=2)
    T = m["tets"].shape[0]
    Dminv, V, _ = orc.tet_rest(m["X"], m["tets"])
    snh = {"tets": m["tets"], "Dminv": Dminv, "V": V, "mu": np.zeros(T), "lam": np.zeros(T)}
    mass = orc.lumped_mass(m["X"].shape[0], m["tets"], V, 1000.0)
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh)
    v0 = np.random.default_rng(0).normal(size=m["X"].shape)
    dt, g = 0.01, np.array([0.0, 0.0, -9.81])
    x, v, st, rep = sc.newton_step(m["X"], v0, dt, gravity=g)
    xt = m["X"] + dt * v0 + dt * dt * g
    assert st == 0 and rep["newton_iters"] == 1
    assert np.allclose(x, xt, rtol=0, atol=1e-14)
    assert np.allclose(v, (xt - m["X"]) / dt, rtol=0, atol=1e-10)


def test_newton_c1_converges_monotone_and_keeps_pins():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    sc, snh = _snh_scene(m)
    X = m["X"]; v0 = np.zeros_like(X); dt = 0.01; g = np.array([0, 0, -9.81])
    x, v, st, rep = sc.newton_step(X, v0, dt, gravity=g)
    assert st == 0 and rep["newton_iters"] >= 1
    xt = X + dt * v0 + dt * dt * g
    E, grad, _, _ = sc.eval(x, xt=xt, dt=dt, level=1)
    free = np.repeat(sc.pinned_mask == 0, 3)
    assert np.linalg.norm(grad[free]) <= 1e-8 * rep["g0_norm"] * 1.0000001
    assert np.array_equal(x[m["pinned"]], X[m["pinned"]])
    energies = []
    for k in range(0, rep["newton_iters"] + 1):
        xk, *_ = sc.newton_step(X, v0, dt, gravity=g, max_newton=k)
        energies.append(sc.eval(xk, xt=xt, dt=dt, level=0)[0])
    assert all(b <= a for a, b in zip(energies, energies[1:]))
    # the cube sags: free nodes move down on average
    assert (x[:, 2] - X[:, 2])[sc.pinned_mask == 0].mean() < 0


def test_newton_forcing_sequence_solves_inexactly_and_converges():
    # forcing option (§7.2 solver paragraph, as read: PCG tolerance
    # max(pcg_tol, min(1/2, sqrt(|g_k|/|g_0|)))): the first Newton direction
    # is an inexact solve (relative residual of the dense system at x0 at most
    # 1/2, far above the fixed 1e-10), and the step still ends at a point whose
    # free gradient meets the Newton tolerance, with fewer PCG iterations.
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    sc, snh = _snh_scene(m, young=3e5)
    X = m["X"]; N = X.shape[0]; dt = 0.01; g = np.array([0, 0, -9.81])
    v0 = np.zeros_like(X); v0[:, 0] = 0.5; v0[m["pinned"]] = 0.0
    xt = X + dt * v0 + dt * dt * g
    free = np.repeat(sc.pinned_mask == 0, 3)
    E0, g0, vals0, _ = sc.eval(X, xt=xt, dt=dt, level=2, project=True)
    H0 = _dense_from_bsr(sc.row_ptr, sc.col, vals0.reshape(-1, 3, 3), N)
    Hf = H0[np.ix_(free, free)]
    x1, *_ = sc.newton_step(X, v0, dt, gravity=g, max_newton=1, forcing=True)
    d = (x1 - X).ravel()[free]
    rel = np.linalg.norm(Hf @ d + g0[free]) / np.linalg.norm(g0[free])
    assert 1e-6 < rel <= 0.5 * (1 + 1e-9)
    xf, vf, st, rf = sc.newton_step(X, v0, dt, gravity=g, forcing=True)
    xe, ve, st2, re_ = sc.newton_step(X, v0, dt, gravity=g)
    assert st == 0 and st2 == 0
    _, gf, _, _ = sc.eval(xf, xt=xt, dt=dt, level=1)
    assert np.linalg.norm(gf[free]) <= 1e-8 * rf["g0_norm"] * (1 + 1e-7)
    assert rf["pcg_iters_total"] < re_["pcg_iters_total"]
    # both end within the Newton tolerance of the same solution
    assert np.abs(xf - xe).max() <= 1e-6 * np.abs(xe - X).max()
