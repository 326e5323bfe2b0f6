"""Lagged IPC friction (§6.4 friction potential) through the C ABI against
the FP64 oracle: the lag (closest-point weights, contact force, separation,
tangent plane), element E/g/H in the stick and slide regimes, assembly,
Newton steps, and the Coulomb impulse of a sliding point in closed form.

The GPU and the oracle choose different tangent bases T; the potential
depends only on T^T T (pinned in the oracle), which is what is compared.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

MU, YH, DT, DHAT, KAPPA = 0.3, 1e-3, 0.01, 1e-3, 1e4


@pytest.fixture(scope="module")
def ctx():
    pytest.importorskip("torch")
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02156_gb300.scene import Context
    c = Context(0)
    yield c
    c.close()


def _sheet_points(n_pairs=700, seed=3, dmax=1.6e-3):
    """A 12 x 12 sheet with points over random triangles at d ~ U(1e-4, dmax)
    (some beyond dhat: no contact force)."""
    sh = scenes.shell_sheet(12, length=0.1, z0=0.0, noise=0.05, seed=seed)
    ns = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], n_pairs, 1e-4, dmax, seed=seed,
                              tri_node_offset=0, point_node_offset=ns)
    X = np.vstack([sh["X"], bp["points"]])
    x = np.vstack([sh["x"], bp["points"]])
    return sh, bp, X, x, ns


def _slid(x, ns, seed, amp):
    """Points moved by random tangential-ish offsets of size ~amp (the sheet
    stays): slides from deep stick to well beyond the threshold."""
    rng = np.random.default_rng(seed)
    y = x.copy()
    P = x.shape[0] - ns
    scale = amp * np.exp(rng.uniform(np.log(1e-3), np.log(30.0), P))
    d = rng.normal(size=(P, 3)); d[:, 2] *= 0.1
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y[ns:] += scale[:, None] * d
    return y


def _gpu_scene(ctx, X, x, pairs, with_barrier=False, pinned=None, mass=None):
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, X)
    if with_barrier:
        s.add_barrier(pairs, DHAT, KAPPA)
    eid = s.add_friction(pairs, MU, YH, DHAT, KAPPA)
    if mass is not None:
        s.add_node_mass(mass)
    if pinned is not None:
        s.set_pinned(pinned)
    s.finalize()
    s.set_state(x=x)
    return s, eid


@pytest.mark.gpu
def test_friction_lag_parity(ctx):
    sh, bp, X, x, ns = _sheet_points()
    s, eid = _gpu_scene(ctx, X, x, bp["pairs"])
    lag0 = s.friction_lag(eid)
    assert not lag0["fn"].any()          # no friction before the first lag
    s.update_friction(DT)
    g = s.friction_lag(eid)
    o = orc.friction_lag(x, bp["pairs"], DHAT, KAPPA)
    assert np.abs(g["beta"] - o["beta"]).max() <= 1e-12
    assert np.allclose(g["fn"], o["fn"], rtol=1e-12, atol=0)
    assert (o["fn"] == 0).any() and (o["fn"] > 0).any()
    d = np.linalg.norm(o["dxt"], axis=1)
    assert (np.linalg.norm(g["dxt"] - o["dxt"], axis=1) <= 1e-12 * d + 1e-18).all()
    # the same tangent plane: T^T T equal
    Pg = np.einsum("pri,prj->pij", g["T"], g["T"])
    Po = np.einsum("pri,prj->pij", o["T"], o["T"])
    assert np.abs(Pg - Po).max() <= 1e-9
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_friction_elements_parity(ctx, precision):
    sh, bp, X, x0, ns = _sheet_points(seed=4)
    s, eid = _gpu_scene(ctx, X, x0, bp["pairs"])
    s.update_friction(DT)
    x = _slid(x0, ns, 5, YH * DT)
    s.set_state(x=x)
    out = s.eval_elements(eid, project=True, precision=precision)
    lag = orc.friction_lag(x0, bp["pairs"], DHAT, KAPPA)
    Ee, ge, He = orc.friction_batch(x, bp["pairs"], lag, MU, YH, DT)
    tol = 1e-10 if precision == sx.SX_FP64 else 1e-4
    k = MU * lag["fn"]
    worst = [0.0, 0.0, 0.0]
    for e in range(Ee.size):
        if k[e] == 0:
            assert out["E"][e] == 0 and not out["g"][e].any() and not out["H"][e].any()
            continue
        sE, sg, sH = k[e] * YH * DT, k[e], k[e] / (YH * DT)
        worst[0] = max(worst[0], abs(out["E"][e] - Ee[e]) / max(abs(Ee[e]), sE))
        worst[1] = max(worst[1], np.linalg.norm(out["g"][e] - ge[e]) /
                       max(np.linalg.norm(ge[e]), sg))
        worst[2] = max(worst[2], np.linalg.norm(out["H"][e] - He[e]) /
                       max(np.linalg.norm(He[e]), 1e-6 * sH))
    assert max(worst) <= tol, worst
    # PSD without projection (none is queued for friction)
    w = np.linalg.eigvalsh(out["H"])
    assert w.min() >= -(1e-9 if precision == sx.SX_FP64 else 1e-6) * np.abs(w).max()
    s.close()


@pytest.mark.gpu
def test_friction_assembly_and_newton_match_oracle(ctx):
    """Barrier + friction over a pinned sheet; points with tangential
    velocities (some stick, some slide) and gravity: assembled E/g/H after a
    lag, and one backward-Euler step."""
    sh, bp, X, x, ns = _sheet_points(n_pairs=300, seed=6, dmax=9e-4)
    N = X.shape[0]
    P = N - ns
    mass = np.concatenate([np.zeros(ns), np.full(P, 1e-3)])
    pinned = np.arange(ns)
    s, eid = _gpu_scene(ctx, X, x, bp["pairs"], with_barrier=True, pinned=pinned, mass=mass)
    s.update_friction(DT)
    y = _slid(x, ns, 8, YH * DT)
    s.set_state(x=y)
    Eg = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, vals = s.bsr()
    sc = orc.Scene(N, mass=mass, pt={"pairs": bp["pairs"], "dhat": DHAT, "kappa": KAPPA},
                   fr={"pairs": bp["pairs"], "mu": MU, "yhat": YH, "dhat": DHAT,
                       "kappa": KAPPA}, pinned=pinned)
    sc.friction_lag(x)
    Eo, go, vo, bad = sc.eval(y, dt=DT, level=2, project=True)
    assert bad == 0
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    assert abs(Eg - Eo) <= 1e-10 * abs(Eo)
    assert np.linalg.norm(vals - vo) <= 1e-10 * np.linalg.norm(vo)
    assert np.linalg.norm(s.grad() - go) <= 1e-10 * np.linalg.norm(go)
    # one Newton step from x with tangential velocities
    rng = np.random.default_rng(9)
    v = np.zeros_like(x)
    v[ns:, :2] = rng.normal(size=(P, 2)) * np.exp(rng.uniform(np.log(1e-4), np.log(0.5), P))[:, None]
    s.set_gravity((0.0, 0.0, -9.81))
    s.set_state(x=x, v=v)
    rc, r = s.newton_step(DT, newton_tol=1e-8, pcg_tol=1e-12)
    assert rc == sx.SX_OK, r
    xg, vg = s.get_state()
    xo, vo_, st, rep = sc.newton_step(x, v, DT, newton_tol=1e-8, pcg_tol=1e-12)
    assert st == 0, rep
    ref = np.abs(xo - x).max()
    assert np.abs(xg - xo).max() <= 1e-8 * ref + 1e-14
    s.close()


@pytest.mark.gpu
def test_coulomb_impulse_of_a_sliding_point(ctx):
    """One free point (m = 1 kg) sliding at 0.5 m/s over a pinned triangle,
    barrier + friction, no gravity: its tangential speed drops by exactly
    mu fn dt / m (the barrier force is normal in the face region)."""
    a = np.array([0.0, 0.0, 0.0]); b = np.array([1.0, 0.1, 0.0]); c = np.array([0.2, 1.0, 0.05])
    n = np.cross(b - a, c - a); n /= np.linalg.norm(n)
    p = 0.3 * a + 0.3 * b + 0.4 * c + 5e-4 * n
    X = np.array([p, a, b, c])
    t = np.cross(n, b - a); t /= np.linalg.norm(t)
    pairs = np.array([[0, 1, 2, 3]], np.int32)
    s, eid = _gpu_scene(ctx, X, X, pairs, with_barrier=True, pinned=[1, 2, 3],
                        mass=np.array([1.0, 1.0, 1.0, 1.0]))
    v = np.zeros((4, 3)); v[0] = 0.5 * t
    s.set_state(x=X, v=v)
    rc, r = s.newton_step(DT, newton_tol=1e-10, pcg_tol=1e-14)
    assert rc == sx.SX_OK, r
    fn = s.friction_lag(eid)["fn"][0]
    assert fn > 0
    v1 = s.get_state()[1][0]
    assert v1 @ t == pytest.approx(0.5 - MU * fn * DT / 1.0, rel=1e-8)
    assert abs(v1 @ np.cross(n, t)) <= 1e-10
    s.close()


@pytest.mark.gpu
def test_friction_pairs_can_be_replaced(ctx):
    sh, bp, X, x, ns = _sheet_points(n_pairs=50, seed=11)
    s, eid = _gpu_scene(ctx, X, x, bp["pairs"])
    s.update_friction(DT)
    s.set_pairs(eid, bp["pairs"][::2].copy())
    lag = s.friction_lag(eid)
    assert lag["fn"].shape == (25,) and not lag["fn"].any()   # reset until the next lag
    s.update_friction(DT)
    o = orc.friction_lag(x, bp["pairs"][::2], DHAT, KAPPA)
    assert np.allclose(s.friction_lag(eid)["fn"], o["fn"], rtol=1e-12, atol=0)
    s.close()


@pytest.mark.gpu
def test_friction_lag_and_elements_in_edge_and_vertex_regions(ctx):
    """Points moved beyond triangle edges and vertices (the closest point on
    an edge or at a vertex) and a few beyond dhat: the lag and the element
    values against the oracle's Voronoi-region classification."""
    from test_gpu_parity import _barrier_scene
    X, x, pairs = _barrier_scene(n_pairs=300, seed=7, regions=True)
    ns = X.shape[0] - pairs.shape[0]
    s, eid = _gpu_scene(ctx, X, x, pairs)
    s.update_friction(DT)
    g = s.friction_lag(eid)
    o = orc.friction_lag(x, pairs, DHAT, KAPPA)
    # the three region kinds are present
    nz = (o["beta"] > 1e-12).sum(1)
    assert (nz == 1).any() and (nz == 2).any() and (nz == 3).any()
    assert np.abs(g["beta"] - o["beta"]).max() <= 1e-12
    assert np.allclose(g["fn"], o["fn"], rtol=1e-12, atol=0)
    d = np.linalg.norm(o["dxt"], axis=1)
    assert (np.linalg.norm(g["dxt"] - o["dxt"], axis=1) <= 1e-12 * d + 1e-18).all()
    Pg = np.einsum("pri,prj->pij", g["T"], g["T"])
    Po = np.einsum("pri,prj->pij", o["T"], o["T"])
    assert np.abs(Pg - Po).max() <= 1e-9
    y = _slid(x, ns, 12, YH * DT)
    s.set_state(x=y)
    out = s.eval_elements(eid, project=False, precision=sx.SX_FP64)
    Ee, ge, He = orc.friction_batch(y, pairs, o, MU, YH, DT)
    k = MU * o["fn"]
    for e in np.flatnonzero(k > 0):
        sE, sg, sH = k[e] * YH * DT, k[e], k[e] / (YH * DT)
        assert abs(out["E"][e] - Ee[e]) <= 1e-10 * max(abs(Ee[e]), sE)
        assert np.linalg.norm(out["g"][e] - ge[e]) <= 1e-10 * max(np.linalg.norm(ge[e]), sg)
        assert np.linalg.norm(out["H"][e] - He[e]) <= 1e-10 * max(np.linalg.norm(He[e]), 1e-6 * sH)
    s.close()
