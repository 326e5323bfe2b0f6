"""CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (normwise, per element, with the element scale s = V mu' for
SNH): FP64 1e-10, FP32 1e-4; pattern, slot maps and diagonal slots
bit-identical. Sizes span several 128-element tiles and a ragged tail.
"""
import re
import os

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL64, TOL32 = 1e-10, 1e-4


def test_library_exports_every_declared_symbol():
    import ctypes
    hdr = open(os.path.join(ROOT, "include", "sx.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|const char\*)\s+(sx_\w+)\s*\(", hdr, re.M))
    assert names == set(sx.EXPORTS)
    L = sx.load()
    for n in names:
        assert hasattr(L, n), n
    assert b"sm_103a" in L.sx_version()


def _relerr(a, b, scale):
    a = np.asarray(a, float); b = np.asarray(b, float)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), scale)


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


def _snh_case(dims=(5, 4, 3), seed=11, jitter=0.04, random_mat=True):
    m = scenes.kuhn_box(*dims, h=0.25, seed=seed)
    T = m["tets"].shape[0]
    if random_mat:
        E, nu = scenes.material_random(T, seed=seed)
    else:
        E, nu = scenes.material_uniform(T, 1e5, 0.3)
    x = scenes.jitter_state(m["X"], jitter * 0.25, seed=seed + 1)
    snh, mass, bad = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    assert bad == 0
    return m, E, nu, x, snh, mass


def _gpu_snh_scene(ctx, m, E, nu, x, finalize=True):
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, m["X"])
    eid = s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    if finalize:
        s.finalize()
    s.set_state(x=x)
    return s, eid


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
@pytest.mark.parametrize("project", [False, True])
def test_snh_elements_parity(ctx, precision, project):
    m, E, nu, x, snh, mass = _snh_case()
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    out = s.eval_elements(eid, project=project, precision=precision)
    Ee, ge, He = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"], snh["lam"],
                               2, project)
    tol = TOL64 if precision == sx.SX_FP64 else TOL32
    scale = snh["V"] * snh["mu"]
    worst = [0.0, 0.0, 0.0]
    for e in range(Ee.size):
        worst[0] = max(worst[0], abs(out["E"][e] - Ee[e]) / max(abs(Ee[e]), scale[e]))
        worst[1] = max(worst[1], _relerr(out["g"][e], ge[e], scale[e]))
        worst[2] = max(worst[2], _relerr(out["H"][e], He[e], scale[e]))
    assert max(worst) <= tol, worst
    if project:
        # every projected Hessian is PSD and the state has indefinite elements
        w = np.linalg.eigvalsh(out["H"])
        psd_tol = 1e-9 if precision == sx.SX_FP64 else 1e-6   # storage rounding
        assert w.min() >= -psd_tol * np.abs(w).max()
    s.close()


@pytest.mark.gpu
def test_pattern_slots_and_assembly_parity(ctx):
    m, E, nu, x, snh, mass = _snh_case(dims=(6, 5, 4), seed=3)
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    N = m["X"].shape[0]
    sc = orc.Scene(N, mass=mass, snh=snh, pinned=m["pinned"])
    # index maps are bit-identical
    out = s.eval_elements(eid, project=True, want_H=False, want_g=False)
    assert np.array_equal(out["slots"], sc.slots)
    xt = m["X"] + np.array([0.0, 0.0, -9.81 * 1e-4])
    for precision, tol in [(sx.SX_FP64, TOL64), (sx.SX_FP32, TOL32)]:
        s.set_inertia(0.01, xt)
        Eg = s.eval(sx.SX_EGH, True, precision)
        rp, col, vals = s.bsr()
        Eo, go, vo, _ = sc.eval(x, xt=xt, dt=0.01, level=2, project=True)
        assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
        assert abs(Eg - Eo) <= tol * max(abs(Eo), 1e-30)
        assert _relerr(s.grad(), go, 1e-30) <= tol
        assert _relerr(vals, vo, 1e-30) <= tol
        # per block row
        for r in range(0, N, 7):
            a, b = rp[r], rp[r + 1]
            assert _relerr(vals[a:b], vo[a:b], 1e-30) <= 10 * tol
    s.close()


@pytest.mark.gpu
def test_assembly_is_deterministic(ctx):
    m, E, nu, x, snh, mass = _snh_case(dims=(8, 8, 8), seed=5)
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    s.eval(sx.SX_EGH, True, sx.SX_FP64)
    a = s.bsr()[2].copy(); ga = s.grad()
    s.eval(sx.SX_EGH, True, sx.SX_FP64)
    b = s.bsr()[2]; gb = s.grad()
    assert np.array_equal(a, b) and np.array_equal(ga, gb)
    s.close()


@pytest.mark.gpu
def test_hinge_parity(ctx):
    from paper_2303_02156_gb300.scene import Scene
    sh = scenes.shell_sheet(13, length=0.5, noise=0.1, seed=4)
    n = sh["hinges"].shape[0]
    s = Scene(ctx, sh["X"])
    eid = s.add_hinge(sh["hinges"], sh["q"], sh["c"], 1e-3)
    s.finalize()
    s.set_state(x=sh["x"])
    Eo, go, Ho = orc.hinge_batch(sh["x"], sh["hinges"], sh["q"], sh["c"], 1e-3, 2)
    for precision, tol in [(sx.SX_FP64, TOL64), (sx.SX_FP32, TOL32)]:
        out = s.eval_elements(eid, project=True, precision=precision)
        for e in range(n):
            sc = 1e-3 * sh["c"][e] * np.sum(sh["q"][e] ** 2) * sh["h"] ** 2
            assert abs(out["E"][e] - Eo[e]) <= tol * max(abs(Eo[e]), sc)
            assert _relerr(out["g"][e], go[e], sc / sh["h"]) <= tol
            assert _relerr(out["H"][e], Ho[e], sc / sh["h"] ** 2) <= tol
    s.close()


def _barrier_scene(n_pairs=300, seed=7, regions=False):
    sh = scenes.shell_sheet(10, length=0.01, noise=0.05, seed=seed)
    nv = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], n_pairs, 1e-4, 1e-3, seed=seed,
                              tri_node_offset=0, point_node_offset=nv)
    pts = bp["points"].copy()
    if regions:
        # move a subset well into edge and vertex regions (away from region
        # boundaries), keeping d in (1e-4, 1e-3) for most of them
        rng = np.random.default_rng(seed)
        for k in range(0, n_pairs, 3):
            t = sh["tris"][bp["tri"][k]]
            A, B, Cc = sh["x"][t]
            nrm = np.cross(B - A, Cc - A); nrm /= np.linalg.norm(nrm)
            if k % 2 == 0:   # beyond vertex A, away from the centroid
                out = A - (A + B + Cc) / 3; out /= np.linalg.norm(out)
                pts[k] = A + rng.uniform(2e-4, 5e-4) * out + rng.uniform(1e-4, 5e-4) * nrm
            else:            # beyond edge AB
                e = B - A; mid = A + rng.uniform(0.3, 0.7) * e
                o = np.cross(e, nrm); o /= np.linalg.norm(o)
                if np.dot(o, Cc - mid) > 0:
                    o = -o
                pts[k] = mid + rng.uniform(2e-4, 5e-4) * o + rng.uniform(1e-4, 5e-4) * nrm
        # a few inactive pairs
        pts[1::17] += 3e-3 * np.array([0, 0, 1.0])
    X = np.vstack([sh["X"], pts])
    x = np.vstack([sh["x"], pts])
    return X, x, bp["pairs"]


@pytest.mark.gpu
@pytest.mark.parametrize("regions", [False, True])
def test_barrier_parity(ctx, regions):
    from paper_2303_02156_gb300.scene import Scene
    X, x, pairs = _barrier_scene(regions=regions)
    s = Scene(ctx, X)
    eid = s.add_barrier(pairs, 1e-3, 1e4)
    s.finalize()
    s.set_state(x=x)
    Eo, go, Ho, act, bad = orc.barrier_batch(x, pairs, 1e-3, 1e4, 2, False)
    _, _, Hp, _, _ = orc.barrier_batch(x, pairs, 1e-3, 1e4, 2, True)
    assert bad == 0 and (act == 1).sum() > 0
    if regions:
        assert (act == 0).sum() > 0
    # element scale of the barrier: kappa dhat^2 (energy), kappa dhat
    # (gradient), kappa (Hessian); b and its derivatives vanish at d = dhat
    sE, sg, sH = 1e4 * 1e-6, 1e4 * 1e-3, 1e4
    for precision, tol in [(sx.SX_FP64, TOL64), (sx.SX_FP32, TOL32)]:
        for project, Href in [(False, Ho), (True, Hp)]:
            out = s.eval_elements(eid, project=project, precision=precision)
            for e in range(pairs.shape[0]):
                if act[e] != 1:
                    assert out["E"][e] == 0 and not out["g"][e].any() and not out["H"][e].any()
                    continue
                ctx_ = (precision, project, e)
                assert abs(out["E"][e] - Eo[e]) <= tol * max(abs(Eo[e]), sE), ctx_
                assert _relerr(out["g"][e], go[e], sg) <= tol, ctx_
                assert _relerr(out["H"][e], Href[e], sH) <= tol, (ctx_, _relerr(out["H"][e], Href[e], sH))
    s.close()


@pytest.mark.gpu
def test_barrier_invalid_state_reported(ctx):
    from paper_2303_02156_gb300.scene import Scene
    X, x, pairs = _barrier_scene(n_pairs=20)
    x = x.copy()
    # put point of pair 0 exactly on a vertex of its triangle
    x[pairs[0, 0]] = x[pairs[0, 1]]
    s = Scene(ctx, X)
    s.add_barrier(pairs, 1e-3, 1e4)
    s.finalize()
    s.set_state(x=x)
    rc, _ = s.eval(sx.SX_E, False, sx.SX_FP64, check=False)
    assert rc == sx.SX_ESTATE
    assert s.stats()["bad_state"] == 1
    s.close()


@pytest.mark.gpu
def test_mixed_blocks_pattern_and_assembly(ctx):
    """SNH block + hinge sheet + barrier pairs as stacked DOF sets (§5.3)."""
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(3, 3, 2, h=0.01, seed=2)
    nt = m["X"].shape[0]
    sh = scenes.shell_sheet(6, length=0.03, z0=0.03, noise=0.05, seed=2, node_offset=nt)
    ns = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"] - nt, 40, 1e-4, 1e-3, seed=2,
                              tri_node_offset=nt, point_node_offset=nt + ns)
    X = np.vstack([m["X"], sh["X"], bp["points"]])
    x = np.vstack([scenes.jitter_state(m["X"], 2e-4, 9), sh["x"], bp["points"]])
    N = X.shape[0]
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, 2)
    s = Scene(ctx, X)
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.add_hinge(sh["hinges"], sh["q"], sh["c"], 1e-3)
    s.add_barrier(bp["pairs"], 1e-3, 1e4)
    extra = np.zeros(N); extra[nt:] = 1e-3
    s.add_node_mass(extra)
    s.finalize()
    s.set_state(x=x)
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    mass_all = np.concatenate([mass, np.zeros(N - nt)]) + extra
    sc = orc.Scene(N, mass=mass_all, snh=snh,
                   hinge={"stencils": sh["hinges"], "q": sh["q"], "c": sh["c"], "kb": 1e-3},
                   pt={"pairs": bp["pairs"], "dhat": 1e-3, "kappa": 1e4})
    xt = x + 1e-5
    s.set_inertia(0.01, xt)
    Eg = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, vals = s.bsr()
    Eo, go, vo, bad = sc.eval(x, xt=xt, dt=0.01, level=2, project=True)
    assert bad == 0
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    assert abs(Eg - Eo) <= TOL64 * abs(Eo)
    assert _relerr(s.grad(), go, 0) <= TOL64
    assert _relerr(vals, vo, 0) <= TOL64
    s.close()


@pytest.mark.gpu
def test_empty_and_single_element_blocks(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.two_tet()
    s = Scene(ctx, m["X"])
    e0 = s.add_snh(m["tets"][:1], 1e5, 0.3, 1000.0)
    e1 = s.add_barrier(np.zeros((0, 4), np.int32), 1e-3, 1e4)
    s.finalize()
    x = m["X"] + 0.01 * np.arange(15).reshape(5, 3) / 15
    s.set_state(x=x)
    out = s.eval_elements(e0, project=True)
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"][:1], [1e5], [0.3])
    Eo, go, Ho = orc.snh_batch(x, m["tets"][:1], snh["Dminv"], snh["V"], snh["mu"],
                               snh["lam"], 2, True)
    assert _relerr(out["H"][0], Ho[0], 0) <= TOL64
    E = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    assert abs(E - Eo[0]) <= TOL64 * abs(Eo[0])
    s.close()


@pytest.mark.gpu
def test_degenerate_rest_tet_rejected(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.two_tet()
    s = Scene(ctx, m["X"])
    with pytest.raises(sx.SxError) as ei:
        s.add_snh(m["tets"][:, [0, 2, 1, 3]], 1e5, 0.3)
    assert ei.value.code == sx.SX_EDEGENERATE
    with pytest.raises(sx.SxError) as ei:
        s.add_snh(np.array([[0, 1, 2, 99]]), 1e5, 0.3)
    assert ei.value.code == sx.SX_EINVAL
    s.close()


def _c1():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    T = m["tets"].shape[0]
    E, nu = scenes.material_uniform(T, 1e5, 0.3)
    return m, E, nu


@pytest.mark.gpu
def test_newton_step_c1_matches_oracle(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m, E, nu = _c1()
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh, pinned=m["pinned"])
    g = (0.0, 0.0, -9.81)
    xo, vo, st, rep = sc.newton_step(m["X"], np.zeros_like(m["X"]), 0.01, gravity=g)
    assert st == 0
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.set_gravity(g)
    s.finalize()
    rc, r = s.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10)
    x, v = s.get_state()
    ref = np.abs(m["X"] - xo).max()
    assert np.abs(x - xo).max() <= 1e-8 * ref + 1e-12
    assert np.abs(v - vo).max() <= (1e-8 * ref + 1e-12) / 0.01
    assert r["newton_iters"] >= 1 and r["g_norm"] <= 1e-8 * r["g0_norm"]
    assert np.array_equal(x[m["pinned"]], m["X"][m["pinned"]])
    s.close()


@pytest.mark.gpu
def test_newton_free_fall_exact(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(2, 2, 2, h=0.5, seed=2)
    T = m["tets"].shape[0]
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], np.zeros(T), np.full(T, 0.3), 1000.0)
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    v0 = np.random.default_rng(0).normal(size=m["X"].shape)
    s.set_state(v=v0)
    rc, r = s.newton_step(0.01)
    x, v = s.get_state()
    xt = m["X"] + 0.01 * v0 + 1e-4 * np.array([0, 0, -9.81])
    assert r["newton_iters"] == 1
    assert np.abs(x - xt).max() <= 1e-14
    s.close()


@pytest.mark.gpu
def test_batched_eval_and_newton_equal_single(ctx):
    from paper_2303_02156_gb300.scene import Scene
    rng = scenes.rng_for(4)
    made = []
    for k in range(3):
        dims = scenes.random_box_dims(rng.uniform(50, 400), rng)
        m = scenes.kuhn_box(*dims, h=0.1, seed=20 + k)
        T = m["tets"].shape[0]
        E, nu = scenes.material_random(T, 30 + k)
        made.append((m, E, nu))

    def build():
        out = []
        for m, E, nu in made:
            s = Scene(ctx, m["X"])
            s.add_snh(m["tets"], E, nu, 1000.0)
            s.set_pinned(m["pinned"])
            s.set_gravity((0, 0, -9.81))
            s.finalize()
            out.append(s)
        return out

    single = build()
    reps1 = [s.newton_step(0.01)[1] for s in single]
    xs1 = [s.get_state()[0] for s in single]
    batch = build()
    rc, reps2 = ctx.newton_step_batch(batch, 0.01)
    for a, b, r1, r2 in zip(single, batch, reps1, reps2):
        assert np.array_equal(a.get_state()[0], b.get_state()[0])
        assert r1["newton_iters"] == r2["newton_iters"] and r1["pcg_iters"] == r2["pcg_iters"]
    Eb = ctx.eval_batch(batch)
    Es = np.array([s.eval() for s in batch])
    assert np.array_equal(Eb, Es)
    for s in single + batch:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_pcg_graph_replay_matches_plain_launches(ctx, precision):
    """The PCG chunk replayed from a captured CUDA graph computes exactly
    what the plain launches compute (same kernels, same order)."""
    from paper_2303_02156_gb300.scene import Scene
    out = {}
    sc = []
    for k, dims in enumerate([(6, 5, 4), (3, 3, 7), (9, 2, 2)]):
        m = scenes.kuhn_box(*dims, h=0.05, seed=30 + k)
        T = m["tets"].shape[0]
        E, nu = scenes.material_random(T, seed=30 + k)
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        sc.append((s, m))
    tol = 1e-8 if precision == sx.SX_FP64 else 1e-6
    for graphs in (0, 1):
        for s, m in sc:
            s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        for step in range(2):
            rc, reps = ctx.newton_step_batch([s for s, _ in sc], 0.01, precision=precision,
                                             newton_tol=tol, pcg_tol=1e-10 if tol == 1e-8 else 1e-6,
                                             graphs=graphs)
            assert rc == sx.SX_OK
        out[graphs] = [s.get_state() for s, _ in sc]
    for (xa, va), (xb, vb) in zip(out[0], out[1]):
        assert np.array_equal(xa, xb) and np.array_equal(va, vb)
    for s, _ in sc:
        s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_launch_shapes_are_bit_identical_and_autotune(ctx, precision):
    """Every projection block size and element grid computes the same bits;
    the autotuner picks one of them and leaves the result unchanged."""
    m, E, nu, x, snh, mass = _snh_case(dims=(9, 8, 7), seed=4)
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    ref = None
    for ct in (32, 64, 128, 256):
        for bps in (-1, 0, 1, 2):
            ctx.set_launch_shape(precision, ct, bps)
            s.eval(sx.SX_EGH, True, precision)
            out = (s.bsr()[2].copy(), s.grad())
            if ref is None:
                ref = out
            else:
                assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1]), (ct, bps)
    rep = ctx.autotune([s], precision)
    assert rep["clamp_threads"] in (32, 64, 128, 256) and rep["candidates"] >= 3
    assert 0 < rep["tuned_ms"] <= rep["default_ms"]
    s.eval(sx.SX_EGH, True, precision)
    assert np.array_equal(s.bsr()[2], ref[0]) and np.array_equal(s.grad(), ref[1])
    ctx.set_launch_shape(precision, 128, -1)   # back to the default
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_projection_parity_strongly_deformed(ctx, precision):
    """Large node jitter (some tets inverted, J < 0): many stencils with
    several negative eigenvalues go through the projection."""
    m, E, nu, x, snh, mass = _snh_case(dims=(6, 5, 4), seed=21, jitter=0.45)
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    out = s.eval_elements(eid, project=True, precision=precision)
    Ee, ge, He = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"], snh["lam"],
                               2, True)
    # the state has inverted tets and strongly indefinite Hessians
    F_dets = []
    for e in range(snh["tets"].shape[0]):
        Ds = (x[snh["tets"][e, 1:]] - x[snh["tets"][e, 0]]).T
        F_dets.append(np.linalg.det(Ds @ snh["Dminv"][e].reshape(3, 3)))
    assert min(F_dets) < 0
    tol = TOL64 if precision == sx.SX_FP64 else TOL32
    scale = snh["V"] * snh["mu"]
    worst = 0.0
    for e in range(Ee.size):
        worst = max(worst, _relerr(out["H"][e], He[e], scale[e]))
    assert worst <= tol, worst
    w = np.linalg.eigvalsh(out["H"])
    assert w.min() >= -(1e-9 if precision == sx.SX_FP64 else 1e-6) * np.abs(w).max()
    s.close()


def _mixed_small():
    m = scenes.kuhn_box(3, 3, 2, h=0.01, seed=2)
    nt = m["X"].shape[0]
    sh = scenes.shell_sheet(6, length=0.03, z0=0.03, noise=0.05, seed=2, node_offset=nt)
    ns = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"] - nt, 40, 2e-4, 8e-4, seed=2,
                              tri_node_offset=nt, point_node_offset=nt + ns)
    X = np.vstack([m["X"], sh["X"], bp["points"]])
    x0 = np.vstack([m["X"], sh["x"], bp["points"]])
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, 2)
    extra = np.zeros(X.shape[0])
    extra[nt:nt + ns] = 1e-4
    extra[nt + ns:] = 1e-3
    return m, sh, bp, X, x0, E, nu, extra, nt


@pytest.mark.gpu
def test_newton_step_mixed_stencils_matches_oracle(ctx):
    """One backward-Euler step of an SNH block + hinge sheet + barrier points
    (line search keeps every barrier distance positive) against the oracle."""
    from paper_2303_02156_gb300.scene import Scene
    m, sh, bp, X, x0, E, nu, extra, nt = _mixed_small()
    N = X.shape[0]
    s = Scene(ctx, X)
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.add_hinge(sh["hinges"], sh["q"], sh["c"], 1e-3)
    s.add_barrier(bp["pairs"], 1e-3, 1e4)
    s.add_node_mass(extra)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    s.set_state(x=x0, v=np.zeros_like(x0))
    rc, r = s.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10)
    assert rc == sx.SX_OK, r
    x, v = s.get_state()
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    mass_all = np.concatenate([mass, np.zeros(N - nt)]) + extra
    sc = orc.Scene(N, mass=mass_all, snh=snh,
                   hinge={"stencils": sh["hinges"], "q": sh["q"], "c": sh["c"], "kb": 1e-3},
                   pt={"pairs": bp["pairs"], "dhat": 1e-3, "kappa": 1e4}, pinned=m["pinned"])
    xo, vo, st, rep = sc.newton_step(x0, np.zeros_like(x0), 0.01)
    assert st == 0
    ref = np.abs(xo - x0).max()
    assert np.abs(x - xo).max() <= 1e-8 * ref + 1e-12
    s.close()


@pytest.mark.gpu
def test_newton_step_fp32_close_to_oracle(ctx):
    """The FP32 form of a C1 step (FP64 projection, residual norms and
    line-search energies) against the FP64 oracle: displacement error
    within 1e-5 of the displacement at Newton tolerance 1e-6."""
    from paper_2303_02156_gb300.scene import Scene
    m, E, nu = _c1()
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh, pinned=m["pinned"])
    xo, vo, st, rep = sc.newton_step(m["X"], np.zeros_like(m["X"]), 0.01)
    assert st == 0
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    rc, r = s.newton_step(0.01, newton_tol=1e-6, pcg_tol=1e-6, precision=sx.SX_FP32)
    assert rc == sx.SX_OK
    x, v = s.get_state()
    assert np.abs(x - xo).max() <= 1e-5 * np.abs(xo - m["X"]).max()
    s.close()


@pytest.mark.gpu
def test_all_pinned_scene_does_not_move(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(2, 2, 2, h=0.5, seed=4)
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], 1e5, 0.3, 1000.0)
    s.set_pinned(np.arange(m["X"].shape[0]))
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    rc, r = s.newton_step(0.01)
    assert rc == sx.SX_OK
    x, v = s.get_state()
    assert np.array_equal(x, m["X"]) and not v.any()
    s.close()


@pytest.mark.gpu
def test_api_misuse_returns_status_codes(ctx):
    import ctypes as C
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.two_tet()
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], 1e5, 0.3, 1000.0)
    # evaluation and stepping need a finalized scene
    rc, _ = s.eval(sx.SX_EGH, True, sx.SX_FP64, check=False)
    assert rc == sx.SX_EORDER
    rc, _ = s.newton_step(0.01, raise_on_error=False)
    assert rc == sx.SX_EORDER
    # node ids out of range, bad level, bad dt
    with pytest.raises(sx.SxError) as ei:
        s.add_barrier(np.array([[0, 1, 2, 7]]), 1e-3, 1e4)
        s.finalize()
    assert ei.value.code == sx.SX_EINVAL
    s.close()
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], 1e5, 0.3, 1000.0)
    s.finalize()
    assert sx.sx_eval(s.h, 7, 1, sx.SX_FP64, None, None) == sx.SX_EINVAL
    o = sx.newton_opts()
    assert sx.sx_newton_step(s.h, 0.0, C.byref(o), None, None) == sx.SX_EINVAL
    h = C.c_void_p()
    X = np.zeros((0, 3))
    assert sx.sx_scene_create(ctx.h, 0, X.ctypes.data, 3, None, C.byref(h)) == sx.SX_EINVAL
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
@pytest.mark.parametrize("jitter", [0.04, 0.45])
def test_material_projection_parity(ctx, precision, jitter):
    """project = 2: the SNH material Hessian clamped in the frame of the
    signed SVD of F (closed form on the GPU) against the oracle's numerical
    clamp of its explicit 9x9 d2psi/dF2."""
    m, E, nu, x, snh, mass = _snh_case(dims=(6, 5, 4), seed=31, jitter=jitter)
    s, eid = _gpu_snh_scene(ctx, m, E, nu, x)
    out = s.eval_elements(eid, project=sx.SX_PROJECT_MATERIAL, precision=precision)
    Ee, ge, He = orc.snh_batch(x, snh["tets"], snh["Dminv"], snh["V"], snh["mu"], snh["lam"],
                               2, 2)
    tol = TOL64 if precision == sx.SX_FP64 else TOL32
    scale = snh["V"] * snh["mu"]
    worst = 0.0
    for e in range(Ee.size):
        worst = max(worst, _relerr(out["H"][e], He[e], scale[e]))
    assert worst <= tol, worst
    w = np.linalg.eigvalsh(out["H"])
    assert w.min() >= -(1e-9 if precision == sx.SX_FP64 else 1e-6) * np.abs(w).max()
    s.close()


@pytest.mark.gpu
def test_material_projection_assembly_and_newton(ctx):
    from paper_2303_02156_gb300.scene import Scene
    # assembled: SNH block (material projection) + barriers (12x12 clamp)
    m, sh, bp, X, x0, E, nu, extra, nt = _mixed_small()
    N = X.shape[0]
    s = Scene(ctx, X)
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.add_hinge(sh["hinges"], sh["q"], sh["c"], 1e-3)
    s.add_barrier(bp["pairs"], 1e-3, 1e4)
    s.add_node_mass(extra)
    s.finalize()
    x = x0.copy()
    x[:nt] = scenes.jitter_state(m["X"], 3e-3, 12)
    s.set_state(x=x)
    Eg = s.eval(sx.SX_EGH, sx.SX_PROJECT_MATERIAL, sx.SX_FP64)
    rp, col, vals = s.bsr()
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    mass_all = np.concatenate([mass, np.zeros(N - nt)]) + extra
    sc = orc.Scene(N, mass=mass_all, snh=snh,
                   hinge={"stencils": sh["hinges"], "q": sh["q"], "c": sh["c"], "kb": 1e-3},
                   pt={"pairs": bp["pairs"], "dhat": 1e-3, "kappa": 1e4})
    Eo, go, vo, bad = sc.eval(x, level=2, project=2)
    assert bad == 0
    assert abs(Eg - Eo) <= TOL64 * abs(Eo)
    assert _relerr(vals, vo, 0) <= TOL64 and _relerr(s.grad(), go, 0) <= TOL64
    assert s.stats()["clamped"] > 0
    s.close()
    # a C1 backward-Euler step with the material projection
    m, E, nu = _c1()
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh, pinned=m["pinned"])
    xo, vo, st, rep = sc.newton_step(m["X"], np.zeros_like(m["X"]), 0.01, project=2)
    assert st == 0
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    rc, r = s.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10, project=sx.SX_PROJECT_MATERIAL)
    assert rc == sx.SX_OK
    xg, vg = s.get_state()
    ref = np.abs(xo - m["X"]).max()
    assert np.abs(xg - xo).max() <= 1e-8 * ref + 1e-12
    s.close()


@pytest.mark.gpu
def test_advance_halves_failed_steps_and_restores_state(ctx):
    """sx_advance: (a) a tolerance no step reaches: every substep fails and
    the state comes back unchanged; (b) with a three-iteration Newton budget
    the call equals the same policy run as single steps with snapshots
    (sx_get_state / sx_set_state), bit for bit."""
    from paper_2303_02156_gb300.scene import Scene
    m, E, nu = _c1()

    def scene():
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        return s

    x0 = scenes.jitter_state(m["X"], 1e-3, seed=4)
    x0[m["pinned"]] = m["X"][m["pinned"]]
    v0 = np.zeros_like(x0)
    v0[:, 0] = 0.1
    v0[m["pinned"]] = 0.0
    s = scene()
    s.set_state(x=x0, v=v0)
    rc, rep, n = s.advance(0.01, max_dt_halvings=2, raise_on_error=False, newton_tol=1e-300,
                           max_newton=2)
    assert rc == sx.SX_ENOTCONV and n == 0 and rep["status"] == rc
    x, v = s.get_state()
    assert np.array_equal(x, x0) and np.array_equal(v, v0)
    # three Newton iterations do not reach 1e-6 on the 0.1 s step (it takes
    # five) but do on shorter ones: a few failed substeps, each redone as halves
    opts = dict(newton_tol=1e-6, max_newton=3, pcg_tol=1e-10)
    s.set_state(x=x0, v=v0)
    rc, rep, n = s.advance(0.1, max_dt_halvings=10, raise_on_error=False, **opts)
    # the recovered failures leave no error text behind a successful call
    err_after = sx.load().sx_last_error(ctx.h).decode()
    xa = s.get_state()[0]
    s2 = scene()
    s2.set_state(x=x0, v=v0)
    todo, taken, rc2, failed = [(0.1, 0)], 0, sx.SX_OK, 0
    sums = {"newton_iters": 0, "pcg_iters": 0, "ls_halvings": 0}
    while todo:
        h, depth = todo.pop()
        xs, vs = s2.get_state()
        r2, rep2 = s2.newton_step(h, raise_on_error=False, **opts)
        if r2 == sx.SX_OK:
            taken += 1
            for k in sums:
                sums[k] += rep2[k]
            continue
        failed += 1
        s2.set_state(x=xs, v=vs)
        if depth >= 10:
            rc2 = r2
            break
        todo += [(h / 2, depth + 1), (h / 2, depth + 1)]
    # the 0.1 s step fails and succeeds only as halves: the
    # restore-then-succeed path ran
    assert rc == sx.SX_OK and rc2 == sx.SX_OK and failed >= 1
    assert n == taken and n > 1
    assert np.array_equal(xa, s2.get_state()[0])
    for k in sums:
        assert rep[k] == sums[k], k
    assert err_after == ""
    s.close(); s2.close()
