"""The other tet4 densities (§6.1 "Non-Linear Material Models", App. B:
Neo-Hookean, St. Venant-Kirchhoff, fixed co-rotational, ARAP with a volume
term; lagged rotations for the last two) through the C ABI against the
FP64 oracle, which differentiates each density by forward-mode arithmetic.

Tolerances as for SNH (normwise per element with the scale V mu: FP64
1e-10, FP32 1e-4); lagged rotations 1e-12; Newton steps 1e-8 of the
displacement.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

TOL = {sx.SX_FP64: 1e-10, sx.SX_FP32: 1e-4}
MODELS = [sx.SX_MODEL_NH, sx.SX_MODEL_STVK, sx.SX_MODEL_COROT, sx.SX_MODEL_ARAP]
LAGGED = (sx.SX_MODEL_COROT, sx.SX_MODEL_ARAP)


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


def _relerr(a, b, scale):
    a = np.asarray(a, float); b = np.asarray(b, float)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), scale)


def _case(model, dims=(6, 5, 4), seed=21, jitter=0.05):
    m = scenes.kuhn_box(*dims, h=0.25, seed=seed)
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=seed)
    inp, mass, bad = orc.tet_scene_inputs(model, m["X"], m["tets"], E, nu, 1000.0)
    assert bad == 0
    x = scenes.jitter_state(m["X"], jitter * 0.25, seed=seed + 1)
    # start-of-step state for the lagged rotations: a rotated, stretched copy
    q, _ = np.linalg.qr(np.random.default_rng(seed).normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] *= -1
    xt = scenes.jitter_state(m["X"], 0.1 * 0.25, seed=seed + 2) @ (0.3 * q + 0.7 * np.eye(3)).T
    return m, E, nu, inp, mass, x, xt


def _gpu(ctx, model, m, E, nu, x, xt=None):
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, m["X"])
    eid = s.add_tet(model, m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.finalize()
    if xt is not None:
        s.set_state(x=xt)
        s.update_rotations()
    s.set_state(x=x)
    return s, eid


@pytest.mark.gpu
@pytest.mark.parametrize("model", MODELS)
def test_lagged_rotations_parity(ctx, model):
    m, E, nu, inp, mass, x, xt = _case(model)
    s, eid = _gpu(ctx, model, m, E, nu, x, xt)
    if model not in LAGGED:
        buf = np.empty(9)
        assert sx.sx_get_rotations(s.h, eid, buf.ctypes.data, None) == sx.SX_EINVAL
        s.close()
        return
    R = s.rotations(eid).reshape(-1, 9)
    Ro = orc.lagged_rotations(xt, m["tets"], inp["Dminv"])
    assert np.abs(R - Ro).max() <= 1e-12
    # set / get round trip
    s.set_rotations(eid, Ro[::-1].copy())
    assert np.array_equal(s.rotations(eid).reshape(-1, 9), Ro[::-1])
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
@pytest.mark.parametrize("project", [False, True])
def test_model_elements_parity(ctx, model, precision, project):
    m, E, nu, inp, mass, x, xt = _case(model, jitter=0.08)
    s, eid = _gpu(ctx, model, m, E, nu, x, xt)
    R = orc.lagged_rotations(xt, m["tets"], inp["Dminv"]) if model in LAGGED else None
    out = s.eval_elements(eid, project=project, precision=precision)
    Ee, ge, He, bad = orc.tet_batch(model, x, m["tets"], inp["Dminv"], inp["V"], inp["mu"],
                                    inp["lam"], R, 2, project)
    assert bad == 0
    scale = inp["V"] * inp["mu"]
    worst = [0.0, 0.0, 0.0]
    for e in range(Ee.size):
        worst[0] = max(worst[0], abs(out["E"][e] - Ee[e]) / max(abs(Ee[e]), scale[e]))
        worst[1] = max(worst[1], _relerr(out["g"][e], ge[e], scale[e]))
        worst[2] = max(worst[2], _relerr(out["H"][e], He[e], scale[e]))
    assert max(worst) <= TOL[precision], worst
    if project:
        w = np.linalg.eigvalsh(out["H"])
        assert w.min() >= -(1e-9 if precision == sx.SX_FP64 else 1e-6) * np.abs(w).max()
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model", MODELS)
def test_model_strong_deformation_projection(ctx, model):
    """Large jitter (many indefinite element Hessians) with projection."""
    # NH is undefined at J <= 0: its case stays uninverted (min J ~ 0.06)
    jitter = 0.25 if model == sx.SX_MODEL_NH else 0.3
    m, E, nu, inp, mass, x, xt = _case(model, dims=(5, 4, 4), seed=5, jitter=jitter)
    F = orc.deformation_gradients(x, m["tets"], inp["Dminv"])
    if model == sx.SX_MODEL_NH:
        assert (np.linalg.det(F) > 0).all()
    s, eid = _gpu(ctx, model, m, E, nu, x, xt)
    R = orc.lagged_rotations(xt, m["tets"], inp["Dminv"]) if model in LAGGED else None
    out = s.eval_elements(eid, project=True, precision=sx.SX_FP64)
    Ee, ge, He, bad = orc.tet_batch(model, x, m["tets"], inp["Dminv"], inp["V"], inp["mu"],
                                    inp["lam"], R, 2, True)
    assert bad == 0
    scale = inp["V"] * inp["mu"]
    worst = max(max(_relerr(out["H"][e], He[e], scale[e]), _relerr(out["g"][e], ge[e], scale[e]))
                for e in range(Ee.size))
    assert worst <= 1e-10, worst
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model", MODELS)
def test_model_assembly_parity(ctx, model):
    m, E, nu, inp, mass, x, xt = _case(model, dims=(5, 5, 4), seed=8)
    s, eid = _gpu(ctx, model, m, E, nu, x, xt)
    if model in LAGGED:
        inp = dict(inp, R=orc.lagged_rotations(xt, m["tets"], inp["Dminv"]))
    for precision in (sx.SX_FP64, sx.SX_FP32):
        Eg = s.eval(sx.SX_EGH, True, precision)
        rp, col, vals = s.bsr()
        sc = orc.Scene(m["X"].shape[0], mass=mass, snh=inp, pinned=m["pinned"])
        Eo, go, vo, bad = sc.eval(x, level=2, project=True)
        assert bad == 0
        assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
        tol = TOL[precision]
        assert abs(Eg - Eo) <= 1e-10 * abs(Eo)   # energies are FP64 in both forms
        assert _relerr(vals, vo, 0) <= tol and _relerr(s.grad(), go, 0) <= tol
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("model", MODELS)
def test_model_newton_steps_match_oracle(ctx, model):
    """Two backward-Euler steps of a box under gravity; the second starts
    deformed, so its lagged rotations differ from the identity."""
    from paper_2303_02156_gb300.scene import Scene
    mb = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    T = mb["tets"].shape[0]
    E, nu = scenes.material_uniform(T, 1e5, 0.3)
    inp, mass, _ = orc.tet_scene_inputs(model, mb["X"], mb["tets"], E, nu, 1000.0)
    sc = orc.Scene(mb["X"].shape[0], mass=mass, snh=inp, pinned=mb["pinned"])
    s = Scene(ctx, mb["X"])
    s.add_tet(model, mb["tets"], E, nu, 1000.0)
    s.set_pinned(mb["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    xo, vo = mb["X"].copy(), np.zeros_like(mb["X"])
    for step in range(2):
        xo, vo, st, rep = sc.newton_step(xo, vo, 0.05)
        assert st == 0, rep
        rc, r = s.newton_step(0.05, newton_tol=1e-8, pcg_tol=1e-10)
        assert rc == sx.SX_OK, r
        xg, vg = s.get_state()
        ref = np.abs(xo - mb["X"]).max()
        assert np.abs(xg - xo).max() <= 1e-8 * ref + 1e-12, (step, np.abs(xg - xo).max(), ref)
        # continue both from the oracle's state so that the steps stay comparable
        s.set_state(x=xo, v=vo)
    if model in LAGGED:
        # the rotations held in the second step were those of its start state
        assert np.abs(s.rotations(0) - np.eye(3)).max() > 1e-6
    s.close()


@pytest.mark.gpu
def test_nh_inverted_tet_is_an_invalid_state(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(3, 3, 3, h=0.25, seed=2)
    T = m["tets"].shape[0]
    s = Scene(ctx, m["X"])
    s.add_tet(sx.SX_MODEL_NH, m["tets"], np.full(T, 1e5), np.full(T, 0.3), 1000.0)
    s.finalize()
    x = m["X"].copy()
    t = m["tets"][7]
    x[t[3]] = x[t[0]] - (x[t[3]] - x[t[0]])   # reflect a vertex: J < 0 in that tet
    s.set_state(x=x)
    E = C.c_double()
    rc = sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP64, C.byref(E), None)
    assert rc == sx.SX_ESTATE
    assert s.stats()["bad_state"] >= 1
    # the same tet under StVK is a valid state
    s2 = Scene(ctx, m["X"])
    s2.add_tet(sx.SX_MODEL_STVK, m["tets"], np.full(T, 1e5), np.full(T, 0.3), 1000.0)
    s2.finalize()
    s2.set_state(x=x)
    assert sx.sx_eval(s2.h, sx.SX_EGH, 1, sx.SX_FP64, C.byref(E), None) == sx.SX_OK
    s.close(); s2.close()


@pytest.mark.gpu
def test_models_mixed_in_one_batch_equal_single(ctx):
    """Scenes of every model (and SNH) in one batched evaluation and one
    batched Newton step: each equal bit for bit to its own call."""
    from paper_2303_02156_gb300.scene import Scene
    sc = []
    for k, model in enumerate([sx.SX_MODEL_SNH] + MODELS):
        mb = scenes.kuhn_box(3 + k % 2, 3, 3, h=0.2, seed=10 + k)
        T = mb["tets"].shape[0]
        s = Scene(ctx, mb["X"])
        s.add_tet(model, mb["tets"], np.full(T, 2e5), np.full(T, 0.35), 1000.0)
        s.set_pinned(mb["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        s.set_state(x=scenes.jitter_state(mb["X"], 0.01, seed=k))
        sc.append((s, mb))
    arr = (C.c_void_p * len(sc))(*[s.h.value for s, _ in sc])
    Eb = (C.c_double * len(sc))()
    assert sx.sx_eval_batch(sc[0][0].ctx.h, arr, len(sc), sx.SX_EGH, 1, sx.SX_FP64, Eb,
                            None) == sx.SX_OK
    vb = [s.bsr()[2].copy() for s, _ in sc]
    for i, (s, _) in enumerate(sc):
        E1 = s.eval(sx.SX_EGH, True, sx.SX_FP64)
        assert E1 == Eb[i] and np.array_equal(s.bsr()[2], vb[i])
    for s, mb in sc:
        s.set_state(x=mb["X"], v=np.zeros_like(mb["X"]))
    reps = (sx.sx_step_report * len(sc))()
    o = sx.newton_opts(newton_tol=1e-8, pcg_tol=1e-10)
    assert sx.sx_newton_step_batch(ctx.h, arr, len(sc), 0.02, C.byref(o), reps, None) == sx.SX_OK
    xb = [s.get_state()[0] for s, _ in sc]
    for i, (s, mb) in enumerate(sc):
        s.set_state(x=mb["X"], v=np.zeros_like(mb["X"]))
        rc, _ = s.newton_step(0.02, newton_tol=1e-8, pcg_tol=1e-10)
        assert rc == sx.SX_OK
        assert np.array_equal(s.get_state()[0], xb[i]), i
    for s, _ in sc:
        s.close()
