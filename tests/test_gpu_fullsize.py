"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on sampled outputs the oracle computes one by one.

* 64^3 Kuhn cube (1,572,864 SNH tets): one ``sx_eval(EGH, project)`` of the
  whole scene; for sampled nodes, every element touching the node is
  evaluated by the oracle (a sub-scene of those elements) and the node's
  assembled BSR row and gradient are compared (pattern bit-identical,
  values normwise per row: FP64 1e-10, FP32 1e-4).
* Mixed stencils (998,250 tets + 2,998,000 hinges + 4,000,000 barrier
  pairs in one scene): the same row check on nodes of each DOF set.
* 512 batched boxes, one batched Newton step: small sampled scenes against
  the oracle's Newton step, and sampled scenes stepped alone equal to their
  batched result bit for bit (the batch changes no scene's arithmetic).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

TOL = {sx.SX_FP64: 1e-10, sx.SX_FP32: 1e-4}


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


def _oracle_rows(X, x, sample, snh=None, hinge=None, pt=None):
    """Oracle rows of the sampled nodes: a sub-scene of every stencil that
    touches one of them, evaluated at E + g + projected H."""
    conns = []
    if snh is not None:
        conns.append(snh["tets"])
    if hinge is not None:
        conns.append(hinge["stencils"])
    if pt is not None:
        conns.append(pt["pairs"])
    sel = [np.isin(c, sample).any(axis=1) for c in conns]
    used = np.unique(np.concatenate([c[s].ravel() for c, s in zip(conns, sel)] + [sample]))
    remap = -np.ones(X.shape[0], dtype=np.int64)
    remap[used] = np.arange(used.size)
    k = 0
    sub = {}
    if snh is not None:
        s = sel[k]; k += 1
        t = remap[snh["tets"][s]].astype(np.int32)
        inp, _, bad = orc.snh_scene_inputs(X[used], t, snh["E"][s], snh["nu"][s], 1000.0)
        assert bad == 0
        sub["snh"] = inp
    if hinge is not None:
        s = sel[k]; k += 1
        sub["hinge"] = {"stencils": remap[hinge["stencils"][s]].astype(np.int32),
                        "q": hinge["q"][s], "c": hinge["c"][s], "kb": hinge["kb"]}
    if pt is not None:
        s = sel[k]; k += 1
        sub["pt"] = {"pairs": remap[pt["pairs"][s]].astype(np.int32), "dhat": pt["dhat"],
                     "kappa": pt["kappa"]}
    sc = orc.Scene(used.size, **sub)
    E, g, vals, bad = sc.eval(x[used], level=2, project=True)
    assert bad == 0
    return used, remap, sc, g, vals


def _check_rows(gpu, X, x, sample, precision, **blocks):
    rp, col, vals = gpu.bsr()
    grad = gpu.grad()
    used, remap, sc, go, vo = _oracle_rows(X, x, sample, **blocks)
    tol = TOL[precision]
    worst = 0.0
    for r in sample:
        a, b = rp[r], rp[r + 1]
        rs = remap[r]
        oa, ob = sc.row_ptr[rs], sc.row_ptr[rs + 1]
        # same columns (in global ids), ascending
        assert np.array_equal(col[a:b], used[sc.col[oa:ob]]), r
        v = vals[a:b].astype(np.float64)
        ref = vo[oa:ob]
        e = np.linalg.norm(v - ref) / max(np.linalg.norm(ref), 1e-300)
        gr = go[3 * rs:3 * rs + 3]
        # the gradient row is compared against the row's stiffness scale
        # times the node's coordinate scale (it is zero at equilibrium)
        eg = np.linalg.norm(grad[3 * r:3 * r + 3] - gr) / max(
            np.linalg.norm(gr), np.linalg.norm(ref) * 1e-6, 1e-300)
        worst = max(worst, e, eg)
    assert worst <= tol, worst
    return worst


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_cube_64_sampled_rows(ctx, precision):
    from paper_2303_02156_gb300.scene import Scene
    n = 64
    m = scenes.kuhn_box(n, n, n, h=1.0 / n, seed=2)
    T = m["tets"].shape[0]
    assert T == 1572864
    E, nu = scenes.material_random(T, seed=2)
    x = scenes.jitter_state(m["X"], 0.02 / n, seed=5)
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.finalize()
    assert s.info()["nnzb"] == 4018753
    s.set_state(x=x)
    s.eval(sx.SX_EGH, True, precision)
    assert s.stats()["nonfinite"] == 0
    N = m["X"].shape[0]
    rng = np.random.default_rng(17)
    sample = np.unique(np.concatenate([[0, N - 1, n, N // 2], rng.integers(0, N, 60)]))
    _check_rows(s, m["X"], x, sample, precision,
                snh={"tets": m["tets"], "E": E, "nu": nu})
    s.close()


@pytest.fixture(scope="module")
def mixed(ctx):
    from paper_2303_02156_gb300.scene import Scene
    w = scenes.mixed_scene()
    s = Scene(ctx, w["X"])
    s.add_snh(w["tets"], w["E"], w["nu"], 1000.0)
    s.add_hinge(w["hinges"], w["q"], w["c"], w["kb"])
    s.add_barrier(w["pairs"], w["dhat"], w["kappa"])
    s.add_node_mass(w["extra_mass"])
    s.set_pinned(w["pinned"])
    s.finalize()
    s.set_state(x=w["x"])
    yield s, w
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP32, sx.SX_FP64])
def test_mixed_full_size_sampled_rows(ctx, mixed, precision):
    s, w = mixed
    s.eval(sx.SX_EGH, True, precision)
    st = s.stats()
    assert st["bad_state"] == 0 and st["nonfinite"] == 0 and st["clamped"] > 0
    nb, ns, npnt = w["n_block_nodes"], w["n_sheet_nodes"], w["n_points"]
    rng = np.random.default_rng(23)
    sample = np.unique(np.concatenate([
        rng.integers(0, nb, 12),                  # SNH block
        nb + rng.integers(0, ns, 12),             # sheet (hinges + barrier triangles)
        nb + ns + rng.integers(0, npnt, 12)]))    # barrier points
    _check_rows(s, w["X"], w["x"], sample, precision,
                snh={"tets": w["tets"], "E": w["E"], "nu": w["nu"]},
                hinge={"stencils": w["hinges"], "q": w["q"], "c": w["c"], "kb": w["kb"]},
                pt={"pairs": w["pairs"], "dhat": w["dhat"], "kappa": w["kappa"]})


@pytest.fixture(scope="module")
def batch512(ctx):
    from paper_2303_02156_gb300.scene import Scene
    boxes = scenes.batch_boxes(512)
    sc = []
    for b in boxes:
        s = Scene(ctx, b["X"])
        s.add_snh(b["tets"], b["E"], b["nu"], 1000.0)
        s.set_pinned(b["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        sc.append(s)
    yield boxes, sc
    for s in sc:
        s.close()


def _oracle_step(b, dt):
    T = b["tets"].shape[0]
    snh, mass, _ = orc.snh_scene_inputs(b["X"], b["tets"], np.full(T, b["E"]),
                                        np.full(T, b["nu"]), 1000.0)
    osc = orc.Scene(b["X"].shape[0], mass=mass, snh=snh, pinned=b["pinned"])
    xo, _, st, _ = osc.newton_step(b["X"], np.zeros_like(b["X"]), dt)
    assert st == 0
    return xo


@pytest.mark.gpu
def test_batched_512_newton_step(ctx, batch512):
    boxes, sc = batch512
    for s, b in zip(sc, boxes):
        s.set_state(x=b["X"], v=np.zeros_like(b["X"]))
    dt = 0.01
    arr = (C.c_void_p * len(sc))(*[s.h.value for s in sc])
    reps = (sx.sx_step_report * len(sc))()
    o = sx.newton_opts(newton_tol=1e-8, pcg_tol=1e-10)
    rc = sx.sx_newton_step_batch(ctx.h, arr, len(sc), dt, C.byref(o), reps, None)
    assert rc == sx.SX_OK, [r.status for r in reps if r.status != 0][:5]
    xb = [s.get_state()[0] for s in sc]
    sizes = np.array([b["tets"].shape[0] for b in boxes])
    # small scenes: the oracle's Newton step (item-10 tolerance of a step)
    for k in np.argsort(sizes)[:3]:
        b = boxes[k]
        xo = _oracle_step(b, dt)
        ref = np.abs(xo - b["X"]).max()
        assert np.abs(xb[k] - xo).max() <= 1e-8 * ref + 1e-12, k
    # sampled scenes alone (the largest, the median, a small one): bitwise
    # equal to their batched result
    order = np.argsort(sizes)
    for k in [order[-1], order[len(order) // 2], order[5]]:
        b = boxes[k]
        sc[k].set_state(x=b["X"], v=np.zeros_like(b["X"]))
        rc, r = sc[k].newton_step(dt, newton_tol=1e-8, pcg_tol=1e-10)
        assert rc == sx.SX_OK
        assert np.array_equal(sc[k].get_state()[0], xb[k]), k


@pytest.mark.gpu
def test_batched_512_newton_step_fp32(ctx, batch512):
    """The FP32 form of the batched step (FP32 element math, BSR values and
    SpMV; FP64 projection, norms, dots and energy sums) at its Newton and PCG
    tolerance 1e-6, against the FP64 oracle's step: displacement error within
    1e-5 of the displacement, on the three smallest scenes and one of median
    size."""
    boxes, sc = batch512
    for s, b in zip(sc, boxes):
        s.set_state(x=b["X"], v=np.zeros_like(b["X"]))
    dt = 0.01
    arr = (C.c_void_p * len(sc))(*[s.h.value for s in sc])
    reps = (sx.sx_step_report * len(sc))()
    o = sx.newton_opts(newton_tol=1e-6, pcg_tol=1e-6, precision=sx.SX_FP32)
    rc = sx.sx_newton_step_batch(ctx.h, arr, len(sc), dt, C.byref(o), reps, None)
    assert rc == sx.SX_OK, [r.status for r in reps if r.status != 0][:5]
    sizes = np.array([b["tets"].shape[0] for b in boxes])
    order = np.argsort(sizes)
    worst = 0.0
    for k in list(order[:3]) + [order[len(order) // 2]]:
        b = boxes[k]
        xo = _oracle_step(b, dt)
        ref = np.abs(xo - b["X"]).max()
        err = np.abs(sc[k].get_state()[0] - xo).max()
        worst = max(worst, err / ref)
        assert err <= 1e-5 * ref, (k, err, ref)
    print(f"FP32 batched step vs FP64 oracle: worst relative displacement error {worst:.2e}")
