"""Changing contact pairs: activation compaction (only pairs with
0 < d < dhat contribute, §6.4 Eq. 15) and a rebuilt fixed pattern when the
pairs of a barrier block change (§5.3), against the oracle built on the
same pair list."""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

TOL = 1e-10


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


def _relerr(a, b, scale=0.0):
    a = np.asarray(a, float); b = np.asarray(b, float)
    return np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), scale, 1e-300)


def _scene_parts(seed=5, n_pairs=120):
    """SNH block, then a barrier block over a sheet (points at d ~ U(1e-4,
    2e-3), so about half are beyond dhat = 1e-3), then the sheet's hinges:
    the barrier block sits between two others, so its size changes shift
    the stencil numbering of the block after it."""
    m = scenes.kuhn_box(3, 3, 2, h=0.01, seed=seed)
    nt = m["X"].shape[0]
    sh = scenes.shell_sheet(6, length=0.03, z0=0.03, noise=0.05, seed=seed, node_offset=nt)
    ns = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"] - nt, n_pairs, 1e-4, 2e-3, seed=seed,
                              tri_node_offset=nt, point_node_offset=nt + ns)
    X = np.vstack([m["X"], sh["X"], bp["points"]])
    x = np.vstack([scenes.jitter_state(m["X"], 2e-4, seed + 1), sh["x"], bp["points"]])
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed)
    extra = np.zeros(X.shape[0])
    extra[nt:] = 1e-4
    return m, sh, bp, X, x, E, nu, extra, nt


def _gpu(ctx, parts, pairs):
    from paper_2303_02156_gb300.scene import Scene
    m, sh, bp, X, x, E, nu, extra, nt = parts
    s = Scene(ctx, X)
    s.add_snh(m["tets"], E, nu, 1000.0)
    eb = s.add_barrier(pairs, 1e-3, 1e4)
    s.add_hinge(sh["hinges"], sh["q"], sh["c"], 1e-3)
    s.add_node_mass(extra)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    s.finalize()
    s.set_state(x=x)
    return s, eb


def _oracle(parts, pairs):
    m, sh, bp, X, x, E, nu, extra, nt = parts
    N = X.shape[0]
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    mass_all = np.concatenate([mass, np.zeros(N - nt)]) + extra
    # registration order of the oracle: tets, hinges, pairs. The pattern and
    # the assembled values do not depend on the order of the blocks.
    return orc.Scene(N, mass=mass_all, snh=snh,
                     hinge={"stencils": sh["hinges"], "q": sh["q"], "c": sh["c"], "kb": 1e-3},
                     pt={"pairs": pairs, "dhat": 1e-3, "kappa": 1e4}, pinned=m["pinned"])


@pytest.mark.gpu
def test_compaction_keeps_active_pairs_and_rebuilds_pattern(ctx):
    parts = _scene_parts()
    m, sh, bp, X, x, E, nu, extra, nt = parts
    pairs = bp["pairs"]
    _, _, _, act, bad = orc.barrier_batch(x, pairs, 1e-3, 1e4, 0, False)
    assert bad == 0 and 0 < (act == 1).sum() < pairs.shape[0]
    s, eb = _gpu(ctx, parts, pairs)
    E0 = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    g0 = s.grad()
    nnz0 = s.info()["nnzb"]
    n_act = s.compact_pairs(eb)
    active = pairs[act == 1]
    assert n_act == active.shape[0]
    E1 = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, vals = s.bsr()
    sc = _oracle(parts, active)
    Eo, go, vo, bado = sc.eval(x, level=2, project=True)
    assert bado == 0
    # pattern and maps of the active set, bit-identical; fewer blocks
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    assert s.info()["nnzb"] == sc.nnzb < nnz0
    assert abs(E1 - Eo) <= TOL * abs(Eo)
    assert _relerr(s.grad(), go) <= TOL and _relerr(vals, vo) <= TOL
    # inactive pairs contributed nothing before either
    assert abs(E1 - E0) <= 1e-12 * abs(E0) and _relerr(s.grad(), g0) <= 1e-12
    # the state is the same
    assert np.array_equal(s.get_state()[0], x)
    s.close()


@pytest.mark.gpu
def test_set_pairs_replaces_pairs_and_keeps_state(ctx):
    parts = _scene_parts(seed=6, n_pairs=60)
    m, sh, bp, X, x, E, nu, extra, nt = parts
    s, eb = _gpu(ctx, parts, bp["pairs"][:10])
    s.eval(sx.SX_EGH, True, sx.SX_FP64)
    # a new pair list (a different subset and order)
    new = bp["pairs"][::-2].copy()
    s.set_pairs(eb, new)
    E1 = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, vals = s.bsr()
    sc = _oracle(parts, new)
    Eo, go, vo, bado = sc.eval(x, level=2, project=True)
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    assert abs(E1 - Eo) <= TOL * abs(Eo)
    assert _relerr(s.grad(), go) <= TOL and _relerr(vals, vo) <= TOL
    # no pairs at all
    s.set_pairs(eb, np.zeros((0, 4), np.int32))
    E2 = s.eval(sx.SX_EGH, True, sx.SX_FP64)
    sc2 = _oracle(parts, np.zeros((0, 4), np.int32))
    Eo2, _, vo2, _ = sc2.eval(x, level=2, project=True)
    assert abs(E2 - Eo2) <= TOL * abs(Eo2) and _relerr(s.bsr()[2], vo2) <= TOL
    s.close()


@pytest.mark.gpu
def test_newton_step_after_compaction_matches_oracle(ctx):
    parts = _scene_parts(seed=7, n_pairs=80)
    m, sh, bp, X, x, E, nu, extra, nt = parts
    pairs = bp["pairs"]
    s, eb = _gpu(ctx, parts, pairs)
    s.set_state(x=x, v=np.zeros_like(x))
    n_act = s.compact_pairs(eb)
    _, _, _, act, _ = orc.barrier_batch(x, pairs, 1e-3, 1e4, 0, False)
    active = pairs[act == 1]
    assert n_act == active.shape[0]
    rc, r = s.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10)
    assert rc == sx.SX_OK, r
    xg, vg = s.get_state()
    sc = _oracle(parts, active)
    xo, vo, st, rep = sc.newton_step(x, np.zeros_like(x), 0.01)
    assert st == 0
    ref = np.abs(xo - x).max()
    assert np.abs(xg - xo).max() <= 1e-8 * ref + 1e-12
    s.close()


@pytest.mark.gpu
def test_pair_updates_reject_other_blocks(ctx):
    import ctypes as C
    parts = _scene_parts(seed=8, n_pairs=20)
    s, eb = _gpu(ctx, parts, parts[2]["pairs"])
    n = C.c_int64()
    assert sx.sx_compact_pairs(s.h, 0, C.byref(n), None) == sx.SX_EINVAL   # the SNH block
    assert sx.sx_set_pairs(s.h, 7, None, 0, None) == sx.SX_EINVAL
    s.close()
