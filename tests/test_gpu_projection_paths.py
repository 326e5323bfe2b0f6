"""Phase 2 of the projection (§5.2 "Projection to positive semi-definiteness")
runs different paths by the size k of a stencil's N block: the certified
subspace refinement (k = 1..3, two passes), the deflation of 1..3 clearly
negative modes of a stencil with k >= 4 (the rest certified by a double
LDL^T), the block-restricted double Jacobi (other k = 4..8) and the
warp-per-stencil Jacobi (bin 9). These tests assemble
scenes whose stencils take each path, read the bin counts of the evaluation
(sx_projection_bins) to show that the path ran, and compare the assembled
system with the FP64 oracle's (FP64 1e-10, FP32 1e-4, normwise over the BSR
values; the pattern bit-identical).
"""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as orc
from paper_2303_02156_gb300 import scenes, sx

TOL64, TOL32 = 1e-10, 1e-4
NBINS = 20


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


def _relerr(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _bins(ctx, s):
    b = (C.c_int * NBINS)()
    ctx.check(sx.sx_projection_bins(ctx.h, b, s.stream))
    return list(b)


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_refinement_passes_match_oracle(ctx, precision):
    """A strongly deformed SNH box (inverted tets, jitter 0.45 h): stencils of
    k = 1..3 go through the refinement, some of them (an N block close to
    the next eigenvalue) through its second pass; tets with 4 or 5 negative
    modes through the block-restricted Jacobi."""
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(10, 9, 8, h=0.25, seed=31)
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=31)
    x = scenes.jitter_state(m["X"], 0.45 * 0.25, seed=32)
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.finalize()
    s.set_state(x=x)
    s.eval(sx.SX_EGH, True, precision)
    bins = _bins(ctx, s)
    rp, col, vals = s.bsr()
    clamped = s.stats()["clamped"]
    snh, mass, bad = orc.snh_scene_inputs(m["X"], m["tets"], E, nu, 1000.0)
    assert bad == 0
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh)
    _, _, vo, bad = sc.eval(x, level=2, project=True)
    assert bad == 0
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    tol = TOL64 if precision == sx.SX_FP64 else TOL32
    err = _relerr(vals, vo)
    # every queued stencil sits in one bin of the float part's (0..9 or a
    # deflation bin); bin 9 also takes what the second pass did not certify
    assert sum(bins[:10]) + sum(bins[17:20]) >= clamped > 0, bins
    assert sum(bins[1:4]) > 0 and sum(bins[11:14]) > 0, bins
    assert sum(bins[4:9]) > 0, bins
    assert err <= tol, (err, bins)
    s.close()


def _barrier_case(n_pairs=600, seed=41):
    sh = scenes.shell_sheet(12, length=0.01, noise=0.05, seed=seed)
    nv = sh["x"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], n_pairs, 1e-4, 1e-3, seed=seed,
                              tri_node_offset=0, point_node_offset=nv)
    X = np.vstack([sh["X"], bp["points"]])
    x = np.vstack([sh["x"], bp["points"]])
    return X, x, bp["pairs"]


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
def test_deflation_matches_oracle(ctx, precision):
    """Point-triangle barrier stencils: their Hessians have a null space
    (four exact zeros in the translation-free 9x9) and two negative modes
    from the distance's curvature, so k = 6 with k' = 2 clearly negative
    modes: the deflation refines those two and certifies the rest."""
    from paper_2303_02156_gb300.scene import Scene
    X, x, pairs = _barrier_case()
    s = Scene(ctx, X)
    s.add_barrier(pairs, 1e-3, 1e4)
    s.finalize()
    s.set_state(x=x)
    s.eval(sx.SX_EGH, True, precision)
    bins = _bins(ctx, s)
    rp, col, vals = s.bsr()
    sc = orc.Scene(X.shape[0], pt={"pairs": pairs, "dhat": 1e-3, "kappa": 1e4})
    _, _, vo, bad = sc.eval(x, level=2, project=True)
    assert bad == 0
    assert np.array_equal(rp, sc.row_ptr) and np.array_equal(col, sc.col)
    tol = TOL64 if precision == sx.SX_FP64 else TOL32
    err = _relerr(vals, vo)
    assert sum(bins[17:20]) > 0, bins
    assert err <= tol, (err, bins)
    s.close()


@pytest.mark.gpu
def test_bins_are_zero_before_any_projection(ctx):
    """The diagnostics of a context that has not projected anything."""
    from paper_2303_02156_gb300.scene import Context
    c = Context(0)
    b = (C.c_int * NBINS)()
    c.check(sx.sx_projection_bins(c.h, b, None))
    assert list(b) == [0] * NBINS
    c.close()
