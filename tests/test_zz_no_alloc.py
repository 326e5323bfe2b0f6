"""sx_eval_elements_noalloc: the element-level evaluation for callers that
cannot let the library allocate device memory during a call (memory held
by their own caching allocator, or a fixed-latency loop that must avoid
cudaMalloc's device-wide synchronization). Its scratch lives in static
device arrays, so its results must equal those of sx_eval_elements (which
allocates its scratch per call), on two calls in a row -- the second call
reuses the static arrays the first one left behind.

Kept in a file of its own that pytest collects last; it passes alone in a
fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2303_02156_gb300 import scenes, sx

TOL64 = 1e-10


@pytest.mark.gpu
def test_noalloc_matches_allocating_path_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02156_gb300.scene import Context, Scene
    ctx = Context(0)
    m = scenes.kuhn_box(6, 5, 4, h=0.25, seed=13)          # 720 tets: several tiles + tail
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=13)
    x = scenes.jitter_state(m["X"], 0.01, seed=14)
    s = Scene(ctx, m["X"])
    eid = s.add_snh(m["tets"], E, nu, 1000.0)
    s.finalize()
    s.set_state(x=x)
    ref = s.eval_elements(eid, project=True, precision=sx.SX_FP64)
    assert ref["H"].shape == (T, 12, 12)
    dev = torch.device("cuda")
    for call in range(2):
        Eo = torch.full((T,), np.nan, dtype=torch.float64, device=dev)
        go = torch.full((T, 12), np.nan, dtype=torch.float64, device=dev)
        Ho = torch.full((T, 12, 12), np.nan, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        rc = sx.sx_eval_elements_noalloc(s.h, eid, 1, sx.SX_FP64, Eo.data_ptr(), go.data_ptr(),
                                         Ho.data_ptr(), None)
        ctx.check(rc)
        torch.cuda.synchronize()
        E_, g_, H_ = Eo.cpu().numpy(), go.cpu().numpy(), Ho.cpu().numpy()
        scale = np.abs(ref["H"]).reshape(T, -1).max(axis=1)
        for e in range(T):
            assert abs(E_[e] - ref["E"][e]) <= TOL64 * max(abs(ref["E"][e]), 1e-30), (call, e)
            assert np.linalg.norm(g_[e] - ref["g"][e]) <= TOL64 * max(np.linalg.norm(ref["g"][e]), 1e-30)
            assert np.linalg.norm(H_[e] - ref["H"][e]) <= TOL64 * scale[e], (call, e)
    # sizes beyond the static scratch are rejected with a clear error
    big = scenes.kuhn_box(24, 24, 24, h=0.05, seed=1)       # 82,944 tets > 65,536
    s2 = Scene(ctx, big["X"])
    e2 = s2.add_snh(big["tets"], 1e5, 0.3)
    s2.finalize()
    rc = sx.sx_eval_elements_noalloc(s2.h, e2, 1, sx.SX_FP64, None, None, None, None)
    assert rc == sx.SX_EINVAL
    assert b"static scratch" in sx.load().sx_last_error(ctx.h)
    s2.close()
    s.close()
    ctx.close()
