"""Failure detection without a GPU fault: non-finite inputs made on the host
come back as SX_ENAN from an evaluation and a Newton step, which leaves the
scene's state as it was; an allocation failure injected on the host
(sx_inject_alloc_failure) comes back as SX_ENOMEM and leaves the context
usable. The time-step halving restart built on these codes (§7 intro) is
tested in test_gpu_parity.py."""
import ctypes as C

import numpy as np
import pytest

from paper_2303_02156_gb300 import scenes, sx


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


def _cube():
    m = scenes.kuhn_box(4, 4, 4, h=0.25, seed=1)
    E, nu = scenes.material_uniform(m["tets"].shape[0], 1e5, 0.3)
    return m, E, nu


def _scene(ctx, m, E, nu, finalize=True):
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, m["X"])
    s.add_snh(m["tets"], E, nu, 1000.0)
    s.set_pinned(m["pinned"])
    s.set_gravity((0.0, 0.0, -9.81))
    if finalize:
        s.finalize()
    return s


def _moving_state(m):
    x0 = scenes.jitter_state(m["X"], 1e-3, seed=3)
    x0[m["pinned"]] = m["X"][m["pinned"]]
    v0 = np.zeros_like(x0)
    v0[:, 0] = 0.2
    v0[m["pinned"]] = 0.0
    return x0, v0


@pytest.mark.gpu
def test_nan_young_modulus_reports_enan_and_keeps_state(ctx):
    m, E, nu = _cube()
    E = E.copy()
    E[17] = np.nan
    s = _scene(ctx, m, E, nu)
    x0, v0 = _moving_state(m)
    s.set_state(x=x0, v=v0)
    rc, _ = s.eval(sx.SX_EGH, True, sx.SX_FP64, check=False)
    assert rc == sx.SX_ENAN
    assert s.stats()["nonfinite"] > 0
    for prec in (sx.SX_FP64, sx.SX_FP32):
        rc, rep = s.newton_step(0.01, raise_on_error=False, precision=prec)
        assert rc == sx.SX_ENAN and rep["status"] == sx.SX_ENAN
        x, v = s.get_state()
        assert np.array_equal(x, x0) and np.array_equal(v, v0)
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("where", ["x", "v"])
def test_nan_state_reports_enan_and_keeps_state(ctx, where):
    m, E, nu = _cube()
    s = _scene(ctx, m, E, nu)
    x0, v0 = _moving_state(m)
    free = np.flatnonzero(~np.isin(np.arange(m["X"].shape[0]), m["pinned"]))
    (x0 if where == "x" else v0)[free[5], 1] = np.nan
    s.set_state(x=x0, v=v0)
    if where == "x":
        rc, _ = s.eval(sx.SX_EGH, True, sx.SX_FP64, check=False)
        assert rc == sx.SX_ENAN
    rc, rep = s.newton_step(0.01, raise_on_error=False)
    assert rc == sx.SX_ENAN
    x, v = s.get_state()
    assert np.array_equal(x, x0, equal_nan=True) and np.array_equal(v, v0, equal_nan=True)
    # the same scene steps normally once the state is finite again
    x1, v1 = _moving_state(m)
    s.set_state(x=x1, v=v1)
    rc, _ = s.newton_step(0.01, raise_on_error=False)
    assert rc == sx.SX_OK
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("nth", [1, 4, 9])
def test_injected_allocation_failure_in_finalize(ctx, nth):
    """The nth allocation of finalize fails: SX_ENOMEM, the scene stays
    unfinalized, a retry succeeds and evaluates bit for bit as a scene that
    never failed; the context keeps working."""
    m, E, nu = _cube()
    ref = _scene(ctx, m, E, nu)
    x0, v0 = _moving_state(m)
    ref.set_state(x=x0, v=v0)
    Er = ref.eval()
    gr = ref.grad()
    s = _scene(ctx, m, E, nu, finalize=False)
    assert sx.sx_inject_alloc_failure(ctx.h, nth) == sx.SX_OK
    rc = sx.sx_finalize(s.h, None)
    assert rc == sx.SX_ENOMEM
    assert "allocation" in sx.load().sx_last_error(ctx.h).decode()
    assert sx.sx_eval(s.h, sx.SX_EGH, 1, sx.SX_FP64, None, None) == sx.SX_EORDER
    assert sx.sx_finalize(s.h, None) == sx.SX_OK
    s.set_state(x=x0, v=v0)
    assert s.eval() == Er
    assert np.array_equal(s.grad(), gr)
    rc, _ = s.newton_step(0.01, raise_on_error=False)
    assert rc == sx.SX_OK
    ref.close(); s.close()


@pytest.mark.gpu
def test_injected_allocation_failure_in_newton_step(ctx):
    """The first FP32 step of a scene allocates its FP32 values; an injected
    failure there returns SX_ENOMEM without moving the scene, and the next
    step (no injection) is taken."""
    m, E, nu = _cube()
    s = _scene(ctx, m, E, nu)
    x0, v0 = _moving_state(m)
    s.set_state(x=x0, v=v0)
    assert sx.sx_inject_alloc_failure(ctx.h, 1) == sx.SX_OK
    rc, _ = s.newton_step(0.01, raise_on_error=False, precision=sx.SX_FP32,
                          newton_tol=1e-6, pcg_tol=1e-6)
    assert rc == sx.SX_ENOMEM
    x, v = s.get_state()
    assert np.array_equal(x, x0) and np.array_equal(v, v0)
    rc, _ = s.newton_step(0.01, raise_on_error=False, precision=sx.SX_FP32,
                          newton_tol=1e-6, pcg_tol=1e-6)
    assert rc == sx.SX_OK
    assert not np.array_equal(s.get_state()[0], x0)
    assert sx.sx_inject_alloc_failure(ctx.h, -1) == sx.SX_EINVAL
    s.close()
