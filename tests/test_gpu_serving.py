"""Serving form: continuous batching of backward-Euler steps (the benchmark spec
"serving"). Each request's result must be the same alone and in the mix;
admission respects the memory budget."""
import time

import numpy as np
import pytest

from paper_2303_02156_gb300 import scenes, sx


def _requests(n, seed, tmin=60, tmax=900):
    rng = scenes.rng_for(seed)
    out = []
    for k in range(n):
        T = float(np.exp(rng.uniform(np.log(tmin), np.log(tmax))))
        dims = scenes.random_box_dims(T, rng)
        m = scenes.kuhn_box(*dims, h=0.05, seed=seed * 100 + k)
        E = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
        nu = float(rng.uniform(0.2, 0.45))
        out.append((m, E, nu))
    return out


def test_footprint_estimate_grows_with_size():
    d = sx.sx_scene_desc()
    import ctypes as C
    last = 0
    for n in [10, 1000, 100000]:
        d.n_nodes = n; d.n_tets = 5 * n; d.n_hinges = 0; d.n_pairs = 0; d.nnzb_hint = 0
        b = C.c_int64()
        assert sx.sx_scene_footprint(C.byref(d), C.byref(b)) == sx.SX_OK
        assert b.value > last
        last = b.value


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2303_02156_gb300.scene import Context
    c = Context(0)
    yield c
    c.close()


@pytest.mark.gpu
@pytest.mark.parametrize("lanes", [None, [], [250, 500]])
def test_alone_equals_mix_with_staggered_arrivals(ctx, lanes):
    from paper_2303_02156_gb300.scene import Scene, Server
    reqs = _requests(6, seed=7)
    steps, dt, g = 3, 0.01, (0.0, 0.0, -9.81)
    alone = []
    for m, E, nu in reqs:
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity(g)
        s.finalize()
        for _ in range(steps):
            s.newton_step(dt)
        alone.append(s.get_state())
        s.close()
    srv = Server(ctx, 8 << 30, lanes=lanes)
    ids = []
    for k, (m, E, nu) in enumerate(reqs):
        ids.append(srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], gravity=g,
                              n_steps=steps, dt=dt))
        if k == 2:
            time.sleep(0.05)   # later requests arrive while the first are on the GPU
    assert srv.drain(120000.0) == sx.SX_OK
    done = {c["req_id"]: c for c in srv.poll()}
    st = srv.stats()
    assert st["completed"] == 6 and st["step_p99_ms"] >= st["step_p50_ms"] > 0
    for rid, (xa, va) in zip(ids, alone):
        assert done[rid]["status"] == sx.SX_OK and done[rid]["steps"] == steps, done[rid]["error"]
        x, v = srv.result(rid)
        assert np.array_equal(x, xa) and np.array_equal(v, va)
    srv.close()


@pytest.mark.gpu
def test_admission_by_budget_and_rejection(ctx):
    from paper_2303_02156_gb300.scene import Server
    reqs = _requests(4, seed=11, tmin=300, tmax=600)
    import ctypes as C
    fps = []
    for m, E, nu in reqs:
        d = sx.sx_scene_desc()
        d.n_nodes = m["X"].shape[0]; d.n_tets = m["tets"].shape[0]
        b = C.c_int64()
        sx.sx_scene_footprint(C.byref(d), C.byref(b))
        fps.append(b.value)
    budget = int(max(fps) * 1.2)   # one scene at a time
    srv = Server(ctx, budget)
    for m, E, nu in reqs:
        srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], n_steps=2, dt=0.01)
    assert srv.drain(120000.0) == sx.SX_OK
    st = srv.stats()
    assert st["completed"] == 4 and st["peak_bytes"] <= budget and st["rejected"] == 0
    big = scenes.kuhn_box(12, 12, 12, h=0.05, seed=1)
    with pytest.raises(sx.SxError) as ei:
        srv.submit(big["X"], big["tets"], 1e5, 0.3, n_steps=1, dt=0.01)
    assert ei.value.code == sx.SX_EBUDGET
    assert srv.stats()["rejected"] == 1
    srv.close()


@pytest.mark.gpu
def test_lanes_fixed_after_first_submit(ctx):
    import ctypes as C
    from paper_2303_02156_gb300.scene import Server
    srv = Server(ctx, 1 << 30)
    b = (C.c_int64 * 2)(100, 50)   # not increasing
    assert sx.sx_server_set_lanes(srv.h, 3, b) == sx.SX_EINVAL
    assert sx.sx_server_set_lanes(srv.h, sx.SX_SERVER_MAX_LANES + 1, b) == sx.SX_EINVAL
    m, E, nu = _requests(1, seed=3)[0]
    srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], n_steps=1, dt=0.01)
    b = (C.c_int64 * 1)(100)
    assert sx.sx_server_set_lanes(srv.h, 2, b) == sx.SX_EORDER
    assert srv.drain(60000.0) == sx.SX_OK
    srv.close()


def _oracle_trajectory(m, E, nu, steps, dt, g, forcing):
    """The oracle's backward-Euler steps (§3 Eqs. 2-3) of one request's
    scene, with the same Newton and PCG options as the server."""
    from oracle import oracle as orc
    T = m["tets"].shape[0]
    Ev = np.full(T, E); nuv = np.full(T, nu)
    snh, mass, bad = orc.snh_scene_inputs(m["X"], m["tets"], Ev, nuv, 1000.0)
    assert bad == 0
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh, pinned=m["pinned"])
    x = m["X"].copy(); v = np.zeros_like(x)
    for _ in range(steps):
        x, v, st, _ = sc.newton_step(x, v, dt, gravity=g, forcing=forcing)
        assert st == 0
    return x, v


@pytest.mark.gpu
def test_served_results_match_oracle_with_forcing_sequence(ctx):
    """Every served request of a staggered mix, run with the forcing-sequence
    PCG tolerance the serving bench uses (§7.2 solver paragraph, as read),
    equals its own alone run bit for bit and the oracle's three steps within
    the Newton-step tolerance: |x - x*| <= 1e-8 max|x* - X| + 1e-12 and the
    same for v scaled by 1/dt (v = (x - x_t)/dt)."""
    from paper_2303_02156_gb300.scene import Scene, Server
    reqs = _requests(6, seed=7)
    steps, dt, g = 3, 0.01, (0.0, 0.0, -9.81)
    alone = []
    for m, E, nu in reqs:
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity(g)
        s.finalize()
        for _ in range(steps):
            s.newton_step(dt, forcing=1)
        alone.append(s.get_state())
        s.close()
    srv = Server(ctx, 8 << 30, forcing=1)
    ids = []
    for k, (m, E, nu) in enumerate(reqs):
        ids.append(srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], gravity=g,
                              n_steps=steps, dt=dt))
        if k == 2:
            time.sleep(0.05)
    assert srv.drain(120000.0) == sx.SX_OK
    done = {c["req_id"]: c for c in srv.poll()}
    worst = 0.0
    for rid, (xa, va), (m, E, nu) in zip(ids, alone, reqs):
        assert done[rid]["status"] == sx.SX_OK and done[rid]["steps"] == steps, done[rid]["error"]
        x, v = srv.result(rid)
        assert np.array_equal(x, xa) and np.array_equal(v, va)
        xo, vo = _oracle_trajectory(m, E, nu, steps, dt, g, True)
        ref = np.abs(xo - m["X"]).max()
        tol = 1e-8 * ref + 1e-12
        dxo = np.abs(x - xo).max()
        worst = max(worst, dxo / ref)
        assert dxo <= tol, (rid, dxo, ref)
        assert np.abs(v - vo).max() <= tol / dt
    srv.close()
    print(f"served vs oracle: worst max|x - x*| / max|x* - X| = {worst:.2e}")


@pytest.mark.gpu
def test_lane_cap_keeps_results_and_serves_everything(ctx):
    """With at most two scenes resident per lane, all requests of a single
    lane are still served, each equal to its alone run bit for bit."""
    from paper_2303_02156_gb300.scene import Scene, Server
    reqs = _requests(5, seed=9)
    steps, dt, g = 2, 0.01, (0.0, 0.0, -9.81)
    alone = []
    for m, E, nu in reqs:
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        s.set_pinned(m["pinned"])
        s.set_gravity(g)
        s.finalize()
        for _ in range(steps):
            s.newton_step(dt)
        alone.append(s.get_state())
        s.close()
    srv = Server(ctx, 8 << 30, lanes=[])
    srv.set_lane_cap(2)
    ids = [srv.submit(m["X"], m["tets"], E, nu, 1000.0, pinned=m["pinned"], gravity=g,
                      n_steps=steps, dt=dt) for m, E, nu in reqs]
    assert srv.drain(120000.0) == sx.SX_OK
    done = {c["req_id"]: c for c in srv.poll()}
    assert srv.stats()["completed"] == 5
    for rid, (xa, va) in zip(ids, alone):
        assert done[rid]["status"] == sx.SX_OK, done[rid]["error"]
        x, v = srv.result(rid)
        assert np.array_equal(x, xa) and np.array_equal(v, va)
    with pytest.raises(sx.SxError):
        srv.set_lane_cap(-1)
    srv.close()
