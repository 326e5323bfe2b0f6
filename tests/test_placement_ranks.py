"""Whole-scene placement across ranks (one process per GPU; here gloo on CPU,
world size 2): every rank computes the same placement from the scenes'
footprints, steps only its own scenes, and rank 0 gathers the results; the
merged results equal the scenes stepped one by one in a single process. The
step here is the oracle's backward-Euler step (a stand-in on CPU for the
batched GPU step: the routing and gathering are what is under test)."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_02156_gb300 import placement  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_place_by_footprint_balances_and_is_deterministic():
    fp = [50, 10, 40, 30, 30, 20, 5]
    d = placement.place_by_footprint(fp, 2)
    assert d == placement.place_by_footprint(fp, 2)
    loads = [sum(f for f, k in zip(fp, d) if k == r) for r in range(2)]
    assert abs(loads[0] - loads[1]) <= max(fp)
    assert sorted(placement.mine(d, 0) + placement.mine(d, 1)) == list(range(len(fp)))
    assert placement.place_by_footprint(fp, 1) == [0] * len(fp)
    with pytest.raises(ValueError):
        placement.place_by_footprint(fp, 0)


def test_route_stream_sends_each_request_to_the_least_loaded_device():
    d = placement.route_stream([10, 10, 5, 30, 1], 3)
    assert d == [0, 1, 2, 2, 0]


def test_merge_checks_every_scene_once():
    assert placement.merge([{0: "a", 2: "c"}, {1: "b"}], 3) == ["a", "b", "c"]
    with pytest.raises(ValueError):
        placement.merge([{0: "a"}, {0: "b"}], 1)
    with pytest.raises(ValueError):
        placement.merge([{0: "a"}], 2)


def _boxes():
    from paper_2303_02156_gb300 import scenes
    dims = [(2, 2, 2), (3, 2, 2), (2, 2, 1), (3, 3, 2), (2, 1, 1), (4, 2, 2)]
    out = []
    for k, d in enumerate(dims):
        m = scenes.kuhn_box(*d, h=0.1, seed=40 + k)
        out.append((m, 10 ** (4 + 0.4 * k), 0.2 + 0.04 * k))
    return out


def _footprint(m):
    import ctypes as C
    from paper_2303_02156_gb300 import sx
    d = sx.sx_scene_desc()
    d.n_nodes = m["X"].shape[0]; d.n_tets = m["tets"].shape[0]
    d.n_hinges = 0; d.n_pairs = 0; d.nnzb_hint = 0
    b = C.c_int64()
    assert sx.sx_scene_footprint(C.byref(d), C.byref(b)) == sx.SX_OK
    return b.value


def _step(m, E, nu):
    from oracle import oracle as orc
    T = m["tets"].shape[0]
    snh, mass, _ = orc.snh_scene_inputs(m["X"], m["tets"], np.full(T, E), np.full(T, nu), 1000.0)
    sc = orc.Scene(m["X"].shape[0], mass=mass, snh=snh, pinned=m["pinned"])
    x, v, st, _ = sc.newton_step(m["X"], np.zeros_like(m["X"]), 0.01)
    assert st == 0
    return x


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_2303_02156_gb300 import placement as pl
    dist.init_process_group("gloo", rank=rank, world_size=world)
    boxes = _boxes()
    dev = pl.place_by_footprint([_footprint(m) for m, _, _ in boxes], world)
    local = {i: _step(*boxes[i]) for i in pl.mine(dev, rank)}
    parts = [None] * world
    dist.all_gather_object(parts, local)
    if rank == 0:
        merged = pl.merge(parts, len(boxes))
        q.put((dev, [x.tolist() for x in merged]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_place_step_and_gather():
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    dev, merged = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert set(dev) == {0, 1}   # both ranks got scenes
    boxes = _boxes()
    for (m, E, nu), x in zip(boxes, merged):
        assert np.array_equal(np.array(x), _step(m, E, nu))
