"""High-order Lagrange tets (§6.2 Eq. 12; 10- and 20-node SNH
elements with a quadrature sum) through the C ABI against the FP64 oracle:
the assembled energy, gradient and BSR Hessian (the oracle's element
matrices assembled densely), with and without the per-point projection, in
both precisions, on curved meshes; and a backward-Euler step whose result
zeroes the oracle's gradient of the incremental potential.
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


def _rule(order):
    return scenes.tet_rule_4point() if order == 2 else scenes.tet_rule_conical(3)


def _mesh(order, dims=(2, 2, 2), seed=3, curve=0.03):
    m = scenes.kuhn_box_ho(*dims, order, h=0.25, seed=seed)
    X = m["X"].copy()
    nv = m["n_vertices"]
    rng = np.random.default_rng(seed)
    X[nv:] += rng.uniform(-curve, curve, X[nv:].shape) * 0.25   # curved elements
    T = m["tets"].shape[0]
    E, nu = scenes.material_random(T, seed=seed)
    mu, lam = orc.snh_lame(E, nu)
    return m, X, E, nu, mu, lam


def _dense_bsr(rp, col, vals, N):
    H = np.zeros((3 * N, 3 * N))
    for r in range(N):
        for k in range(rp[r], rp[r + 1]):
            H[3 * r:3 * r + 3, 3 * col[k]:3 * col[k] + 3] = vals[k]
    return H


def _gpu(ctx, order, m, X, E, nu, x):
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, X)
    eid = s.add_tet_ho(order, m["tets"], E, nu, 1000.0, _rule(order))
    s.set_pinned(m["pinned"])
    s.finalize()
    s.set_state(x=x)
    return s, eid


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("precision", [sx.SX_FP64, sx.SX_FP32])
@pytest.mark.parametrize("project", [False, True])
def test_high_order_assembly_parity(ctx, order, precision, project):
    m, X, E, nu, mu, lam = _mesh(order)
    x = scenes.jitter_state(X, 0.15 * 0.25, seed=7)
    s, eid = _gpu(ctx, order, m, X, E, nu, x)
    K = m["tets"].shape[1]
    n_el = m["tets"].shape[0]
    kind, ns = C.c_int(), C.c_int64()
    assert sx.sx_block_info(s.h, eid, C.byref(kind), C.byref(ns)) == sx.SX_OK
    assert kind.value == sx.SX_KIND_TET_HO and ns.value == n_el * (10 if order == 2 else 38)
    Eg = s.eval(sx.SX_EGH, project, precision)
    rp, col, vals = s.bsr()
    N = X.shape[0]
    Ee, ge, He, bad = orc.tetho_batch(K, X, x, m["tets"], _rule(order), mu, lam, 2, project)
    assert bad == 0
    go, Ho = orc.tetho_assemble(N, m["tets"], ge, He)
    Hg = _dense_bsr(rp, col, vals.astype(np.float64), N)
    tol = TOL[precision]
    assert abs(Eg - Ee.sum()) <= 1e-10 * abs(Ee.sum())     # energies are FP64 in both forms
    assert np.linalg.norm(s.grad() - go) <= tol * np.linalg.norm(go)
    assert np.linalg.norm(Hg - Ho) <= tol * np.linalg.norm(Ho)
    if project:
        w = np.linalg.eigvalsh(Hg)
        assert w.min() >= -(1e-9 if precision == sx.SX_FP64 else 1e-6) * np.abs(w).max()
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3])
def test_high_order_element_level_outputs_sum_to_the_element(ctx, order):
    """sx_eval_elements reports S sub-stencils per element: their energies
    sum to the element energy; the assembled gradient is the elements'."""
    m, X, E, nu, mu, lam = _mesh(order, dims=(2, 1, 1), seed=4)
    x = scenes.jitter_state(X, 0.1 * 0.25, seed=9)
    s, eid = _gpu(ctx, order, m, X, E, nu, x)
    K = m["tets"].shape[1]
    S = 10 if order == 2 else 38
    out = s.eval_elements(eid, project=False, precision=sx.SX_FP64)
    Ee, ge, He, bad = orc.tetho_batch(K, X, x, m["tets"], _rule(order), mu, lam, 1, False)
    assert bad == 0
    n_el = m["tets"].shape[0]
    Es = out["E"].reshape(n_el, S).sum(1)
    assert np.allclose(Es, Ee, rtol=1e-10, atol=1e-10 * np.abs(Ee).max())
    # the assembled gradient (sub-stencil gradients scattered by the
    # library's own maps) equals the oracle's element gradients assembled
    N = X.shape[0]
    go, _ = orc.tetho_assemble(N, m["tets"], ge, None)
    s.eval(sx.SX_EG, False, sx.SX_FP64)
    assert np.linalg.norm(s.grad() - go) <= 1e-10 * np.linalg.norm(go)
    s.close()


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3])
def test_high_order_newton_step_zeroes_the_oracle_gradient(ctx, order):
    """One backward-Euler step under gravity; at the GPU's result the
    oracle's gradient of the incremental potential (inertia with the lumped
    mass rho V_e / K per node + the elements) vanishes on the free DOFs."""
    from paper_2303_02156_gb300.scene import Scene
    m, X, E, nu, mu, lam = _mesh(order, dims=(2, 2, 3), seed=5, curve=0.0)
    K = m["tets"].shape[1]
    rule = _rule(order)
    s = Scene(ctx, X)
    s.add_tet_ho(order, m["tets"], np.full(len(E), 1e5), np.full(len(E), 0.3), 1000.0, rule)
    s.set_pinned(m["pinned"])
    g_ext = np.array([0.0, 0.0, -9.81])
    s.set_gravity(tuple(g_ext))
    s.finalize()
    dt = 0.01
    rc, r = s.newton_step(dt, newton_tol=1e-9, pcg_tol=1e-12)
    assert rc == sx.SX_OK, r
    x1 = s.get_state()[0]
    assert np.abs(x1 - X).max() > 0
    # oracle side: element volumes by its own shape gradients
    N = X.shape[0]
    mass = np.zeros(N)
    for t in m["tets"]:
        V = 0.0
        for w, *xi in rule:
            _, dN = orc.tetho_shape(K, np.array(xi))
            V += w * np.linalg.det(X[t].T @ dN)
        mass[t] += 1000.0 * V / K
    mu1, lam1 = orc.snh_lame(np.full(len(E), 1e5), np.full(len(E), 0.3))
    Ee, ge, _, bad = orc.tetho_batch(K, X, x1, m["tets"], rule, mu1, lam1, 1, False)
    assert bad == 0
    g_el, _ = orc.tetho_assemble(N, m["tets"], ge, None)
    xt = X + dt * dt * g_ext                     # x_t + dt v + dt^2 g, v = 0
    g = (mass[:, None] * (x1 - xt)).ravel() / dt ** 2 + g_el
    free = np.ones(N, bool); free[m["pinned"]] = False
    gf = g.reshape(N, 3)[free]
    fext = np.linalg.norm((mass[:, None] * g_ext)[free])
    assert np.linalg.norm(gf) <= 1e-7 * fext, (np.linalg.norm(gf), fext)
    assert np.array_equal(x1[m["pinned"]], X[m["pinned"]])
    s.close()


@pytest.mark.gpu
def test_high_order_rejects_bad_input(ctx):
    from paper_2303_02156_gb300.scene import Scene
    m, X, E, nu, mu, lam = _mesh(2, dims=(1, 1, 1))
    s = Scene(ctx, X)
    rule = _rule(2)
    t = m["tets"].copy()
    bad = t.copy(); bad[0, [1, 2]] = bad[0, [2, 1]]; bad[0, [4, 6]] = bad[0, [6, 4]]
    bad[0, [8, 9]] = bad[0, [9, 8]]
    eid = C.c_int()
    rc = sx.sx_add_tet_ho(s.h, 2, bad.ctypes.data, len(bad), E.ctypes.data, nu.ctypes.data,
                          1000.0, rule.ctypes.data, len(rule), None, C.byref(eid))
    assert rc == sx.SX_EDEGENERATE
    rc = sx.sx_add_tet_ho(s.h, 4, t.ctypes.data, len(t), E.ctypes.data, nu.ctypes.data,
                          1000.0, rule.ctypes.data, len(rule), None, C.byref(eid))
    assert rc == sx.SX_EINVAL
    rc = sx.sx_add_tet_ho(s.h, 2, t.ctypes.data, len(t), E.ctypes.data, nu.ctypes.data,
                          1000.0, rule.ctypes.data, 0, None, C.byref(eid))
    assert rc == sx.SX_EINVAL
    s.close()


@pytest.mark.gpu
def test_every_kind_in_one_scene_composes(ctx):
    """One scene holding a quadratic-tet box, a co-rotational linear box and
    a sheet with barrier + friction pairs (the every-kind instantiation):
    its assembled energy, gradient and BSR values equal the sum of the three
    parts evaluated as separate scenes (each part is checked against the
    oracle elsewhere); and a batched Newton step of it equals its single
    step bit for bit."""
    from paper_2303_02156_gb300.scene import Scene
    ho = scenes.kuhn_box_ho(2, 2, 2, 2, h=0.05, seed=11)
    lin = scenes.kuhn_box(2, 2, 2, h=0.05, seed=12, origin=(0.3, 0.0, 0.0))
    sh = scenes.shell_sheet(6, length=0.1, z0=0.3, noise=0.05, seed=13)
    n1, n2, n3 = ho["X"].shape[0], lin["X"].shape[0], sh["X"].shape[0]
    bp = scenes.barrier_pairs(sh["x"], sh["tris"], 40, 1e-4, 9e-4, seed=14,
                              tri_node_offset=n1 + n2, point_node_offset=n1 + n2 + n3)
    X = np.vstack([ho["X"], lin["X"], sh["X"], bp["points"]])
    N = X.shape[0]
    x = scenes.jitter_state(X, 2e-4, seed=15)
    x[n1 + n2:n1 + n2 + n3] = sh["x"]
    x[n1 + n2 + n3:] = bp["points"]
    T1, T2 = ho["tets"].shape[0], lin["tets"].shape[0]
    hinge = sh["hinges"] + n1 + n2

    def build(parts):
        s = Scene(ctx, X)
        if "ho" in parts:
            s.add_tet_ho(2, ho["tets"], np.full(T1, 2e5), np.full(T1, 0.35), 1000.0,
                         scenes.tet_rule_4point())
        if "lin" in parts:
            s.add_tet(sx.SX_MODEL_COROT, lin["tets"] + n1, np.full(T2, 1e5), np.full(T2, 0.3),
                      1000.0)
        if "sheet" in parts:
            s.add_hinge(hinge, sh["q"], sh["c"], 1e-3)
            s.add_barrier(bp["pairs"], 1e-3, 1e4)
            s.add_friction(bp["pairs"], 0.3, 1e-3, 1e-3, 1e4)
            s.add_node_mass(np.concatenate([np.zeros(n1 + n2), np.full(N - n1 - n2, 1e-4)]))
        s.finalize()
        s.set_state(x=x)
        s.update_friction(0.01)
        return s

    full = build(("ho", "lin", "sheet"))
    Ef = full.eval(sx.SX_EGH, True, sx.SX_FP64)
    rp, col, vf = full.bsr()
    gf = full.grad()
    Es, gs = 0.0, np.zeros(3 * N)
    Hs = np.zeros((3 * N, 3 * N))
    for part in ("ho", "lin", "sheet"):
        s = build((part,))
        Es += s.eval(sx.SX_EGH, True, sx.SX_FP64)
        gs += s.grad()
        r2, c2, v2 = s.bsr()
        Hs += _dense_bsr(r2, c2, v2, N)
        s.close()
    Hf = _dense_bsr(rp, col, vf, N)
    assert abs(Ef - Es) <= 1e-12 * abs(Es)
    assert np.linalg.norm(gf - gs) <= 1e-12 * np.linalg.norm(gs)
    assert np.linalg.norm(Hf - Hs) <= 1e-12 * np.linalg.norm(Hs)
    # batched Newton step (with a second scene) equals the single step
    full.set_pinned(np.concatenate([ho["pinned"], lin["pinned"] + n1,
                                    np.arange(n1 + n2, n1 + n2 + n3)]).astype(np.int32))
    full.set_gravity((0.0, 0.0, -9.81))
    other = build(("lin",))
    # its other nodes have neither mass nor elements: pinned
    other.set_pinned(np.concatenate([np.arange(n1), np.arange(n1 + n2, N)]).astype(np.int32))
    other.set_gravity((0.0, 0.0, -9.81))
    v0 = np.zeros_like(x)
    v0[n1 + n2 + n3:, 0] = 0.05
    full.set_state(x=x, v=v0)
    other.set_state(x=x, v=np.zeros_like(x))
    arr = (C.c_void_p * 2)(full.h.value, other.h.value)
    reps = (sx.sx_step_report * 2)()
    o = sx.newton_opts(newton_tol=1e-8, pcg_tol=1e-10)
    assert sx.sx_newton_step_batch(ctx.h, arr, 2, 0.01, C.byref(o), reps, None) == sx.SX_OK, \
        [reps[i].status for i in range(2)]
    xb = full.get_state()[0]
    full.set_state(x=x, v=v0)
    rc, r = full.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10)
    assert rc == sx.SX_OK, r
    assert np.array_equal(full.get_state()[0], xb)
    full.close(); other.close()


@pytest.mark.gpu
def test_empty_blocks_of_the_newer_kinds(ctx):
    """Blocks with no element of every newer kind (another density, lagged
    friction, high-order tets) next to a small linear block: the scene
    evaluates and steps as if they were absent."""
    from paper_2303_02156_gb300.scene import Scene
    m = scenes.kuhn_box(2, 2, 2, h=0.1, seed=21)
    T = m["tets"].shape[0]
    E, nu = np.full(T, 1e5), np.full(T, 0.3)

    def build(with_empty):
        s = Scene(ctx, m["X"])
        s.add_snh(m["tets"], E, nu, 1000.0)
        if with_empty:
            s.add_tet(sx.SX_MODEL_STVK, np.zeros((0, 4), np.int32), np.zeros(0), np.zeros(0))
            s.add_friction(np.zeros((0, 4), np.int32), 0.3, 1e-3, 1e-3, 1e4)
            s.add_tet_ho(2, np.zeros((0, 10), np.int32), np.zeros(0), np.zeros(0), 1000.0,
                         scenes.tet_rule_4point())
        s.set_pinned(m["pinned"])
        s.set_gravity((0.0, 0.0, -9.81))
        s.finalize()
        s.set_state(x=scenes.jitter_state(m["X"], 0.003, seed=3))
        return s

    a, b = build(False), build(True)
    Ea = a.eval(sx.SX_EGH, True, sx.SX_FP64)
    Eb = b.eval(sx.SX_EGH, True, sx.SX_FP64)
    assert Ea == Eb and np.array_equal(a.grad(), b.grad())
    assert np.array_equal(a.bsr()[2], b.bsr()[2])
    for s in (a, b):
        s.set_state(x=m["X"], v=np.zeros_like(m["X"]))
        rc, _ = s.newton_step(0.01, newton_tol=1e-8, pcg_tol=1e-10)
        assert rc == sx.SX_OK
    assert np.array_equal(a.get_state()[0], b.get_state()[0])
    a.close(); b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("order", [2, 3])
def test_single_high_order_element(ctx, order):
    """One element alone (a tile shorter than the others, no neighbour)."""
    m, X, E, nu, mu, lam = _mesh(order, dims=(1, 1, 1), seed=8)
    t = m["tets"][:1]
    used = np.unique(t)
    remap = -np.ones(X.shape[0], np.int64); remap[used] = np.arange(used.size)
    t1 = remap[t].astype(np.int32)
    X1 = X[used]
    x1 = scenes.jitter_state(X1, 0.01, seed=2)
    from paper_2303_02156_gb300.scene import Scene
    s = Scene(ctx, X1)
    s.add_tet_ho(order, t1, E[:1], nu[:1], 1000.0, _rule(order))
    s.finalize()
    s.set_state(x=x1)
    Eg = s.eval(sx.SX_EGH, False, sx.SX_FP64)
    K = t1.shape[1]
    Ee, ge, He, bad = orc.tetho_batch(K, X1, x1, t1, _rule(order), mu[:1], lam[:1], 2, False)
    assert bad == 0
    go, Ho = orc.tetho_assemble(X1.shape[0], t1, ge, He)
    rp, col, vals = s.bsr()
    assert abs(Eg - Ee[0]) <= 1e-10 * abs(Ee[0])
    assert np.linalg.norm(s.grad() - go) <= 1e-10 * np.linalg.norm(go)
    assert np.linalg.norm(_dense_bsr(rp, col, vals, X1.shape[0]) - Ho) <= 1e-10 * np.linalg.norm(Ho)
    s.close()
