"""Thin object wrapper over the C ABI (include/sx.h) for Python callers.

Marshalling only: numpy inputs are passed as host pointers (the library
copies them to the device), element-level outputs land in torch CUDA
tensors, and every computation happens inside libsx.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import sx


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class Context:
    def __init__(self, device: int = 0):
        opt = sx.sx_options()
        opt.device = device
        h = C.c_void_p()
        rc = sx.sx_create(C.byref(h), C.byref(opt))
        if rc != sx.SX_OK:
            raise sx.SxError(rc, "sx_create failed (no CUDA device?)")
        self.h = h

    def check(self, rc):
        return sx.check(self.h, rc)

    def close(self):
        if self.h:
            sx.sx_destroy(self.h)
            self.h = None

    def eval_batch(self, scenes, level=sx.SX_EGH, project=True, precision=sx.SX_FP64,
                   stream=0, want_energy=True):
        arr = (C.c_void_p * len(scenes))(*[s.h.value for s in scenes])
        E = (C.c_double * len(scenes))()
        rc = sx.sx_eval_batch(self.h, arr, len(scenes), level, int(project), precision,
                              E if want_energy else None, stream)
        self.check(rc)
        return np.array(E[:]) if want_energy else None

    def autotune(self, scenes, precision=sx.SX_FP64, stream=0):
        """Pick the fastest launch shape for this batch (sx_autotune)."""
        arr = (C.c_void_p * len(scenes))(*[s.h.value for s in scenes])
        rep = sx.sx_tune_report()
        self.check(sx.sx_autotune(self.h, arr, len(scenes), precision, C.byref(rep), stream))
        return {k: getattr(rep, k) for k, _ in sx.sx_tune_report._fields_}

    def set_launch_shape(self, precision, clamp_threads, elem_blocks_per_sm):
        self.check(sx.sx_set_launch_shape(self.h, precision, clamp_threads, elem_blocks_per_sm))

    def newton_step_batch(self, scenes, dt, stream=0, raise_on_error=True, **opts):
        arr = (C.c_void_p * len(scenes))(*[s.h.value for s in scenes])
        reps = (sx.sx_step_report * len(scenes))()
        o = sx.newton_opts(**opts)
        rc = sx.sx_newton_step_batch(self.h, arr, len(scenes), float(dt), C.byref(o), reps,
                                     stream)
        if raise_on_error:
            self.check(rc)
        return rc, [_rep(r) for r in reps]


def _rep(r):
    return {k: getattr(r, k) for k, _ in sx.sx_step_report._fields_}


class Scene:
    """One scene: a DOF set of n nodes with energy blocks."""

    def __init__(self, ctx: Context, X, stream=0):
        X = _f64(X).reshape(-1, 3)
        self.ctx = ctx
        self.N = X.shape[0]
        self.stream = stream
        h = C.c_void_p()
        ctx.check(sx.sx_scene_create(ctx.h, self.N, X.ctypes.data, 3, stream, C.byref(h)))
        self.h = h
        self.blocks = []

    def close(self):
        if self.h:
            sx.sx_scene_destroy(self.h)
            self.h = None

    def _id(self, rc, eid, kind, n):
        self.ctx.check(rc)
        self.blocks.append((kind, n))
        return eid.value

    def add_snh(self, tets, young, poisson, density=1000.0, literal=False):
        tets = _i32(tets); n = tets.shape[0]
        E = _f64(np.broadcast_to(young, (n,))); nu = _f64(np.broadcast_to(poisson, (n,)))
        eid = C.c_int()
        rc = sx.sx_add_snh_tet4(self.h, tets.ctypes.data, n, E.ctypes.data, nu.ctypes.data,
                                float(density), int(literal), self.stream, C.byref(eid))
        return self._id(rc, eid, sx.SX_KIND_SNH_TET4, n)

    def add_tet(self, model, tets, young, poisson, density=1000.0):
        """Linear tets of density ``model`` (sx.SX_MODEL_*)."""
        tets = _i32(tets); n = tets.shape[0]
        E = _f64(np.broadcast_to(young, (n,))); nu = _f64(np.broadcast_to(poisson, (n,)))
        eid = C.c_int()
        rc = sx.sx_add_tet4(self.h, int(model), tets.ctypes.data, n, E.ctypes.data,
                            nu.ctypes.data, float(density), self.stream, C.byref(eid))
        return self._id(rc, eid, sx.SX_KIND_TET4, n)

    def add_tet_ho(self, order, tets, young, poisson, density, rule):
        """High-order (order 2: 10-node, 3: 20-node) SNH tets with the
        quadrature rule ``rule`` (nq x (w, xi0, xi1, xi2))."""
        K = 10 if order == 2 else 20
        tets = _i32(tets).reshape(-1, K); n = tets.shape[0]
        E = _f64(np.broadcast_to(young, (n,))); nu = _f64(np.broadcast_to(poisson, (n,)))
        rule = _f64(rule).reshape(-1, 4)
        eid = C.c_int()
        rc = sx.sx_add_tet_ho(self.h, int(order), tets.ctypes.data, n, E.ctypes.data,
                              nu.ctypes.data, float(density), rule.ctypes.data, rule.shape[0],
                              self.stream, C.byref(eid))
        self.ctx.check(rc)
        kind, ns = C.c_int(), C.c_int64()
        self.ctx.check(sx.sx_block_info(self.h, eid.value, C.byref(kind), C.byref(ns)))
        self.blocks.append((kind.value, ns.value))
        return eid.value

    def add_friction(self, pairs, mu, yhat, dhat, kappa):
        """Lagged IPC friction on point-triangle pairs (no friction until
        the first lag: update_friction or a Newton step)."""
        pr = _i32(pairs); n = pr.shape[0]
        eid = C.c_int()
        rc = sx.sx_add_pt_friction(self.h, pr.ctypes.data if n else None, n, float(mu),
                                   float(yhat), float(dhat), float(kappa), self.stream,
                                   C.byref(eid))
        return self._id(rc, eid, sx.SX_KIND_PT_FRICTION, n)

    def update_friction(self, dt):
        """Lag the friction blocks at the current state with step dt."""
        self.ctx.check(sx.sx_update_friction(self.h, float(dt), self.stream))

    def friction_lag(self, energy_id):
        n = self.blocks[energy_id][1]
        beta = np.empty((n, 3)); T = np.empty((n, 6)); fn = np.empty(n); dxl = np.empty((n, 3))
        self.ctx.check(sx.sx_get_friction_lag(self.h, energy_id, beta.ctypes.data,
                                              T.ctypes.data, fn.ctypes.data, dxl.ctypes.data,
                                              self.stream))
        return {"beta": beta, "T": T.reshape(n, 2, 3), "fn": fn, "dxt": dxl}

    def update_rotations(self):
        """Lagged rotations of the COROT / ARAP blocks := polar rotations of
        F at the current state."""
        self.ctx.check(sx.sx_update_rotations(self.h, self.stream))

    def rotations(self, energy_id):
        """Lagged rotations of a COROT / ARAP block, n x 3 x 3."""
        n = self.blocks[energy_id][1]
        R = np.empty((n, 9))
        self.ctx.check(sx.sx_get_rotations(self.h, energy_id, R.ctypes.data if n else None,
                                           self.stream))
        return R.reshape(n, 3, 3)

    def set_rotations(self, energy_id, R):
        R = _f64(R).reshape(-1, 9)
        self.ctx.check(sx.sx_set_rotations(self.h, energy_id,
                                           R.ctypes.data if R.shape[0] else None, self.stream))

    def add_hinge(self, stencils, q, c, kb):
        st = _i32(stencils); n = st.shape[0]
        q = _f64(q); c = _f64(c)
        eid = C.c_int()
        rc = sx.sx_add_hinge4(self.h, st.ctypes.data, n, q.ctypes.data, c.ctypes.data,
                              float(kb), self.stream, C.byref(eid))
        return self._id(rc, eid, sx.SX_KIND_HINGE4, n)

    def add_barrier(self, pairs, dhat, kappa):
        pr = _i32(pairs); n = pr.shape[0]
        eid = C.c_int()
        rc = sx.sx_add_pt_barrier(self.h, pr.ctypes.data, n, float(dhat), float(kappa),
                                  self.stream, C.byref(eid))
        return self._id(rc, eid, sx.SX_KIND_PT_BARRIER, n)

    def set_pairs(self, energy_id, pairs):
        """Replace the pairs of a barrier block (the pattern is rebuilt)."""
        pr = _i32(pairs)
        n = pr.shape[0]
        self.ctx.check(sx.sx_set_pairs(self.h, energy_id, pr.ctypes.data if n else None, n,
                                       self.stream))
        kind, _ = self.blocks[energy_id]
        self.blocks[energy_id] = (kind, n)

    def compact_pairs(self, energy_id):
        """Keep only the pairs active at the current state; returns their count."""
        c = C.c_int64()
        self.ctx.check(sx.sx_compact_pairs(self.h, energy_id, C.byref(c), self.stream))
        kind, _ = self.blocks[energy_id]
        self.blocks[energy_id] = (kind, c.value)
        return c.value

    def add_node_mass(self, m):
        m = _f64(m)
        self.ctx.check(sx.sx_add_node_mass(self.h, m.ctypes.data, self.stream))

    def set_pinned(self, nodes):
        nd = _i32(nodes)
        self.ctx.check(sx.sx_set_pinned(self.h, nd.ctypes.data if nd.size else None, nd.size,
                                        self.stream))

    def set_gravity(self, g):
        arr = (C.c_double * 3)(*[float(v) for v in g])
        self.ctx.check(sx.sx_set_gravity(self.h, arr))

    def finalize(self):
        self.ctx.check(sx.sx_finalize(self.h, self.stream))

    def set_state(self, x=None, v=None):
        x = None if x is None else _f64(x)
        v = None if v is None else _f64(v)
        self.ctx.check(sx.sx_set_state(self.h, sx.ptr(x), sx.ptr(v), self.stream))

    def get_state(self):
        x = np.empty((self.N, 3)); v = np.empty((self.N, 3))
        self.ctx.check(sx.sx_get_state(self.h, x.ctypes.data, v.ctypes.data, self.stream))
        return x, v

    def set_inertia(self, dt, x_tilde):
        xt = None if x_tilde is None else _f64(x_tilde)
        self.ctx.check(sx.sx_set_inertia(self.h, float(dt), sx.ptr(xt), self.stream))

    def eval(self, level=sx.SX_EGH, project=True, precision=sx.SX_FP64, check=True):
        E = C.c_double()
        rc = sx.sx_eval(self.h, level, int(project), precision, C.byref(E), self.stream)
        if check:
            self.ctx.check(rc)
            return E.value
        return rc, E.value

    def stats(self):
        c, b, nf = C.c_int(), C.c_int(), C.c_int()
        self.ctx.check(sx.sx_eval_stats(self.h, C.byref(c), C.byref(b), C.byref(nf),
                                        self.stream))
        return {"clamped": c.value, "bad_state": b.value, "nonfinite": nf.value}

    def info(self):
        n, nnz, nst, nb = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int()
        self.ctx.check(sx.sx_scene_info(self.h, C.byref(n), C.byref(nnz), C.byref(nst),
                                        C.byref(nb)))
        return {"n_nodes": n.value, "nnzb": nnz.value, "n_stencils": nst.value,
                "n_blocks": nb.value}

    def bsr(self):
        inf = self.info()
        rp = np.empty(self.N + 1, dtype=np.int32)
        col = np.empty(inf["nnzb"], dtype=np.int32)
        dt = C.c_int()
        self.ctx.check(sx.sx_copy_bsr(self.h, rp.ctypes.data, col.ctypes.data, None,
                                      C.byref(dt), self.stream))
        vals = np.empty((inf["nnzb"], 3, 3),
                        dtype=np.float32 if dt.value == sx.SX_FP32 else np.float64)
        self.ctx.check(sx.sx_copy_bsr(self.h, None, None, vals.ctypes.data, None,
                                      self.stream))
        return rp, col, vals

    def grad(self):
        g = np.empty(3 * self.N)
        self.ctx.check(sx.sx_copy_grad(self.h, g.ctypes.data, self.stream))
        return g

    def eval_elements(self, energy_id, project=True, precision=sx.SX_FP64, want_H=True,
                      want_g=True):
        import torch
        kind, n = self.blocks[energy_id]
        dev = torch.device("cuda")
        E = torch.empty(max(n, 1), dtype=torch.float64, device=dev)
        g = torch.empty((max(n, 1), 12), dtype=torch.float64, device=dev) if want_g else None
        H = torch.empty((max(n, 1), 12, 12), dtype=torch.float64, device=dev) if want_H else None
        sl = torch.empty((max(n, 1), 16), dtype=torch.int32, device=dev)
        torch.cuda.synchronize()
        self.ctx.check(sx.sx_eval_elements(self.h, energy_id, int(project), precision,
                                           sx.ptr(E), sx.ptr(g), sx.ptr(H), sx.ptr(sl),
                                           self.stream))
        torch.cuda.synchronize()
        out = {"E": E[:n].cpu().numpy(), "slots": sl[:n].cpu().numpy()}
        if want_g:
            out["g"] = g[:n].cpu().numpy()
        if want_H:
            out["H"] = H[:n].cpu().numpy()
        return out

    def newton_step(self, dt, raise_on_error=True, **opts):
        o = sx.newton_opts(**opts)
        r = sx.sx_step_report()
        rc = sx.sx_newton_step(self.h, float(dt), C.byref(o), C.byref(r), self.stream)
        if raise_on_error:
            self.ctx.check(rc)
        return rc, _rep(r)

    def advance(self, dt, max_dt_halvings=4, raise_on_error=True, **opts):
        """Advance by dt; failed Newton steps are redone as two half steps
        (sx_advance). Returns (status, report, substeps)."""
        o = sx.newton_opts(**opts)
        r = sx.sx_step_report()
        n = C.c_int()
        rc = sx.sx_advance(self.h, float(dt), C.byref(o), int(max_dt_halvings), C.byref(r),
                           C.byref(n), self.stream)
        if raise_on_error:
            self.ctx.check(rc)
        return rc, _rep(r), n.value

    def nbytes(self):
        b = C.c_int64()
        self.ctx.check(sx.sx_scene_bytes(self.h, C.byref(b)))
        return b.value


class Server:
    """Continuous-batching request loop (include/sx.h serving section)."""

    def __init__(self, ctx: Context, budget_bytes: int, lanes=None, **opts):
        """lanes: None (the default size classes) or the increasing tet-count
        bounds of the lanes (e.g. [] for a single lane)."""
        self.ctx = ctx
        o = sx.newton_opts(**opts)
        h = C.c_void_p()
        ctx.check(sx.sx_server_create(ctx.h, int(budget_bytes), C.byref(o), C.byref(h)))
        self.h = h
        self._keep = {}
        if lanes is not None:
            b = (C.c_int64 * max(len(lanes), 1))(*[int(v) for v in lanes])
            rc = sx.sx_server_set_lanes(self.h, len(lanes) + 1, b if lanes else None)
            if rc != sx.SX_OK:
                raise sx.SxError(rc, "server lanes")

    def set_lane_cap(self, max_resident):
        """At most max_resident scenes resident per lane (0: no limit)."""
        rc = sx.sx_server_set_lane_cap(self.h, int(max_resident))
        if rc != sx.SX_OK:
            raise sx.SxError(rc, "server lane cap")

    def submit(self, X, tets, young, poisson, density=1000.0, pinned=None,
               gravity=(0.0, 0.0, -9.81), n_steps=10, dt=0.01):
        X = _f64(X).reshape(-1, 3); tets = _i32(tets)
        n = tets.shape[0]
        E = _f64(np.broadcast_to(young, (n,))); nu = _f64(np.broadcast_to(poisson, (n,)))
        pn = None if pinned is None else _i32(pinned)
        sp = sx.sx_snh_scene_spec()
        sp.n_nodes = X.shape[0]; sp.X = X.ctypes.data
        sp.n_tets = n; sp.tets = tets.ctypes.data
        sp.young = E.ctypes.data; sp.poisson = nu.ctypes.data
        sp.density = float(density)
        sp.n_pinned = 0 if pn is None else pn.size
        sp.pinned = None if pn is None or pn.size == 0 else pn.ctypes.data
        for i in range(3):
            sp.gravity[i] = float(gravity[i])
        rid = C.c_int64()
        rc = sx.sx_server_submit(self.h, C.byref(sp), int(n_steps), float(dt), C.byref(rid))
        if rc != sx.SX_OK:
            raise sx.SxError(rc, "server submit")
        self._keep[rid.value] = X.shape[0]
        return rid.value

    def poll(self, max_n=1024):
        arr = (sx.sx_completion * max_n)()
        n = C.c_int()
        self.ctx.check(sx.sx_server_poll(self.h, arr, max_n, C.byref(n)))
        return [{k: getattr(arr[i], k) for k, _ in sx.sx_completion._fields_}
                for i in range(n.value)]

    def result(self, req_id):
        N = self._keep.pop(req_id)
        x = np.empty((N, 3)); v = np.empty((N, 3))
        self.ctx.check(sx.sx_server_result(self.h, int(req_id), x.ctypes.data, v.ctypes.data))
        return x, v

    def drain(self, timeout_ms=600000.0):
        return sx.sx_server_drain(self.h, float(timeout_ms))

    def stats(self):
        st = sx.sx_serve_stats()
        self.ctx.check(sx.sx_server_stats(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in sx.sx_serve_stats._fields_}

    def close(self):
        if self.h:
            sx.sx_server_destroy(self.h)
            self.h = None
