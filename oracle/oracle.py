"""ctypes wrapper of the FP64 CPU oracle (``sx_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py``. The product (CUDA library and its
binding) never imports this module, and this module imports nothing from
the product package.

Every function mirrors one of the oracle's C entry points; the C source
cites the paper passage each one follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")

LEVEL_E, LEVEL_EG, LEVEL_EGH = 0, 1, 2
ORC_ENOTCONV, ORC_ELINESEARCH = -5, -9


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP over element loops)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    L = C.CDLL(build())
    L.orc_num_threads.restype = C.c_int
    L.orc_set_num_threads.argtypes = [C.c_int]
    L.orc_snh_lame.argtypes = [C.c_int, _dp, _dp, C.c_int, _dp, _dp]
    L.orc_tet_rest.argtypes = [C.c_int, _dp, _ip, _dp, _dp]
    L.orc_tet_rest.restype = C.c_int
    L.orc_lumped_mass.argtypes = [C.c_int, C.c_int, _ip, _dp, _dp, _dp]
    L.orc_snh_element.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                  _dp, _dp, _dp]
    L.orc_snh_dPdF.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp]
    L.orc_snh_element_fproj.argtypes = [_dp, _dp, C.c_double, C.c_double, C.c_double,
                                        _dp, _dp, _dp]
    L.orc_snh_batch.argtypes = [C.c_int, _dp, _ip, _dp, _dp, _dp, _dp, C.c_int,
                                C.c_int, _dp, C.c_void_p, C.c_void_p]
    L.orc_tet_element.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_double, C.c_double,
                                  C.c_void_p, _dp, _dp, _dp]
    L.orc_tet_element.restype = C.c_int
    L.orc_tet_batch.argtypes = [C.c_int, C.c_int, _dp, _ip, _dp, _dp, _dp, _dp, C.c_void_p,
                                C.c_int, C.c_int, _dp, C.c_void_p, C.c_void_p]
    L.orc_tet_batch.restype = C.c_int
    L.orc_tetho_shape.argtypes = [C.c_int, _dp, _dp, _dp]
    L.orc_tetho_element.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_double, C.c_double,
                                    C.c_int, _dp, _dp, _dp]
    L.orc_tetho_element.restype = C.c_int
    L.orc_tetho_batch.argtypes = [C.c_int, C.c_int, _dp, _dp, _ip, C.c_int, _dp, _dp, _dp,
                                  C.c_int, C.c_int, _dp, C.c_void_p, C.c_void_p]
    L.orc_tetho_batch.restype = C.c_int
    L.orc_friction_lag_batch.argtypes = [C.c_int, _dp, _ip, C.c_double, C.c_double, _dp, _dp,
                                         _dp, _dp]
    L.orc_friction_element.argtypes = [_dp, _dp, _dp, C.c_double, _dp, C.c_double, C.c_double,
                                       C.c_double, _dp, _dp, _dp]
    L.orc_friction_batch.argtypes = [C.c_int, _dp, _ip, _dp, _dp, _dp, _dp, C.c_double,
                                     C.c_double, C.c_double, C.c_int, _dp, C.c_void_p,
                                     C.c_void_p]
    L.orc_hinge_element.argtypes = [_dp, _dp, C.c_double, C.c_double, _dp, _dp, _dp]
    L.orc_hinge_batch.argtypes = [C.c_int, _dp, _ip, _dp, _dp, C.c_double, C.c_int,
                                  _dp, C.c_void_p, C.c_void_p]
    L.orc_pt_region.argtypes = [_dp]
    L.orc_pt_region.restype = C.c_int
    L.orc_pt_distance.argtypes = [_dp]
    L.orc_pt_distance.restype = C.c_double
    L.orc_barrier_1d.argtypes = [C.c_double, C.c_double, C.c_double,
                                 C.POINTER(C.c_double), C.POINTER(C.c_double),
                                 C.POINTER(C.c_double)]
    L.orc_barrier_element.argtypes = [_dp, C.c_double, C.c_double, _dp, _dp, _dp]
    L.orc_barrier_element.restype = C.c_int
    L.orc_barrier_batch.argtypes = [C.c_int, _dp, _ip, C.c_double, C.c_double,
                                    C.c_int, C.c_int, _dp, C.c_void_p, C.c_void_p,
                                    C.c_void_p]
    L.orc_barrier_batch.restype = C.c_int
    L.orc_clamp_psd.argtypes = [C.c_int, _dp]
    L.orc_clamp_psd.restype = C.c_int
    L.orc_sym_eigvals.argtypes = [C.c_int, _dp, _dp]
    L.orc_sym_eigvals.restype = C.c_int
    L.orc_bsr_pattern.argtypes = [C.c_int, C.c_int, _ip, _ip, C.c_void_p]
    L.orc_bsr_pattern.restype = C.c_longlong
    L.orc_bsr_slots.argtypes = [C.c_int, _ip, _ip, C.c_int, _ip, _ip, _ip]
    L.orc_assemble_elements.argtypes = [C.c_int, _ip, _ip, _dp, C.c_void_p,
                                        C.c_void_p, C.c_void_p]
    L.orc_inertia.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp, C.c_void_p,
                              C.c_void_p, C.c_void_p]
    L.orc_inertia.restype = C.c_double
    L.orc_pcg.argtypes = [C.c_int, _ip, _ip, _dp, _ip, C.c_void_p, _dp, C.c_double,
                          C.c_int, _dp, C.POINTER(C.c_int), C.POINTER(C.c_double)]
    L.orc_pcg.restype = C.c_int
    L.orc_scene_eval.argtypes = [C.c_void_p, _dp, C.c_void_p, C.c_double, C.c_int,
                                 C.c_int, C.POINTER(C.c_double), C.c_void_p,
                                 C.c_void_p]
    L.orc_scene_eval.restype = C.c_int
    L.orc_newton_step.argtypes = [C.c_void_p, C.c_double, _dp, C.c_void_p, _dp, _dp,
                                  C.c_void_p]
    L.orc_newton_step.restype = C.c_int
    _lib = L
    return L


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_num_threads(n: int) -> None:
    lib().orc_set_num_threads(int(n))


# ---------------------------------------------------------------- SNH
def snh_lame(E, nu, literal=False):
    E = _f64(np.atleast_1d(E)); nu = _f64(np.atleast_1d(nu))
    mu = np.empty_like(E); lam = np.empty_like(E)
    lib().orc_snh_lame(E.size, E, nu, int(literal), mu, lam)
    return mu, lam


def tet_rest(X, tets):
    X = _f64(X); tets = _i32(tets)
    T = tets.shape[0]
    Dminv = np.empty((T, 9)); V = np.empty(T)
    bad = lib().orc_tet_rest(T, X, tets, Dminv, V)
    return Dminv, V, bad


def lumped_mass(N, tets, V, rho):
    tets = _i32(tets); V = _f64(V)
    rho = _f64(np.broadcast_to(rho, V.shape))
    m = np.empty(N)
    lib().orc_lumped_mass(N, tets.shape[0], tets, V, rho, m)
    return m


def snh_element(xe, Dminv, V, mu, lam):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_snh_element(_f64(xe).ravel(), _f64(Dminv).ravel(), float(V), float(mu),
                          float(lam), E, g, H)
    return E[0], g, H.reshape(12, 12)


def snh_dPdF(xe, Dminv, mu, lam):
    """d2psi/dF2 (9x9, vec index 3i+j) of one SNH tet."""
    A = np.zeros(81)
    lib().orc_snh_dPdF(_f64(xe), _f64(Dminv), float(mu), float(lam), A)
    return A.reshape(9, 9)


def snh_element_fproj(xe, Dminv, V, mu, lam):
    """E, g and the element Hessian with d2psi/dF2 clamped to PSD (F-space
    projection)."""
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_snh_element_fproj(_f64(xe), _f64(Dminv), float(V), float(mu), float(lam), E, g, H)
    return E[0], g, H.reshape(12, 12)


def snh_batch(x, tets, Dminv, V, mu, lam, level=LEVEL_EGH, project=False):
    """project: False/0 none, True/1 clamp of the 12x12, 2 clamp of d2psi/dF2."""
    tets = _i32(tets); T = tets.shape[0]
    E = np.empty(T)
    g = np.empty((T, 12)) if level >= 1 else None
    H = np.empty((T, 12, 12)) if level >= 2 else None
    lib().orc_snh_batch(T, _f64(x), tets, _f64(Dminv), _f64(V), _f64(mu), _f64(lam),
                        level, int(project), E, _ptr(g), _ptr(H))
    return E, g, H


# ---------------------------------------------------------------- other models
MODEL_SNH, MODEL_NH, MODEL_STVK, MODEL_COROT, MODEL_ARAP = 0, 1, 2, 3, 4


def tet_element(model, xe, Dminv, V, mu, lam, R=None):
    """E, g, H of one tet of any model; returns (bad, E, g, H), bad = 1 for
    an invalid state (Neo-Hookean J <= 0)."""
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    Rp = None if R is None else _f64(R).ravel()
    bad = lib().orc_tet_element(int(model), _f64(xe).ravel(), _f64(Dminv).ravel(), float(V),
                                float(mu), float(lam), _ptr(Rp), E, g, H)
    return bad, E[0], g, H.reshape(12, 12)


def tet_batch(model, x, tets, Dminv, V, mu, lam, R=None, level=LEVEL_EGH, project=False):
    tets = _i32(tets); T = tets.shape[0]
    E = np.empty(T)
    g = np.empty((T, 12)) if level >= 1 else None
    H = np.empty((T, 12, 12)) if level >= 2 else None
    Rp = None if R is None else _f64(R).reshape(T, 9)
    bad = lib().orc_tet_batch(int(model), T, _f64(x), tets, _f64(Dminv), _f64(V), _f64(mu),
                              _f64(lam), _ptr(Rp), level, int(project), E, _ptr(g), _ptr(H))
    return E, g, H, bad


def deformation_gradients(x, tets, Dminv):
    """F = Ds Dm^-1 per tet (T x 3 x 3), numpy."""
    x = _f64(x).reshape(-1, 3); tets = np.asarray(tets)
    Ds = np.stack([x[tets[:, k]] - x[tets[:, 0]] for k in (1, 2, 3)], axis=2)
    return Ds @ _f64(Dminv).reshape(-1, 3, 3)


def lagged_rotations(x, tets, Dminv):
    """Rotation of the polar decomposition of F per tet (T x 9 row-major),
    by numpy's SVD (library routine): F = U S V^T, R = U V^T, with the
    column of U of the smallest singular value negated when det(U V^T) < 0,
    so R is a rotation (the nearest one to F)."""
    F = deformation_gradients(x, tets, Dminv)
    U, _, Vt = np.linalg.svd(F)
    neg = np.linalg.det(U @ Vt) < 0
    U[neg, :, 2] *= -1
    return (U @ Vt).reshape(-1, 9)


# ---------------------------------------------------------------- high-order tets
def tetho_shape(K, xi):
    N = np.zeros(K); dN = np.zeros(3 * K)
    lib().orc_tetho_shape(int(K), _f64(xi), N, dN)
    return N, dN.reshape(K, 3)


def tetho_element(K, rule, Xe, xe, mu, lam, project=False):
    rule = _f64(rule).reshape(-1, 4)
    n3 = 3 * K
    E = np.zeros(1); g = np.zeros(n3); H = np.zeros(n3 * n3)
    bad = lib().orc_tetho_element(int(K), rule.shape[0], rule, _f64(Xe).ravel(),
                                  _f64(xe).ravel(), float(mu), float(lam), int(project), E, g, H)
    return bad, E[0], g, H.reshape(n3, n3)


def tetho_batch(K, X, x, tets, rule, mu, lam, level=LEVEL_EGH, project=False):
    tets = _i32(tets).reshape(-1, K); T = tets.shape[0]
    rule = _f64(rule).reshape(-1, 4)
    n3 = 3 * K
    E = np.empty(T)
    g = np.empty((T, n3)) if level >= 1 else None
    H = np.empty((T, n3, n3)) if level >= 2 else None
    bad = lib().orc_tetho_batch(int(K), T, _f64(X), _f64(x), tets, rule.shape[0], rule,
                                _f64(mu), _f64(lam), level, int(project), E, _ptr(g), _ptr(H))
    return E, g, H, bad


def tetho_assemble(N, tets, g_e, H_e):
    """Dense assembly (small scenes): sum over elements of their K-node
    gradients and Hessians into the 3N vector and the 3N x 3N matrix."""
    tets = np.asarray(tets)
    K = tets.shape[1]
    g = np.zeros(3 * N)
    H = np.zeros((3 * N, 3 * N)) if H_e is not None else None
    for e in range(tets.shape[0]):
        idx = (3 * tets[e][:, None] + np.arange(3)[None, :]).ravel()
        g[idx] += g_e[e]
        if H is not None:
            H[np.ix_(idx, idx)] += H_e[e]
    return g, H


# ---------------------------------------------------------------- friction
def friction_lag(x, pairs, dhat, kappa):
    """Lagged contact data per pair at state x: closest-point weights beta
    (P x 3), tangent basis T (P x 2 x 3), contact force fn (P), separation
    dxt = p - c (P x 3)."""
    pairs = _i32(pairs).reshape(-1, 4); P = pairs.shape[0]
    beta = np.zeros((P, 3)); T = np.zeros((P, 6)); fn = np.zeros(P); dxt = np.zeros((P, 3))
    lib().orc_friction_lag_batch(P, _f64(x).ravel(), pairs, float(dhat), float(kappa), beta, T,
                                 fn, dxt)
    return {"beta": beta, "T": T.reshape(P, 2, 3), "fn": fn, "dxt": dxt}


def friction_element(xe, beta, T, fn, dxt, mu, yhat, dt):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_friction_element(_f64(xe).ravel(), _f64(beta), _f64(T).ravel(), float(fn),
                               _f64(dxt), float(mu), float(yhat), float(dt), E, g, H)
    return E[0], g, H.reshape(12, 12)


def friction_batch(x, pairs, lag, mu, yhat, dt, level=LEVEL_EGH):
    pairs = _i32(pairs).reshape(-1, 4); P = pairs.shape[0]
    E = np.empty(P)
    g = np.empty((P, 12)) if level >= 1 else None
    H = np.empty((P, 12, 12)) if level >= 2 else None
    lib().orc_friction_batch(P, _f64(x).ravel(), pairs, _f64(lag["beta"]),
                             _f64(lag["T"]).reshape(P, 6), _f64(lag["fn"]), _f64(lag["dxt"]),
                             float(mu), float(yhat), float(dt), level, E, _ptr(g), _ptr(H))
    return E, g, H


# ---------------------------------------------------------------- hinge
def hinge_element(xe, q, c, kb):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    lib().orc_hinge_element(_f64(xe).ravel(), _f64(q), float(c), float(kb), E, g, H)
    return E[0], g, H.reshape(12, 12)


def hinge_batch(x, st, q, c, kb, level=LEVEL_EGH):
    st = _i32(st); S = st.shape[0]
    E = np.empty(S)
    g = np.empty((S, 12)) if level >= 1 else None
    H = np.empty((S, 12, 12)) if level >= 2 else None
    lib().orc_hinge_batch(S, _f64(x), st, _f64(q), _f64(c), float(kb), level, E,
                          _ptr(g), _ptr(H))
    return E, g, H


# ---------------------------------------------------------------- barrier
def pt_region(xe):
    return lib().orc_pt_region(_f64(xe).ravel())


def pt_distance(xe):
    return lib().orc_pt_distance(_f64(xe).ravel())


def barrier_1d(d, dhat, kappa):
    b, b1, b2 = C.c_double(), C.c_double(), C.c_double()
    lib().orc_barrier_1d(float(d), float(dhat), float(kappa), C.byref(b), C.byref(b1),
                         C.byref(b2))
    return b.value, b1.value, b2.value


def barrier_element(xe, dhat, kappa):
    E = np.zeros(1); g = np.zeros(12); H = np.zeros(144)
    st = lib().orc_barrier_element(_f64(xe).ravel(), float(dhat), float(kappa), E, g, H)
    return st, E[0], g, H.reshape(12, 12)


def barrier_batch(x, pairs, dhat, kappa, level=LEVEL_EGH, project=False):
    pairs = _i32(pairs); P = pairs.shape[0]
    E = np.empty(P)
    g = np.empty((P, 12)) if level >= 1 else None
    H = np.empty((P, 12, 12)) if level >= 2 else None
    act = np.empty(P, dtype=np.int32)
    bad = lib().orc_barrier_batch(P, _f64(x), pairs, float(dhat), float(kappa), level,
                                  int(project), E, _ptr(g), _ptr(H), _ptr(act))
    return E, g, H, act, bad


# ---------------------------------------------------------------- clamp
def clamp_psd(H):
    A = _f64(H).copy()
    n = A.shape[0]
    sweeps = lib().orc_clamp_psd(n, A.ravel())
    return A, sweeps


def sym_eigvals(H):
    A = _f64(H)
    lam = np.empty(A.shape[0])
    lib().orc_sym_eigvals(A.shape[0], A.ravel(), lam)
    return np.sort(lam)


# ---------------------------------------------------------------- pattern / assembly
def bsr_pattern(N, conn):
    conn = _i32(conn).reshape(-1, 4)
    rp = np.empty(N + 1, dtype=np.int32)
    nnz = lib().orc_bsr_pattern(N, conn.shape[0], conn, rp, None)
    col = np.empty(int(nnz), dtype=np.int32)
    lib().orc_bsr_pattern(N, conn.shape[0], conn, rp, _ptr(col))
    return rp, col


def bsr_slots(N, rp, col, conn):
    conn = _i32(conn).reshape(-1, 4)
    slots = np.empty((conn.shape[0], 16), dtype=np.int32)
    diag = np.empty(N, dtype=np.int32)
    lib().orc_bsr_slots(N, _i32(rp), _i32(col), conn.shape[0], conn, slots, diag)
    return slots, diag


def assemble_elements(conn, slots, g_e, H_e, grad, vals):
    conn = _i32(conn).reshape(-1, 4)
    lib().orc_assemble_elements(conn.shape[0], conn, _i32(slots), _f64(g_e),
                                _ptr(None if H_e is None else _f64(H_e)),
                                _ptr(grad), _ptr(vals))


def inertia(m, dt, x, xt, diag_slot=None, grad=None, vals=None):
    return lib().orc_inertia(m.size, _f64(m), float(dt), _f64(x), _f64(xt),
                             _ptr(None if diag_slot is None else _i32(diag_slot)),
                             _ptr(grad), _ptr(vals))


def pcg(rp, col, vals, diag_slot, pinned_mask, b, tol, maxit=10000):
    N = rp.size - 1
    x = np.zeros(3 * N)
    it = C.c_int(); rr = C.c_double()
    pm = None if pinned_mask is None else np.ascontiguousarray(pinned_mask, dtype=np.uint8)
    st = lib().orc_pcg(N, _i32(rp), _i32(col), _f64(vals), _i32(diag_slot), _ptr(pm),
                       _f64(b).ravel(), float(tol), int(maxit), x, C.byref(it),
                       C.byref(rr))
    return x, st, it.value, rr.value


# ---------------------------------------------------------------- scene
class _OrcScene(C.Structure):
    _fields_ = [
        ("N", C.c_int), ("mass", C.c_void_p),
        ("n_snh", C.c_int), ("snh_tets", C.c_void_p), ("snh_Dminv", C.c_void_p),
        ("snh_V", C.c_void_p), ("snh_mu", C.c_void_p), ("snh_lam", C.c_void_p),
        ("n_hinge", C.c_int), ("hinge", C.c_void_p), ("hinge_q", C.c_void_p),
        ("hinge_c", C.c_void_p), ("kb", C.c_double),
        ("n_pt", C.c_int), ("pt", C.c_void_p), ("dhat", C.c_double),
        ("kappa", C.c_double), ("pinned", C.c_void_p),
        ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("slots", C.c_void_p),
        ("diag_slot", C.c_void_p), ("nnzb", C.c_longlong),
        ("snh_model", C.c_int), ("snh_R", C.c_void_p),
        ("n_fr", C.c_int), ("fr", C.c_void_p), ("fr_mu", C.c_double),
        ("fr_yhat", C.c_double), ("fr_dhat", C.c_double), ("fr_kappa", C.c_double),
        ("fr_beta", C.c_void_p), ("fr_T", C.c_void_p), ("fr_fn", C.c_void_p),
        ("fr_dxt", C.c_void_p),
    ]


class _OrcOpts(C.Structure):
    _fields_ = [("newton_tol", C.c_double), ("pcg_tol", C.c_double),
                ("max_newton", C.c_int), ("max_pcg", C.c_int),
                ("max_halvings", C.c_int), ("armijo_c", C.c_double),
                ("project", C.c_int), ("forcing", C.c_int)]


class _OrcReport(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int),
                ("pcg_iters_total", C.c_int), ("g0_norm", C.c_double),
                ("g_norm", C.c_double), ("E_final", C.c_double)]


class Scene:
    """A scene for the oracle: DOF count, mass, energy blocks in
    registration order (SNH tets, hinges, point-triangle pairs), pinned
    nodes; the pattern and slot maps are built at construction."""

    def __init__(self, N, mass=None, snh=None, hinge=None, pt=None, pinned=None, fr=None):
        self.N = int(N)
        self._keep = []
        self.R = None
        self.model = MODEL_SNH
        s = _OrcScene()
        s.N = self.N
        self.mass = None if mass is None else _f64(mass)
        s.mass = _ptr(self.mass)
        conns = []
        if snh is not None:
            tets, Dminv, V, mu, lam = (_i32(snh["tets"]), _f64(snh["Dminv"]),
                                       _f64(snh["V"]), _f64(snh["mu"]), _f64(snh["lam"]))
            self._keep += [tets, Dminv, V, mu, lam]
            s.n_snh = tets.shape[0]
            s.snh_tets, s.snh_Dminv, s.snh_V = _ptr(tets), _ptr(Dminv), _ptr(V)
            s.snh_mu, s.snh_lam = _ptr(mu), _ptr(lam)
            s.snh_model = int(snh.get("model", MODEL_SNH))
            self.model = s.snh_model
            self.tets, self.Dminv = tets, Dminv
            self.R = None
            if s.snh_model in (MODEL_COROT, MODEL_ARAP):
                R = snh.get("R")
                self.R = (np.tile(np.eye(3).ravel(), (tets.shape[0], 1)) if R is None
                          else _f64(R).reshape(-1, 9).copy())
                s.snh_R = _ptr(self.R)
            conns.append(tets)
        if hinge is not None:
            st, q, c = _i32(hinge["stencils"]), _f64(hinge["q"]), _f64(hinge["c"])
            self._keep += [st, q, c]
            s.n_hinge = st.shape[0]
            s.hinge, s.hinge_q, s.hinge_c = _ptr(st), _ptr(q), _ptr(c)
            s.kb = float(hinge["kb"])
            conns.append(st)
        if pt is not None:
            pr = _i32(pt["pairs"])
            self._keep.append(pr)
            s.n_pt = pr.shape[0]
            s.pt = _ptr(pr)
            s.dhat, s.kappa = float(pt["dhat"]), float(pt["kappa"])
            conns.append(pr)
        self.fr = None
        if fr is not None:
            pr = _i32(fr["pairs"]).reshape(-1, 4)
            P = pr.shape[0]
            self.fr = {"pairs": pr, "beta": np.zeros((P, 3)), "T": np.zeros((P, 6)),
                       "fn": np.zeros(P), "dxt": np.zeros((P, 3))}
            s.n_fr = P
            s.fr = _ptr(pr)
            s.fr_mu, s.fr_yhat = float(fr["mu"]), float(fr["yhat"])
            s.fr_dhat, s.fr_kappa = float(fr["dhat"]), float(fr["kappa"])
            s.fr_beta, s.fr_T = _ptr(self.fr["beta"]), _ptr(self.fr["T"])
            s.fr_fn, s.fr_dxt = _ptr(self.fr["fn"]), _ptr(self.fr["dxt"])
            conns.append(pr)
        self.pinned_mask = np.zeros(self.N, dtype=np.uint8)
        if pinned is not None and len(pinned):
            self.pinned_mask[np.asarray(pinned)] = 1
        s.pinned = _ptr(self.pinned_mask)
        conn = (np.concatenate(conns, 0) if conns else np.zeros((0, 4), np.int32))
        self.conn = _i32(conn)
        self.row_ptr, self.col = bsr_pattern(self.N, self.conn)
        self.slots, self.diag_slot = bsr_slots(self.N, self.row_ptr, self.col, self.conn)
        s.row_ptr, s.col = _ptr(self.row_ptr), _ptr(self.col)
        s.slots, s.diag_slot = _ptr(self.slots), _ptr(self.diag_slot)
        s.nnzb = self.col.size
        self._s = s

    @property
    def nnzb(self):
        return self.col.size

    def eval(self, x, xt=None, dt=1.0, level=LEVEL_EGH, project=True):
        x = _f64(x).ravel()
        E = C.c_double()
        grad = np.zeros(3 * self.N) if level >= 1 else None
        vals = np.zeros((self.nnzb, 3, 3)) if level >= 2 else None
        xt_ = None if xt is None else _f64(xt).ravel()
        bad = lib().orc_scene_eval(C.byref(self._s), x, _ptr(xt_), float(dt), level,
                                   int(project), C.byref(E), _ptr(grad), _ptr(vals))
        return E.value, grad, vals, bad

    def friction_lag(self, x):
        """Lag the friction block's contact data at the state x (what a
        Newton step does at its start)."""
        f = self.fr
        lib().orc_friction_lag_batch(f["pairs"].shape[0], _f64(x).ravel(), f["pairs"],
                                     self._s.fr_dhat, self._s.fr_kappa, f["beta"], f["T"],
                                     f["fn"], f["dxt"])

    def set_rotations(self, R):
        """Lagged rotations of the tet block (COROT / ARAP), 9 per tet."""
        self.R[:] = _f64(R).reshape(self.R.shape)

    def newton_step(self, x, v, dt, gravity=(0.0, 0.0, -9.81), newton_tol=1e-8,
                    pcg_tol=1e-10, max_newton=100, max_pcg=10000, max_halvings=30,
                    armijo_c=1e-4, project=True, forcing=False):
        """One backward-Euler step. The lagged rotations of a COROT / ARAP
        block are taken at the start-of-step state and held for the step
        (§6.1: rotations constant per time step). forcing: PCG tolerance
        max(pcg_tol, min(1/2, sqrt(|g_k| / |g_0|))) per Newton iteration (the
        §7.2 solver's forcing sequence, as read here)."""
        x = _f64(x).ravel().copy(); v = _f64(v).ravel().copy()
        if self.R is not None:
            self.set_rotations(lagged_rotations(x.reshape(-1, 3), self.tets, self.Dminv))
        o = _OrcOpts(newton_tol, pcg_tol, max_newton, max_pcg, max_halvings, armijo_c,
                     int(project), int(forcing))
        r = _OrcReport()
        st = lib().orc_newton_step(C.byref(self._s), float(dt), _f64(gravity),
                                   C.byref(o), x, v, C.byref(r))
        rep = {k: getattr(r, k) for k, _ in _OrcReport._fields_}
        return x.reshape(-1, 3), v.reshape(-1, 3), st, rep


def tet_scene_inputs(model, X, tets, E, nu, rho=1000.0):
    """Rest precompute of a tet block of any model: the SNH model takes the
    re-parameterized (mu', lambda'), the others the plain Lame pair."""
    d, m, bad = snh_scene_inputs(X, tets, E, nu, rho, literal=(model != MODEL_SNH))
    d["model"] = model
    return d, m, bad


def snh_scene_inputs(X, tets, E, nu, rho=1000.0, literal=False):
    """Oracle-side registration (rest precompute) of an SNH tet block:
    Lame conversion, Dm^-1, volumes, lumped mass."""
    Dminv, V, bad = tet_rest(X, tets)
    mu, lam = snh_lame(E, nu, literal)
    m = lumped_mass(X.shape[0], tets, V, rho)
    return {"tets": tets, "Dminv": Dminv, "V": V, "mu": mu, "lam": lam}, m, bad
