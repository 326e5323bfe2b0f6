"""Seeded synthetic scene generators (inputs only).

This module produces meshes, connectivity, per-element material inputs and
deformed states for the workloads the library is measured on. It holds none
of the method's arithmetic: no Lamé conversion, no rest-shape precompute, no
energy, derivative, projection or assembly. Both the CUDA path and the CPU
oracle read the arrays made here, and every random draw comes from a numpy
PCG64 stream seeded by the caller.

Workloads (stand-ins for the paper's stretched cube / beam scenes, §7.2 and
Table 3, which are not available as data):

* ``kuhn_box``: an ``nx x ny x nz`` grid of cubes, each split into 6 tets
  along the main diagonal (Kuhn/Freudenthal split), rest vertices jittered by
  a seeded uniform amount. The k = 0 layer is the pinned "bottom face".
* ``material_uniform`` / ``material_random``: Young's modulus and Poisson
  ratio per element (uniform, or log-uniform E in [1e4, 1e6] Pa and uniform
  nu in [0.2, 0.45]).
* ``shell_sheet``: a flat quad-split triangle sheet with its interior-edge
  hinge stencils (4 nodes: the edge, then the two opposite vertices) and the
  per-stencil hinge inputs of Bergou et al.'s quadratic bending form (the
  cotangent edge weights ``q`` of the flat rest hinge and the scale
  ``c = 3/(A0+A1)``), which the paper takes as precomputed (§6.3, Eq. 13).
* ``barrier_pairs``: point-triangle contact pairs with the point placed over
  the interior of a triangle at a seeded distance (§6.4, Eq. 15 inputs).
* ``random_box_dims``: grid dimensions for a box with a target tet count and
  a random aspect ratio (batched and served scenes).
* ``mixed_scene``: one scene holding an SNH Kuhn block, a hinge sheet and
  point-triangle pairs as stacked DOF sets (mixed-stencil workload).
* ``batch_boxes``: independent Kuhn boxes with log-uniform tet counts and
  per-scene materials (batched workload).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "rng_for", "kuhn_box", "two_tet", "material_uniform", "material_random",
    "jitter_state", "shell_sheet", "barrier_pairs", "random_box_dims",
    "mixed_scene", "batch_boxes", "GRAVITY",
]

GRAVITY = (0.0, 0.0, -9.81)


def rng_for(seed: int) -> np.random.Generator:
    """Return the PCG64 stream every generator here draws from."""
    return np.random.Generator(np.random.PCG64(int(seed)))


def _node_id(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def _kuhn_offsets():
    """Six corner paths (0,0,0) -> (1,1,1) of the unit cube, one per
    permutation of the axes, each oriented so that its rest volume is
    positive (swap of the two middle vertices where needed)."""
    out = []
    for perm in itertools.permutations(range(3)):
        c = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = c[-1].copy()
            nxt[ax] += 1
            c.append(nxt)
        c = np.stack(c)  # 4 x 3 corner offsets
        d = np.linalg.det((c[1:] - c[0]).T.astype(float))
        if d < 0:
            c = c[[0, 2, 1, 3]]
        out.append(c)
    return np.stack(out)  # 6 x 4 x 3


def kuhn_box(nx: int, ny: int, nz: int, h=1.0, jitter: float = 0.1,
             seed: int = 1, origin=(0.0, 0.0, 0.0)):
    """Grid of ``nx*ny*nz`` cubes of edge ``h`` (scalar or 3-tuple), 6 tets each.

    Node id is ``i + (nx+1)*(j + (ny+1)*k)``. Rest positions are jittered
    per coordinate by U(-jitter*h, +jitter*h) from the PCG64 stream of
    ``seed`` (0.1 keeps every tet positively oriented: the smallest Kuhn
    altitude is h/sqrt(2) and two vertices move at most 0.35 h closer).

    Returns dict with ``X`` (N,3) float64, ``tets`` (T,4) int32 and
    ``pinned`` (the k = 0 layer) int32.
    """
    hv = np.broadcast_to(np.asarray(h, dtype=np.float64), (3,)).copy()
    rng = rng_for(seed)
    ii, jj, kk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1),
                             np.arange(nz + 1), indexing="ij")
    # node order: i fastest, then j, then k
    ii = ii.transpose(2, 1, 0).ravel()
    jj = jj.transpose(2, 1, 0).ravel()
    kk = kk.transpose(2, 1, 0).ravel()
    X = np.stack([ii * hv[0], jj * hv[1], kk * hv[2]], axis=1).astype(np.float64)
    X += np.asarray(origin, dtype=np.float64)
    if jitter > 0.0:
        X += rng.uniform(-1.0, 1.0, size=X.shape) * (jitter * hv)
    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    ci = ci.transpose(2, 1, 0).ravel()
    cj = cj.transpose(2, 1, 0).ravel()
    ck = ck.transpose(2, 1, 0).ravel()
    offs = _kuhn_offsets()  # 6 x 4 x 3
    tets = np.empty((ci.size, 6, 4), dtype=np.int64)
    for p in range(6):
        for v in range(4):
            o = offs[p, v]
            tets[:, p, v] = _node_id(ci + o[0], cj + o[1], ck + o[2], nx, ny)
    tets = tets.reshape(-1, 4).astype(np.int32)
    pinned = np.flatnonzero(kk == 0).astype(np.int32)
    return {"X": X, "tets": tets, "pinned": pinned,
            "dims": (nx, ny, nz), "h": hv}


def two_tet():
    """Two tets sharing a face (5 nodes): the smallest mesh with a shared
    off-diagonal block, for brute-force checks."""
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0],
                  [0.0, 0.0, 1.0], [1.0, 1.0, 1.0]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    # orient the second tet positively
    d = np.linalg.det((X[tets[1, 1:]] - X[tets[1, 0]]).T)
    if d < 0:
        tets[1] = tets[1, [0, 2, 1, 3]]
    return {"X": X, "tets": tets, "pinned": np.array([0], dtype=np.int32)}


def material_uniform(n: int, young: float, poisson: float):
    """Per-element (E, nu) arrays with one value each."""
    return (np.full(n, float(young)), np.full(n, float(poisson)))


def material_random(n: int, seed: int, e_range=(1e4, 1e6), nu_range=(0.2, 0.45)):
    """Per-element E ~ log-uniform(e_range), nu ~ uniform(nu_range)."""
    rng = rng_for(seed)
    lo, hi = np.log(e_range[0]), np.log(e_range[1])
    E = np.exp(rng.uniform(lo, hi, size=n))
    nu = rng.uniform(nu_range[0], nu_range[1], size=n)
    return E, nu


def jitter_state(X: np.ndarray, amp: float, seed: int, fixed=None):
    """A deformed state ``X + U(-amp, amp)`` per coordinate; nodes listed
    in ``fixed`` keep their rest position."""
    rng = rng_for(seed)
    x = X + rng.uniform(-amp, amp, size=X.shape)
    if fixed is not None and len(fixed):
        x[fixed] = X[fixed]
    return x


def _cot2d(u, v):
    """Cotangent of the angle between rows of u and v (planar vectors)."""
    dot = (u * v).sum(axis=1)
    crs = np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
    return dot / crs


def shell_sheet(n: int, length: float = 1.0, z0: float = 0.0,
                noise: float = 0.1, seed: int = 3, node_offset: int = 0):
    """Flat ``n x n`` quad sheet split into ``2 n^2`` triangles.

    Returns the rest vertices ``X`` ((n+1)^2, 3), the deformed vertices ``x``
    (seeded U(-noise*h, noise*h) along z), the triangles, the hinge stencils
    ``(e0, e1, o0, o1)`` of every interior edge (edge e0-e1, o0 opposite in
    the first triangle, o1 in the second), and per stencil the inputs of
    Bergou et al.'s quadratic hinge form: cotangent weights
    ``q = (cot b0 + cot b1, cot a0 + cot a1, -(cot a0 + cot b0),
    -(cot a1 + cot b1))`` (a = angle at e0, b = angle at e1, in the two
    triangles) and ``c = 3 / (A0 + A1)``. Node ids are shifted by
    ``node_offset`` so that the sheet can be stacked after other DOF sets.
    """
    h = length / n
    rng = rng_for(seed)
    g = np.arange(n + 1)
    gi, gj = np.meshgrid(g, g, indexing="xy")  # gi varies fastest
    X = np.stack([gi.ravel() * h, gj.ravel() * h,
                  np.full(gi.size, z0)], axis=1).astype(np.float64)
    x = X.copy()
    x[:, 2] += rng.uniform(-noise * h, noise * h, size=X.shape[0])
    ci, cj = np.meshgrid(np.arange(n), np.arange(n), indexing="xy")
    ci = ci.ravel(); cj = cj.ravel()
    v00 = ci + (n + 1) * cj
    v10 = v00 + 1
    v01 = v00 + (n + 1)
    v11 = v01 + 1
    tris = np.concatenate([np.stack([v00, v10, v11], 1),
                           np.stack([v00, v11, v01], 1)], 0).astype(np.int64)
    # interior edges: match half-edges (a,b) with (b,a)
    nt = tris.shape[0]
    a = tris.ravel()
    b = tris[:, [1, 2, 0]].ravel()
    opp = tris[:, [2, 0, 1]].ravel()
    lo = np.minimum(a, b); hi = np.maximum(a, b)
    key = lo * (X.shape[0]) + hi
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = np.flatnonzero(ks[1:] == ks[:-1])
    h0 = order[same]; h1 = order[same + 1]
    e0 = a[h0]; e1 = b[h0]
    o0 = opp[h0]; o1 = opp[h1]
    P = X[:, :2]
    x0, x1, x2, x3 = P[e0], P[e1], P[o0], P[o1]
    a0 = _cot2d(x1 - x0, x2 - x0); b0 = _cot2d(x0 - x1, x2 - x1)
    a1 = _cot2d(x1 - x0, x3 - x0); b1 = _cot2d(x0 - x1, x3 - x1)
    q = np.stack([b0 + b1, a0 + a1, -(a0 + b0), -(a1 + b1)], axis=1)

    def area(p, r, s):
        return 0.5 * np.abs((r[:, 0] - p[:, 0]) * (s[:, 1] - p[:, 1])
                            - (r[:, 1] - p[:, 1]) * (s[:, 0] - p[:, 0]))
    c = 3.0 / (area(x0, x1, x2) + area(x0, x1, x3))
    stencils = (np.stack([e0, e1, o0, o1], axis=1) + node_offset).astype(np.int32)
    return {"X": X, "x": x, "tris": (tris + node_offset).astype(np.int32),
            "hinges": stencils, "q": q.astype(np.float64), "c": c,
            "h": h, "n_tri": nt}


def barrier_pairs(tri_x: np.ndarray, tris_local: np.ndarray, n_pairs: int,
                  dmin: float, dmax: float, seed: int, tri_node_offset: int,
                  point_node_offset: int, bary_min: float = 0.05):
    """Point-triangle pairs: pair i uses a fresh point node and a triangle
    ``t_i ~ U``; the point sits over barycentric ``beta`` (Dirichlet(1,1,1)
    mapped into ``beta >= bary_min``) at distance ``d_i ~ U(dmin, dmax)``
    along the unit normal of the triangle in the state ``tri_x``.

    ``tris_local`` index ``tri_x``; node ids in the returned pairs are
    shifted by ``tri_node_offset`` (triangle nodes) and
    ``point_node_offset`` (points). Returns dict with ``points`` (P,3),
    ``pairs`` (P,4) int32 as (point, t0, t1, t2) and ``d`` (P,).
    """
    rng = rng_for(seed)
    t = rng.integers(0, tris_local.shape[0], size=n_pairs)
    beta = rng.dirichlet(np.ones(3), size=n_pairs)
    beta = bary_min + (1.0 - 3.0 * bary_min) * beta
    d = rng.uniform(dmin, dmax, size=n_pairs)
    tv = tris_local[t]
    A = tri_x[tv[:, 0]]; B = tri_x[tv[:, 1]]; C = tri_x[tv[:, 2]]
    nrm = np.cross(B - A, C - A)
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    pts = beta[:, :1] * A + beta[:, 1:2] * B + beta[:, 2:] * C + d[:, None] * nrm
    pairs = np.empty((n_pairs, 4), dtype=np.int64)
    pairs[:, 0] = point_node_offset + np.arange(n_pairs)
    pairs[:, 1:] = tv + tri_node_offset
    return {"points": pts, "pairs": pairs.astype(np.int32), "d": d,
            "tri": t, "beta": beta}


def random_box_dims(n_tets_target: float, rng: np.random.Generator,
                    max_aspect: float = 8.0):
    """Integer grid dims (nx, ny, nz) with 6*nx*ny*nz close to the target and
    side ratios drawn log-uniformly so that max/min <= max_aspect."""
    r = np.exp(rng.uniform(0.0, math.log(max_aspect), size=3))
    r /= r.min()
    if r.max() > max_aspect:
        r = 1.0 + (r - 1.0) * (max_aspect - 1.0) / (r.max() - 1.0)
    cells = max(n_tets_target / 6.0, 1.0)
    s = (cells / np.prod(r)) ** (1.0 / 3.0)
    dims = np.maximum(1, np.rint(r * s)).astype(int)
    return tuple(int(v) for v in dims)


def mixed_scene(n_grid: int = 55, n_sheet: int = 1000, n_pairs: int = 4_000_000,
                seed: int = 3, kb: float = 1e-3, dhat: float = 1e-3, kappa: float = 1e4,
                pair_dmax: float = 1e-3):
    """SNH Kuhn block (``n_grid``^3 cubes, h = 1/n_grid, pinned bottom layer),
    a flat ``n_sheet`` x ``n_sheet`` quad sheet 1 m wide above it (hinge
    stencils, z noise 0.1 h_s) and ``n_pairs`` free points, each over its
    own seeded sheet triangle at d ~ U(1e-4, pair_dmax) m (pair_dmax > dhat
    leaves the farther pairs inactive). Nodes are stacked
    block, then sheet, then points.

    Extra lumped masses (not given by the workload; a reading): sheet
    vertices 0.1 kg/m^2 times a third of their incident triangle area,
    points 1 g each. Returns dict with ``X``, ``x`` (the evaluated state: the
    block jittered by U(+-0.02 h)), ``tets``, ``E``, ``nu``, ``hinges``,
    ``q``, ``c``, ``kb``, ``pairs``, ``dhat``, ``kappa``, ``extra_mass``,
    ``pinned`` and the counts.
    """
    m = kuhn_box(n_grid, n_grid, n_grid, h=1.0 / n_grid, seed=seed)
    nt = m["X"].shape[0]
    T = m["tets"].shape[0]
    E, nu = material_random(T, seed)
    xb = jitter_state(m["X"], 0.02 / n_grid, seed + 1)
    sh = shell_sheet(n_sheet, length=1.0, z0=1.5, noise=0.1, seed=seed + 2, node_offset=nt)
    ns = sh["x"].shape[0]
    bp = barrier_pairs(sh["x"], sh["tris"] - nt, n_pairs, 1e-4, pair_dmax, seed=seed + 3,
                       tri_node_offset=nt, point_node_offset=nt + ns)
    X = np.vstack([m["X"], sh["X"], bp["points"]])
    x = np.vstack([xb, sh["x"], bp["points"]])
    extra = np.zeros(X.shape[0])
    extra[nt:nt + ns] = 0.1 * sh["h"] ** 2      # 6 half-cells x h^2/2 / 3 per vertex
    extra[nt + ns:] = 1e-3
    return {"X": X, "x": x, "tets": m["tets"], "E": E, "nu": nu,
            "hinges": sh["hinges"], "q": sh["q"], "c": sh["c"], "kb": kb,
            "pairs": bp["pairs"], "dhat": dhat, "kappa": kappa,
            "extra_mass": extra, "pinned": m["pinned"],
            "n_block_nodes": nt, "n_sheet_nodes": ns, "n_points": n_pairs}


def batch_boxes(n_scenes: int = 512, t_min: float = 1e3, t_max: float = 2e5, seed: int = 4,
                h: float = 0.02):
    """``n_scenes`` independent Kuhn boxes: tet count log-uniform in
    [t_min, t_max], aspect ratio up to 8:1 (``random_box_dims``), edge ``h``,
    per-scene E ~ logU[1e4, 1e6] Pa and nu ~ U[0.2, 0.45]. Returns a list of
    dicts with the ``kuhn_box`` fields plus ``E``, ``nu`` (scalars)."""
    rng = rng_for(seed)
    out = []
    for k in range(n_scenes):
        T = float(np.exp(rng.uniform(np.log(t_min), np.log(t_max))))
        dims = random_box_dims(T, rng)
        m = kuhn_box(*dims, h=h, seed=seed * 100000 + k)
        m["E"] = float(np.exp(rng.uniform(np.log(1e4), np.log(1e6))))
        m["nu"] = float(rng.uniform(0.2, 0.45))
        out.append(m)
    return out


# ------------------------------------------------------------------ high-order tets
_HO_EDGES = ((0, 1), (1, 2), (2, 0), (0, 3), (1, 3), (2, 3))
_HO_FACES = ((0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3))


def kuhn_box_ho(nx: int, ny: int, nz: int, order: int, h=1.0, jitter: float = 0.1,
                seed: int = 1):
    """The Kuhn box of ``kuhn_box`` with quadratic (order 2: 10 nodes) or
    cubic (order 3: 20 nodes) tets: straight-sided elements whose extra
    nodes are shared between neighbours (edge nodes by edge, face nodes by
    face) and placed at the Lagrange positions between the vertices.

    Local node order: the four vertices; order 2: one node per edge in the
    order 01, 12, 20, 03, 13, 23; order 3: two per edge in that order (first
    the one nearer the edge's first vertex), then one per face in the order
    012, 013, 123, 023. Returns dict with ``X`` (N,3), ``tets`` (T,K),
    ``pinned`` (nodes on the k = 0 layer) and ``n_vertices``.
    """
    m = kuhn_box(nx, ny, nz, h=h, jitter=jitter, seed=seed)
    X0, t4 = m["X"], m["tets"].astype(np.int64)
    nv = X0.shape[0]
    pts = [X0]
    count = nv
    K = 10 if order == 2 else 20
    tets = np.empty((t4.shape[0], K), dtype=np.int64)
    tets[:, :4] = t4
    # edges: a sorted vertex pair -> its node id(s) along (lo -> hi)
    keys = np.sort(np.stack([t4[:, list(e)] for e in _HO_EDGES], axis=1), axis=2)   # T x 6 x 2
    flat = keys.reshape(-1, 2)
    uniq, inv = np.unique(flat, axis=0, return_inverse=True)
    inv = inv.reshape(t4.shape[0], 6)
    A, B = X0[uniq[:, 0]], X0[uniq[:, 1]]
    if order == 2:
        pts.append(0.5 * (A + B))
        tets[:, 4:10] = count + inv
        count += uniq.shape[0]
    else:
        pts.append((2.0 * A + B) / 3.0)        # node nearer lo
        pts.append((A + 2.0 * B) / 3.0)        # node nearer hi
        near_lo = count + inv
        near_hi = count + uniq.shape[0] + inv
        count += 2 * uniq.shape[0]
        for e, (i, j) in enumerate(_HO_EDGES):
            first_is_lo = t4[:, i] < t4[:, j]
            tets[:, 4 + 2 * e] = np.where(first_is_lo, near_lo[:, e], near_hi[:, e])
            tets[:, 5 + 2 * e] = np.where(first_is_lo, near_hi[:, e], near_lo[:, e])
        fkeys = np.sort(np.stack([t4[:, list(f)] for f in _HO_FACES], axis=1), axis=2)
        funiq, finv = np.unique(fkeys.reshape(-1, 3), axis=0, return_inverse=True)
        pts.append(X0[funiq].mean(axis=1))
        tets[:, 16:20] = count + finv.reshape(t4.shape[0], 4)
        count += funiq.shape[0]
    X = np.vstack(pts)
    z0 = X0[m["pinned"], 2].max()
    pinned = np.flatnonzero(X[:, 2] <= z0 + 1e-12 * max(abs(z0), 1.0)).astype(np.int32)
    if jitter > 0.0:
        pinned = np.unique(np.concatenate([m["pinned"], pinned[pinned >= nv]]))
        # extra nodes of bottom-face elements: those whose defining vertices are all pinned
        bot = np.zeros(count, dtype=bool)
        bot[m["pinned"]] = True
        for e in range(6):
            i, j = _HO_EDGES[e]
            both = bot[t4[:, i]] & bot[t4[:, j]]
            cols = [4 + e] if order == 2 else [4 + 2 * e, 5 + 2 * e]
            for c in cols:
                bot[tets[both, c]] = True
        if order == 3:
            for f, (i, j, k) in enumerate(_HO_FACES):
                allp = bot[t4[:, i]] & bot[t4[:, j]] & bot[t4[:, k]]
                bot[tets[allp, 16 + f]] = True
        pinned = np.flatnonzero(bot).astype(np.int32)
    return {"X": X, "tets": tets.astype(np.int32), "pinned": pinned, "n_vertices": nv}


def tet_rule_4point():
    """The symmetric 4-point tet rule of degree 2 (reference tet volume 1/6):
    the points are the permutations of the barycentric (a, b, b, b) with
    a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20, weights 1/24. Rows (w, xi)."""
    a = (5.0 + 3.0 * math.sqrt(5.0)) / 20.0
    b = (5.0 - math.sqrt(5.0)) / 20.0
    rows = []
    for k in range(4):
        L = [b, b, b, b]
        L[k] = a
        rows.append([1.0 / 24.0, L[1], L[2], L[3]])
    return np.array(rows)


def tet_rule_conical(n: int):
    """Conical-product (Duffy) rule with n^3 points on the reference tet:
    Gauss-Legendre points on [0, 1] per direction (numpy's leggauss), the
    map xi0 = u, xi1 = v (1 - u), xi2 = w (1 - u)(1 - v) and its Jacobian
    (1 - u)^2 (1 - v) in the weights. Exact for polynomials of degree
    <= 2n - 3 on the tet. Rows (w, xi)."""
    t, wt = np.polynomial.legendre.leggauss(n)
    t = 0.5 * (t + 1.0); wt = 0.5 * wt
    rows = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                u, v, w = t[i], t[j], t[k]
                rows.append([wt[i] * wt[j] * wt[k] * (1 - u) ** 2 * (1 - v),
                             u, v * (1 - u), w * (1 - u) * (1 - v)])
    return np.array(rows)
