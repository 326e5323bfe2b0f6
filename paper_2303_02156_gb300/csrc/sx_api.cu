// sx_api.cu -- the C ABI of include/sx.h: contexts, scenes, registration,
// evaluation, element-level outputs and the batched backward-Euler Newton
// step. Host code only orchestrates; every step of the numerical path runs
// in the kernels of sx_elements.cu, sx_graph.cu, sx_assemble.cu and
// sx_solve.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "sx_internal.cuh"

using namespace sx;

// ------------------------------------------------------------------ helpers
namespace {

struct BlockHost {
    int kind = 0;
    int model = SX_MODEL_SNH;   // tet4 blocks
    double* Rot = nullptr;      // [9][n] lagged rotations (COROT, ARAP)
    int64_t n = 0;
    int64_t base = 0;
    int4* conn = nullptr;
    double* Dminv = nullptr;
    double* V = nullptr;
    double* mu = nullptr;
    double* lam = nullptr;
    double rho = 0.0;
    double* q = nullptr;
    double* c = nullptr;
    double kb = 0.0;
    double dhat = 0.0, kappa = 0.0;
    // friction: lag [13][n] (beta, T, fn, dx_lag), mu, yhat, dt of the lag
    double* flag = nullptr;
    double mu_f = 0.0, yhat = 0.0, dt_f = 1.0;
    // high-order tets (n = ho_n ho_S sub-stencils)
    int ho_K = 0, ho_S = 0, ho_nq = 0;
    int64_t ho_n = 0;
    int* ho_conn = nullptr;
    double* ho_Jinv = nullptr;
    double* ho_wdet = nullptr;
    double* ho_dN = nullptr;
    int* ho_sub = nullptr;
    int* ho_own = nullptr;
    double* ho_modes = nullptr;
    double* ho_rec = nullptr;
    int* ho_flag = nullptr;
    int* ho_pair = nullptr;
    int* ho_gown = nullptr;
    int ho_ept = 1;   // whole elements per element-kernel tile
};

constexpr int kNodeTile = 256;

}  // namespace

struct Batch;

struct ProfRec {
    int phase;
    cudaEvent_t a, b;
};

struct sx_ctx {
    int device = 0;
    int sm_count = 0;
    bool prof_on = false;
    std::vector<ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[SX_PH_COUNT] = {0};
    int64_t prof_launches[SX_PH_COUNT] = {0};
    // occupancy limit of the element kernel [precision][instantiation]
    int elem_occ[2][kElemVariants] = {{1, 1, 1, 1, 1, 1}, {1, 1, 1, 1, 1, 1}};
    bool share_sms = false;
    // launch shapes per precision (sx_autotune / sx_set_launch_shape):
    // projection block size, and element-kernel blocks per SM of the
    // persistent grid (0: one tile per block)
    int clamp_threads[2] = {128, 128};
    int elem_bps[2] = {-1, -1};   // -1: as many as fit; 0: one tile per block
    std::string err;
    // fault injection (sx_inject_alloc_failure): scene allocations left
    // until one fails; 0 = off
    int fail_alloc_in = 0;
    int* queue = nullptr;
    // pinned host staging of per-scene scalars and controls, shared by the
    // batches of this context (a context runs one call at a time); grown on
    // demand, freed with the context
    SceneScal* h_scal = nullptr;
    int* h_ctl_i = nullptr;
    double* h_ctl_d = nullptr;
    int h_cap = 0;
    std::vector<std::unique_ptr<Batch>> batch_cache;
    // projection queue shared by every evaluation of this context (grown on
    // demand; a context runs one evaluation at a time)
    double* clampM = nullptr;
    ClampRef* clampRef = nullptr;
    // two-launch projection scratch (same capacity as the queue)
    float* clampX = nullptr;
    double* clampFro = nullptr;
    int* clampBucket = nullptr;
    int* clampBucketCount = nullptr;
    int* clampCount = nullptr;   // [0] count, [1] failures
    int64_t clamp_cap = 0;
};

struct sx_scene {
    // stream of the latest call on this scene: device memory is allocated
    // and freed in order on it (stream-ordered pool memory)
    cudaStream_t stream = nullptr;
    sx_ctx* ctx = nullptr;
    int64_t N = 0;
    double* X = nullptr;
    double* x = nullptr;
    double* v = nullptr;
    double* x_start = nullptr;
    double* x_tilde = nullptr;
    double* x_trial = nullptr;
    double* dx = nullptr;
    double* mass = nullptr;
    double* extra_mass = nullptr;
    uint8_t* pinned = nullptr;
    double gravity[3] = {0.0, 0.0, 0.0};
    std::vector<BlockHost> blocks;
    bool finalized = false;
    PatternOut pat{};
    double* Ee = nullptr;
    double* ge = nullptr;
    double* He = nullptr;   // 90 doubles per stencil; float staging reuses it
    double* vals64 = nullptr;
    float* vals32 = nullptr;
    // the PCG's sliced-ELLPACK copy of the values (32-row slices)
    int* sell_ptr = nullptr;   // [nslices + 1] steps before each slice
    int* sell_col = nullptr;   // [32 steps]
    double* sell_v64 = nullptr;   // [9 x 32 steps]
    float* sell_v32 = nullptr;
    int64_t sell_steps = 0;
    float* p32 = nullptr;
    double* grad = nullptr;
    double *r = nullptr, *z = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr;
    double* Minv = nullptr;
    SceneScal* sc = nullptr;
    int last_precision = SX_FP64;
    int last_level = -1;
    bool inertia_on = false;
    int inertia_mode = 0;
    double dt = 1.0;
    int64_t nst = 0;
    int64_t bytes = 0;
    uint64_t version = 1;   // bumps whenever the device descriptor changes
    std::vector<void*> allocs;
    // the part of allocs that finalize made (pattern, per-stencil staging,
    // assembled outputs, solver vectors): released when the topology changes
    std::vector<void*> fin_allocs;
    int64_t fin_bytes = 0;
};

// ---------------------------------------------------------------- batches
struct Batch {
    std::vector<sx_scene*> scenes;
    std::vector<uint64_t> versions;
    SceneDev* d_desc = nullptr;
    SceneDev* d_desc_trial = nullptr;
    std::vector<Tile> elem_tiles, node_tiles, slot_tiles, row_tiles;
    Tile* d_elem = nullptr;
    Tile* d_row = nullptr;           // SpMV tiles (spmv_rows_per_tile() rows)
    int* d_row_beg = nullptr;
    int* d_row_end = nullptr;
    double* d_part_row = nullptr;
    Tile* d_node = nullptr;
    Tile* d_slot = nullptr;
    int* d_elem_beg = nullptr;
    int* d_elem_end = nullptr;
    int* d_node_beg = nullptr;
    int* d_node_end = nullptr;
    double* d_part_elem = nullptr;   // 1 per elem tile
    double* d_part_node = nullptr;   // 2 per node tile
    int* d_bad = nullptr;
    int* d_nonfin = nullptr;
    int* d_clamped = nullptr;
    SceneScal* d_scal = nullptr;     // gathered scalars
    SceneScal* h_scal = nullptr;     // pinned host mirror (the context's staging)
    int* d_ctl_i = nullptr;
    double* d_ctl_d = nullptr;
    int* h_ctl_i = nullptr;          // (the context's staging)
    double* h_ctl_d = nullptr;
    // stream of the latest call that used the batch: its memory is freed in
    // order on it (stream-ordered pool memory, no device-wide synchronization)
    cudaStream_t stream = nullptr;
    // per-scene tile ranges of the full node and row lists (host copies)
    std::vector<int> h_nb, h_ne, h_rb, h_re;
    // PCG tile lists compacted to the scenes still iterating (same tiles in
    // the same order per scene, so every per-scene sum is unchanged)
    Tile* d_node_c = nullptr;
    Tile* d_row_c = nullptr;
    int *d_nb_c = nullptr, *d_ne_c = nullptr, *d_rb_c = nullptr, *d_re_c = nullptr;
    int64_t clamp_need = 0;          // projectable stencils of the batch
    int kinds = 0;                   // stencil kinds present (bit mask)
    // the PCG chunk (8 iterations) as an instantiated graph, per precision,
    // with the tolerance and cap it was built with
    cudaGraphExec_t pcg_graph[2] = {nullptr, nullptr};
    double pcg_graph_tol[2] = {0.0, 0.0};
    int pcg_graph_max[2] = {0, 0};
    bool pcg_graph_failed = false;
    ~Batch()
    {
        for (auto& g : pcg_graph)
            if (g) cudaGraphExecDestroy(g);
        for (void* p : {(void*)d_row, (void*)d_row_beg, (void*)d_row_end, (void*)d_part_row,
                        (void*)d_desc, (void*)d_desc_trial, (void*)d_elem, (void*)d_node,
                        (void*)d_slot, (void*)d_elem_beg, (void*)d_elem_end, (void*)d_node_beg,
                        (void*)d_node_end, (void*)d_part_elem, (void*)d_part_node, (void*)d_bad,
                        (void*)d_nonfin, (void*)d_clamped, (void*)d_scal, (void*)d_ctl_i,
                        (void*)d_ctl_d, (void*)d_node_c, (void*)d_row_c, (void*)d_nb_c,
                        (void*)d_ne_c, (void*)d_rb_c, (void*)d_re_c})
            if (p) cudaFreeAsync(p, stream);
    }
};

namespace {

// one projection thread per stencil that can be queued
int clamp_grid_for(int64_t max_queued, int threads)
{
    const int64_t t = threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>((max_queued + t - 1) / t, INT32_MAX));
}

// element-kernel grid for `ntiles` tiles of the given kinds under the
// context's launch shape
int elem_grid(const sx_ctx* ctx, int precision, int kinds, int project, int ntiles)
{
    const int p = precision == SX_FP32 ? 1 : 0;
    const int occ = ctx->elem_occ[p][elements_variant(kinds, project)];
    const int bps = ctx->elem_bps[p] < 0 ? occ : std::min(ctx->elem_bps[p], occ);
    const int g = bps == 0 ? ntiles : std::min<int>(ntiles, ctx->sm_count * bps);
    return std::max(g, 1);
}

// instantiation bits of a block (tets of a density other than SNH add 16)
// units the element kernel's tiles count (stencils) and the tile length:
// a high-order tile holds whole elements (one thread per sub-stencil)
int64_t tile_units(const BlockHost& b) { return b.n; }
int64_t tile_step(const BlockHost& b, int et)
{
    return b.kind == SX_KIND_TET_HO ? (int64_t)b.ho_ept * b.ho_S : et;
}

int kind_bit(const BlockHost& b)
{
    if (b.kind == SX_KIND_SNH_TET4) return b.model == SX_MODEL_SNH ? 1 : 1 | 16;
    if (b.kind == SX_KIND_PT_FRICTION) return 32;
    if (b.kind == SX_KIND_TET_HO) return 64;
    return b.kind == SX_KIND_HINGE4 ? 2 : 4;
}

bool lagged_model(const BlockHost& b)
{
    return b.kind == SX_KIND_SNH_TET4 && (b.model == SX_MODEL_COROT || b.model == SX_MODEL_ARAP);
}

int fail(sx_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int cuda_fail(sx_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, SX_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                         \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);         \
    } while (0)

cudaEvent_t prof_event(sx_ctx* ctx)
{
    if (!ctx->prof_pool.empty()) {
        cudaEvent_t e = ctx->prof_pool.back();
        ctx->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void prof_drain(sx_ctx* ctx)
{
    for (auto& r : ctx->prof_pending) {
        float ms = 0.0f;
        cudaEventSynchronize(r.b);
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) ctx->prof_ms[r.phase] += ms;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
}

// profiled launch: counts `nl` kernel launches in `phase`, and when tracing
// is on brackets the call with events on its stream
#define PL(phase, nl, call)                                                   \
    do {                                                                      \
        cudaEvent_t a_ = nullptr;                                             \
        if (ctx->prof_on) {                                                   \
            a_ = prof_event(ctx);                                             \
            cudaEventRecord(a_, st);                                          \
        }                                                                     \
        CK(call);                                                             \
        ctx->prof_launches[phase] += (nl);                                    \
        if (ctx->prof_on) {                                                   \
            cudaEvent_t b_ = prof_event(ctx);                                 \
            cudaEventRecord(b_, st);                                          \
            ctx->prof_pending.push_back(ProfRec{phase, a_, b_});              \
            if (ctx->prof_pending.size() > 4096) prof_drain(ctx);             \
        }                                                                     \
    } while (0)

// Scene memory comes from the device's stream-ordered pool on the scene's
// current stream: unlike cudaMalloc/cudaFree, neither allocation nor release
// synchronizes the whole device, so contexts serving other requests on other
// streams keep running. The stream is synchronized so that the memory is
// ready for any stream when the call returns.
template <typename T>
int dalloc(sx_scene* s, T** p, size_t count)
{
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (s->ctx && s->ctx->fail_alloc_in > 0 && --s->ctx->fail_alloc_in == 0) {
        *p = nullptr;   // an injected failure: as if the pool were exhausted
        return SX_ENOMEM;
    }
    if (cudaMallocAsync((void**)p, bytes, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return SX_ENOMEM;
    }
    s->allocs.push_back((void*)*p);
    s->bytes += (int64_t)bytes;
    return SX_OK;
}

// allocation that belongs to the finalized topology (see fin_allocs)
template <typename T>
int dalloc_fin(sx_scene* s, T** p, size_t count)
{
    const int64_t before = s->bytes;
    const int rc = dalloc(s, p, count);
    if (rc == SX_OK) {
        s->fin_allocs.push_back((void*)*p);
        s->fin_bytes += s->bytes - before;
    }
    return rc;
}

// frees one scene allocation now (stream-ordered) and forgets it
void free_scene_alloc(sx_scene* s, void* p, int64_t bytes)
{
    auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
    if (it != s->allocs.end()) s->allocs.erase(it);
    cudaFreeAsync(p, s->stream);
    s->bytes -= bytes;
}

SceneDev make_desc(const sx_scene* s, bool trial)
{
    SceneDev d{};
    d.N = s->N;
    d.nst = s->nst;
    d.nnzb = s->pat.nnzb;
    d.nblocks = (int)s->blocks.size();
    d.inertia_on = s->inertia_on ? 1 : 0;
    d.inertia_mode = s->inertia_mode;
    d.dt = s->dt;
    d.inv_dt2 = 1.0 / (s->dt * s->dt);
    for (size_t b = 0; b < s->blocks.size(); ++b) {
        const BlockHost& h = s->blocks[b];
        ElemBlock& e = d.blk[b];
        e.kind = h.kind;
        e.model = h.model;
        e.R = h.Rot;
        e.n = h.n;
        e.base = h.base;
        e.conn = h.conn;
        e.Dminv = h.Dminv;
        e.V = h.V;
        e.mu = h.mu;
        e.lam = h.lam;
        e.q = h.q;
        e.c = h.c;
        e.kb = h.kb;
        e.dhat = h.dhat;
        e.kappa = h.kappa;
        e.flag = h.flag;
        e.mu_f = h.mu_f;
        e.yhat = h.yhat;
        e.dt_f = h.dt_f;
        e.ho_K = h.ho_K;
        e.ho_S = h.ho_S;
        e.ho_nq = h.ho_nq;
        e.ho_n = h.ho_n;
        e.ho_conn = h.ho_conn;
        e.ho_Jinv = h.ho_Jinv;
        e.ho_wdet = h.ho_wdet;
        e.ho_dN = h.ho_dN;
        e.ho_sub = h.ho_sub;
        e.ho_own = h.ho_own;
        e.ho_modes = h.ho_modes;
        e.ho_rec = h.ho_rec;
        e.ho_flag = h.ho_flag;
        e.ho_pair = h.ho_pair;
        e.ho_gown = h.ho_gown;
    }
    d.x = trial ? s->x_trial : s->x;
    d.v = s->v;
    d.x_start = s->x_start;
    d.x_tilde = s->x_tilde;
    d.x_trial = s->x_trial;
    d.dx = s->dx;
    d.mass = s->mass;
    d.pinned = s->pinned;
    d.grad = s->grad;
    d.Ee = s->Ee;
    d.ge = s->ge;
    d.He = s->He;
    d.row_ptr = s->pat.row_ptr;
    d.col = s->pat.col;
    d.diag_slot = s->pat.diag_slot;
    d.slots = s->pat.slots;
    d.slot_ptr = s->pat.slot_ptr;
    d.slot_src = s->pat.slot_src;
    d.slot_order = s->pat.slot_order;
    d.node_ptr = s->pat.node_ptr;
    d.node_src = s->pat.node_src;
    d.vals64 = s->vals64;
    d.vals32 = s->vals32;
    d.sell_ptr = s->sell_ptr;
    d.sell_col = s->sell_col;
    d.sell_v64 = s->sell_v64;
    d.sell_v32 = s->sell_v32;
    d.r = s->r;
    d.z = s->z;
    d.p0 = s->p0;
    d.p1 = s->p1;
    d.p32 = s->p32;
    d.q = s->q;
    d.Minv = s->Minv;
    d.sc = s->sc;
    return d;
}

template <typename T>
int upload(sx_ctx* ctx, T** dptr, const std::vector<T>& v, cudaStream_t st)
{
    if (*dptr) CK(cudaFreeAsync(*dptr, st));
    *dptr = nullptr;
    CK(cudaMallocAsync((void**)dptr, std::max<size_t>(v.size(), 1) * sizeof(T), st));
    if (!v.empty()) CK(cudaMemcpyAsync(*dptr, v.data(), v.size() * sizeof(T),
                                       cudaMemcpyHostToDevice, st));
    return SX_OK;
}

// builds (or refreshes the descriptors of) a batch for `scenes`
int prepare_batch(sx_ctx* ctx, Batch* B, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    std::vector<SceneDev> desc(n), desc_t(n);
    for (int i = 0; i < n; ++i) {
        desc[i] = make_desc(B->scenes[i], false);
        desc_t[i] = make_desc(B->scenes[i], true);
    }
    if (B->d_desc == nullptr) {
        std::vector<int> eb(n), ee(n), nb(n), ne(n), rb(n), re(n);
        const int rt = spmv_rows_per_tile();
        for (int i = 0; i < n; ++i) {
            sx_scene* s = B->scenes[i];
            eb[i] = (int)B->elem_tiles.size();
            const int et = sx::elements_block_threads();
            for (size_t b = 0; b < s->blocks.size(); ++b) {
                const int64_t nu = tile_units(s->blocks[b]), st = tile_step(s->blocks[b], et);
                for (int64_t k = 0; k < nu; k += st)
                    B->elem_tiles.push_back(Tile{i, (int)b, k, (int)std::min<int64_t>(st, nu - k), 0});
            }
            ee[i] = (int)B->elem_tiles.size();
            nb[i] = (int)B->node_tiles.size();
            for (int64_t k = 0; k < s->N; k += kNodeTile)
                B->node_tiles.push_back(
                    Tile{i, 0, k, (int)std::min<int64_t>(kNodeTile, s->N - k), 0});
            ne[i] = (int)B->node_tiles.size();
            rb[i] = (int)B->row_tiles.size();
            for (int64_t k = 0; k < s->N; k += rt)
                B->row_tiles.push_back(Tile{i, 0, k, (int)std::min<int64_t>(rt, s->N - k), 0});
            re[i] = (int)B->row_tiles.size();
            for (int64_t k = 0; k < s->pat.nnzb; k += kSlotTile)
                B->slot_tiles.push_back(
                    Tile{i, 0, k, (int)std::min<int64_t>(kSlotTile, s->pat.nnzb - k), 0});
        }
        int rc;
        if ((rc = upload(ctx, &B->d_elem, B->elem_tiles, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_node, B->node_tiles, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_slot, B->slot_tiles, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_elem_beg, eb, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_elem_end, ee, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_node_beg, nb, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_node_end, ne, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_row, B->row_tiles, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_row_beg, rb, st)) != SX_OK) return rc;
        if ((rc = upload(ctx, &B->d_row_end, re, st)) != SX_OK) return rc;
        B->h_nb = nb;
        B->h_ne = ne;
        B->h_rb = rb;
        B->h_re = re;
        CK(cudaMallocAsync((void**)&B->d_part_row,
                           std::max<size_t>(B->row_tiles.size(), 1) * sizeof(double), st));
        const size_t net = std::max<size_t>(B->elem_tiles.size(), 1);
        const size_t nnt = std::max<size_t>(B->node_tiles.size(), 1);
        CK(cudaMallocAsync((void**)&B->d_part_elem, net * sizeof(double), st));
        CK(cudaMallocAsync((void**)&B->d_part_node, 2 * nnt * sizeof(double), st));
        CK(cudaMallocAsync((void**)&B->d_bad, net * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_nonfin, net * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_clamped, net * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_scal, n * sizeof(SceneScal), st));
        CK(cudaMallocAsync((void**)&B->d_ctl_i, n * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_ctl_d, n * sizeof(double), st));
        int64_t cap = 0;
        B->kinds = 0;
        for (sx_scene* s : B->scenes)
            for (auto& b : s->blocks) {
                // hinges and friction are PSD by construction: never queued
                // (high-order tets project per quadrature point in the element kernel)
                if (b.kind != SX_KIND_HINGE4 && b.kind != SX_KIND_PT_FRICTION &&
                    b.kind != SX_KIND_TET_HO)
                    cap += b.n;
                if (b.n) B->kinds |= kind_bit(b);
            }
        if (!B->kinds) B->kinds = 1;
        B->clamp_need = std::max<int64_t>(cap, 1);
        CK(cudaMallocAsync((void**)&B->d_desc, n * sizeof(SceneDev), st));
        CK(cudaMallocAsync((void**)&B->d_desc_trial, n * sizeof(SceneDev), st));
        B->versions.assign(n, 0);
    }
    // host staging: the context's pinned buffers (grown when a larger batch
    // comes; pinned allocation is the only synchronizing call left, and it
    // happens once per context growth)
    if (ctx->h_cap < n) {
        cudaFreeHost(ctx->h_scal);
        cudaFreeHost(ctx->h_ctl_i);
        cudaFreeHost(ctx->h_ctl_d);
        ctx->h_scal = nullptr;
        ctx->h_ctl_i = nullptr;
        ctx->h_ctl_d = nullptr;
        ctx->h_cap = 0;
        const int cap = std::max(n, 64);
        CK(cudaMallocHost((void**)&ctx->h_scal, cap * sizeof(SceneScal)));
        CK(cudaMallocHost((void**)&ctx->h_ctl_i, cap * sizeof(int)));
        CK(cudaMallocHost((void**)&ctx->h_ctl_d, cap * sizeof(double)));
        ctx->h_cap = cap;
    }
    B->h_scal = ctx->h_scal;
    B->h_ctl_i = ctx->h_ctl_i;
    B->h_ctl_d = ctx->h_ctl_d;
    B->stream = st;
    bool dirty = false;
    for (int i = 0; i < n; ++i) dirty |= B->versions[i] != B->scenes[i]->version;
    if (dirty) {
        CK(cudaMemcpyAsync(B->d_desc, desc.data(), n * sizeof(SceneDev), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(B->d_desc_trial, desc_t.data(), n * sizeof(SceneDev),
                           cudaMemcpyHostToDevice, st));
        // the pageable source vectors must stay valid until the copies ran
        CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) B->versions[i] = B->scenes[i]->version;
    }
    return SX_OK;
}

// Fills the batch's compacted PCG tile lists with the tiles of the scenes
// flagged in `keep` (node and row tiles, and per-scene ranges; other scenes
// get empty ranges). Returns the tile counts through nnt_c, nrt_c.
int compact_pcg_tiles(sx_ctx* ctx, Batch* B, const std::vector<int>& keep, int* nnt_c,
                      int* nrt_c, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    if (!B->d_node_c) {
        CK(cudaMallocAsync((void**)&B->d_node_c, std::max<size_t>(B->node_tiles.size(), 1) * sizeof(Tile), st));
        CK(cudaMallocAsync((void**)&B->d_row_c, std::max<size_t>(B->row_tiles.size(), 1) * sizeof(Tile), st));
        CK(cudaMallocAsync((void**)&B->d_nb_c, n * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_ne_c, n * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_rb_c, n * sizeof(int), st));
        CK(cudaMallocAsync((void**)&B->d_re_c, n * sizeof(int), st));
    }
    std::vector<Tile> nodes, rows;
    std::vector<int> nb(n, 0), ne(n, 0), rb(n, 0), re(n, 0);
    for (int i = 0; i < n; ++i) {
        if (!keep[i]) continue;
        nb[i] = (int)nodes.size();
        nodes.insert(nodes.end(), B->node_tiles.begin() + B->h_nb[i], B->node_tiles.begin() + B->h_ne[i]);
        ne[i] = (int)nodes.size();
        rb[i] = (int)rows.size();
        rows.insert(rows.end(), B->row_tiles.begin() + B->h_rb[i], B->row_tiles.begin() + B->h_re[i]);
        re[i] = (int)rows.size();
    }
    if (!nodes.empty())
        CK(cudaMemcpyAsync(B->d_node_c, nodes.data(), nodes.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
    if (!rows.empty())
        CK(cudaMemcpyAsync(B->d_row_c, rows.data(), rows.size() * sizeof(Tile), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B->d_nb_c, nb.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B->d_ne_c, ne.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B->d_rb_c, rb.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(B->d_re_c, re.data(), n * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));   // the host vectors are pageable
    *nnt_c = (int)nodes.size();
    *nrt_c = (int)rows.size();
    return SX_OK;
}

// grows the context's projection queue to hold `need` stencils
int ensure_clamp_queue(sx_ctx* ctx, int64_t need, cudaStream_t st)
{
    if (need > (int64_t)INT32_MAX) return fail(ctx, SX_EINVAL, "eval: too many projectable stencils");
    if (ctx->clamp_cap >= need && ctx->clampM) return SX_OK;
    for (void* p : {(void*)ctx->clampM, (void*)ctx->clampRef, (void*)ctx->clampX,
                    (void*)ctx->clampFro, (void*)ctx->clampBucket})
        if (p) cudaFreeAsync(p, st);
    ctx->clampM = nullptr;
    ctx->clampRef = nullptr;
    ctx->clampX = nullptr;
    ctx->clampFro = nullptr;
    ctx->clampBucket = nullptr;
    if (!ctx->clampCount) CK(cudaMallocAsync((void**)&ctx->clampCount, 2 * sizeof(int), st));
    if (!ctx->clampBucketCount)
        CK(cudaMallocAsync((void**)&ctx->clampBucketCount, kClampBins * sizeof(int), st));
    if (cudaMallocAsync((void**)&ctx->clampM, (size_t)need * 45 * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&ctx->clampRef, (size_t)need * sizeof(ClampRef), st) != cudaSuccess ||
        cudaMallocAsync((void**)&ctx->clampX, (size_t)need * kClampRec * sizeof(float), st) != cudaSuccess ||
        cudaMallocAsync((void**)&ctx->clampFro, (size_t)need * sizeof(double), st) != cudaSuccess ||
        cudaMallocAsync((void**)&ctx->clampBucket, (size_t)need * kClampBins * sizeof(int), st) != cudaSuccess) {
        cudaGetLastError();
        for (void* p : {(void*)ctx->clampM, (void*)ctx->clampRef, (void*)ctx->clampX,
                        (void*)ctx->clampFro, (void*)ctx->clampBucket})
            if (p) cudaFreeAsync(p, st);
        ctx->clampM = nullptr;
        ctx->clampRef = nullptr;
        ctx->clampX = nullptr;
        ctx->clampFro = nullptr;
        ctx->clampBucket = nullptr;
        ctx->clamp_cap = 0;
        return fail(ctx, SX_ENOMEM, "eval: device allocation failed (projection queue)");
    }
    ctx->clamp_cap = need;
    return SX_OK;
}

Batch* get_batch(sx_ctx* ctx, sx_scene* const* scenes, int n)
{
    for (auto& b : ctx->batch_cache) {
        if ((int)b->scenes.size() != n) continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i) same = b->scenes[i] == scenes[i];
        if (same) return b.get();
    }
    if (ctx->batch_cache.size() >= 8) ctx->batch_cache.erase(ctx->batch_cache.begin());
    auto B = std::make_unique<Batch>();
    B->scenes.assign(scenes, scenes + n);
    ctx->batch_cache.push_back(std::move(B));
    return ctx->batch_cache.back().get();
}

void drop_batches_with(sx_ctx* ctx, sx_scene* s)
{
    auto& v = ctx->batch_cache;
    v.erase(std::remove_if(v.begin(), v.end(),
                           [s](const std::unique_ptr<Batch>& b) {
                               return std::find(b->scenes.begin(), b->scenes.end(), s) !=
                                      b->scenes.end();
                           }),
            v.end());
}

int set_active(sx_ctx* ctx, Batch* B, const std::vector<int>& act, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    for (int i = 0; i < n; ++i) B->h_ctl_i[i] = act[i];
    CK(cudaMemcpyAsync(B->d_ctl_i, B->h_ctl_i, n * sizeof(int), cudaMemcpyHostToDevice, st));
    PL(SX_PH_OTHER, 1, launch_set_scal(B->d_desc, n, B->d_ctl_i, nullptr, nullptr, st));
    return SX_OK;
}

int set_alpha(sx_ctx* ctx, Batch* B, const std::vector<double>& a, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    for (int i = 0; i < n; ++i) B->h_ctl_d[i] = a[i];
    CK(cudaMemcpyAsync(B->d_ctl_d, B->h_ctl_d, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PL(SX_PH_OTHER, 1, launch_set_scal(B->d_desc, n, nullptr, B->d_ctl_d, nullptr, st));
    return SX_OK;
}

int set_pcg_tol(sx_ctx* ctx, Batch* B, const std::vector<double>& t, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    for (int i = 0; i < n; ++i) B->h_ctl_d[i] = t[i];
    CK(cudaMemcpyAsync(B->d_ctl_d, B->h_ctl_d, n * sizeof(double), cudaMemcpyHostToDevice, st));
    PL(SX_PH_OTHER, 1, launch_set_scal(B->d_desc, n, nullptr, nullptr, B->d_ctl_d, st));
    return SX_OK;
}

int read_scal(sx_ctx* ctx, Batch* B, cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    PL(SX_PH_OTHER, 1, launch_gather_scal(B->d_desc, n, B->d_scal, st));
    CK(cudaMemcpyAsync(B->h_scal, B->d_scal, n * sizeof(SceneScal), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SX_OK;
}

// The SpMV's sliced copy of the pattern: slice widths, their prefix sum,
// the padded column array and the (zeroed) FP64 value array.
int build_sell(sx_scene* s, cudaStream_t st)
{
    sx_ctx* ctx = s->ctx;
    const int64_t nsl = (s->N + 31) / 32;
    int* w = nullptr;
    if (dalloc_fin(s, &s->sell_ptr, (size_t)nsl + 1) != SX_OK)
        return fail(ctx, SX_ENOMEM, "finalize: device allocation failed (SpMV layout)");
    CK(cudaMallocAsync((void**)&w, std::max<int64_t>(nsl, 1) * sizeof(int), st));
    CK(launch_sell_widths(s->pat.row_ptr, s->N, w, st));
    std::string err;
    const int rc = scan_counts(w, nsl, s->sell_ptr, st, &err);
    cudaFreeAsync(w, st);
    if (rc != SX_OK) return fail(ctx, rc, err);
    int steps = 0;
    CK(cudaMemcpyAsync(&steps, s->sell_ptr + nsl, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    s->sell_steps = steps;
    if (dalloc_fin(s, &s->sell_col, 32 * (size_t)steps + 32) != SX_OK ||
        dalloc_fin(s, &s->sell_v64, 288 * (size_t)steps + 32) != SX_OK)
        return fail(ctx, SX_ENOMEM, "finalize: device allocation failed (SpMV layout)");
    CK(launch_sell_cols(s->pat.row_ptr, s->pat.col, s->N, s->sell_ptr, s->sell_col, st));
    CK(cudaMemsetAsync(s->sell_v64, 0, (288 * (size_t)steps + 32) * sizeof(double), st));
    return SX_OK;
}

int ensure_vals32(sx_ctx* ctx, sx_scene* s)
{
    if (s->vals32 && s->p32 && s->sell_v32) return SX_OK;
    // each array once (a call that failed part-way leaves the others for the
    // next one)
    if ((!s->vals32 && dalloc_fin(s, &s->vals32, 9 * (size_t)s->pat.nnzb + 16) != SX_OK) ||
        (!s->p32 && dalloc_fin(s, &s->p32, 3 * (size_t)s->N + 4) != SX_OK))
        return fail(ctx, SX_ENOMEM, "eval: device allocation failed (FP32 values)");
    if (!s->sell_v32) {
        if (dalloc_fin(s, &s->sell_v32, 288 * (size_t)s->sell_steps + 64) != SX_OK)
            return fail(ctx, SX_ENOMEM, "eval: device allocation failed (FP32 values)");
        // pad entries (and the lanes past the last row) stay zero
        CK(cudaMemsetAsync(s->sell_v32, 0, (288 * (size_t)s->sell_steps + 64) * sizeof(float),
                           s->stream));
    }
    s->version++;
    return SX_OK;
}

// phase 1 of every high-order block of the batch's scenes (before the
// element kernel, which reads its records)
int launch_ho_points(sx_ctx* ctx, const std::vector<sx_scene*>& scenes, const ElemLaunch& L,
                     cudaStream_t st)
{
    if (!(L.kinds & 64)) return SX_OK;
    for (size_t i = 0; i < scenes.size(); ++i)
        for (size_t b = 0; b < scenes[i]->blocks.size(); ++b) {
            const BlockHost& h = scenes[i]->blocks[b];
            if (h.kind != SX_KIND_TET_HO || h.ho_n == 0) continue;
            PL(SX_PH_ELEMENTS, 1, launch_tetho_points(L, (int)i, (int)b, h.ho_n, h.ho_nq, st));
            PL(SX_PH_ELEMENTS, 1, launch_tetho_blocks(L, (int)i, (int)b, h.ho_n, h.ho_K, h.ho_nq, st));
        }
    return SX_OK;
}

// E / E+g / E+g+H over every active scene of the batch
int run_eval(sx_ctx* ctx, Batch* B, int level, int project, int precision, bool trial,
             cudaStream_t st)
{
    const int n = (int)B->scenes.size();
    const SceneDev* desc = trial ? B->d_desc_trial : B->d_desc;
    ElemLaunch L{};
    L.scenes = desc;
    L.tiles = B->d_elem;
    L.ntiles = (int)B->elem_tiles.size();
    L.level = level;
    L.project = project;
    L.precision = precision;
    L.tile_E = B->d_part_elem;
    L.tile_bad = B->d_bad;
    L.tile_nonfinite = B->d_nonfin;
    L.tile_clamped = B->d_clamped;
    L.queue = ctx->queue;
    if (level >= 2 && project) {
        int rq = ensure_clamp_queue(ctx, B->clamp_need, st);
        if (rq != SX_OK) return rq;
    }
    L.clamp_M = ctx->clampM;
    L.clamp_ref = ctx->clampRef;
    L.clamp_count = ctx->clampCount;
    L.clamp_failed = ctx->clampCount + 1;
    L.clamp_cap = (int)std::min<int64_t>(ctx->clamp_cap, INT32_MAX);
    if (level >= 2 && project) {
        L.clamp_X = ctx->clampX;
        L.clamp_fro = ctx->clampFro;
        L.clamp_bucket = ctx->clampBucket;
        L.clamp_bucket_count = ctx->clampBucketCount;
    }
    const int pidx = precision == SX_FP32 ? 1 : 0;
    L.clamp_threads = ctx->clamp_threads[pidx];
    L.clamp_grid = clamp_grid_for(B->clamp_need, L.clamp_threads);
    L.share_sms = ctx->share_sms;
    L.kinds = B->kinds;
    const int grid = elem_grid(ctx, precision, L.kinds, level >= 2 ? project : 0, L.ntiles);
    int rc = launch_ho_points(ctx, B->scenes, L, st);
    if (rc != SX_OK) return rc;
    PL(SX_PH_ELEMENTS, 1, launch_elements(L, grid, st));
    if (level >= 2 && project) PL(SX_PH_CLAMP, 1, launch_clamp(L, st));
    PL(SX_PH_REDUCE, 1, launch_scene_reduce(B->d_part_elem, 1, 0, B->d_elem_beg, B->d_elem_end,
                                            n, desc, F_E, 0, st));
    PL(SX_PH_REDUCE, 1, launch_scene_reduce_flags(B->d_bad, B->d_nonfin, B->d_clamped,
                                                  B->d_elem_beg, B->d_elem_end, n, desc, st));
    const int nnt = (int)B->node_tiles.size();
    if (level >= 1)
        PL(SX_PH_GRAD, 1, launch_assemble_grad(desc, B->d_node, nnt, B->d_part_node, st));
    else
        PL(SX_PH_GRAD, 1, launch_inertia_energy(desc, B->d_node, nnt, nullptr, B->d_part_node, 0, st));
    PL(SX_PH_REDUCE, 1, launch_scene_reduce(B->d_part_node, 2, 0, B->d_node_beg, B->d_node_end,
                                            n, desc, F_E, 1, st));
    if (level >= 1)
        PL(SX_PH_REDUCE, 1, launch_scene_reduce(B->d_part_node, 2, 1, B->d_node_beg,
                                                B->d_node_end, n, desc, F_GNORM2, 0, st));
    if (level >= 2) {
        AsmLaunch A{desc, B->d_slot, (int)B->slot_tiles.size(), precision};
        PL(SX_PH_ASSEMBLE, 1, launch_assemble_vals(A, st));
        PL(SX_PH_ASSEMBLE, 1, launch_inertia_diag(desc, B->d_node, nnt, precision, st));
        for (sx_scene* s : B->scenes) s->last_precision = precision;
    }
    for (sx_scene* s : B->scenes) s->last_level = std::max(s->last_level, level);
    return SX_OK;
}

int check_scene_ready(sx_scene* s)
{
    if (!s) return SX_EINVAL;
    if (!s->finalized) return fail(s->ctx, SX_EORDER, "scene is not finalized");
    return SX_OK;
}

__global__ void k_set_pinned(const int32_t* nodes, int64_t n, int64_t N, uint8_t* pinned,
                             int* bad)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int v = nodes[i];
    if (v < 0 || v >= N) {
        atomicAdd(bad, 1);
        return;
    }
    pinned[v] = 1;
}

__global__ void k_add_vec(double* dst, const double* src, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] += src[i];
}

__global__ void k_copy_conn(const int32_t* src, int64_t n, int4* dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = make_int4(src[4 * i], src[4 * i + 1], src[4 * i + 2], src[4 * i + 3]);
}

__global__ void k_soa4(const double* src, int64_t n, double* dst)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        for (int a = 0; a < 4; ++a) dst[(int64_t)a * n + i] = src[4 * i + a];
}

// full 12x12 from staged upper blocks is done in the element kernel; this
// kernel copies a block's slot map
int copy_conn(sx_ctx* ctx, sx_scene* s, const int32_t* src, int64_t n, int4** out,
              cudaStream_t st)
{
    if (dalloc(s, out, (size_t)n) != SX_OK) return fail(ctx, SX_ENOMEM, "add: allocation failed");
    int32_t* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, std::max<int64_t>(n, 1) * 4 * sizeof(int32_t), st));
    if (n) CK(cudaMemcpyAsync(tmp, src, n * 4 * sizeof(int32_t), cudaMemcpyDefault, st));
    if (n) k_copy_conn<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp, n, *out);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(tmp, st));
    return SX_OK;
}

int add_block_common(sx_scene* s, const char* what)
{
    if (!s) return SX_EINVAL;
    if ((int)s->blocks.size() >= SX_MAX_BLOCKS)
        return fail(s->ctx, SX_EINVAL, std::string(what) + ": too many energy blocks");
    return SX_OK;
}

void register_block(sx_scene* s, BlockHost&& b, int* energy_id)
{
    b.base = s->nst;
    s->nst += b.n;
    s->blocks.push_back(b);
    s->finalized = false;
    s->version++;
    if (energy_id) *energy_id = (int)s->blocks.size() - 1;
}

}  // namespace

// ==================================================================== ABI
extern "C" {

const char* sx_version(void) { return "libsx 1.0 (sm_103a)"; }

int sx_create(sx_ctx** out, const sx_options* opt)
{
    if (!out) return SX_EINVAL;
    *out = nullptr;
    auto* ctx = new sx_ctx();
    if (opt && opt->device >= 0) {
        cudaError_t e = cudaSetDevice(opt->device);
        if (e != cudaSuccess) {
            delete ctx;
            return SX_ECUDA;
        }
    }
    if (cudaGetDevice(&ctx->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device) !=
            cudaSuccess) {
        delete ctx;
        return SX_ECUDA;
    }
    ctx->share_sms = opt && opt->share_sms;
    for (int p = 0; p < 2; ++p)
        for (int v = 0; v < kElemVariants; ++v) {
            int nb = 1;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, elements_kernel(p, v),
                                                          elements_block_threads(), 0);
            // sharing: the persistent element grid holds one block per SM less
            ctx->elem_occ[p][v] = std::max(ctx->share_sms ? nb - 1 : nb, 1);
        }
    {
        // keep released pool memory mapped and cached for the next
        // stream-ordered allocation (scenes and batches come and go)
        cudaMemPool_t pool = nullptr;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (cudaMalloc((void**)&ctx->queue, sizeof(int)) != cudaSuccess) {
        delete ctx;
        return SX_ENOMEM;
    }
    *out = ctx;
    return SX_OK;
}

int sx_destroy(sx_ctx* ctx)
{
    if (!ctx) return SX_EINVAL;
    prof_drain(ctx);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    ctx->batch_cache.clear();
    cudaFreeHost(ctx->h_scal);
    cudaFreeHost(ctx->h_ctl_i);
    cudaFreeHost(ctx->h_ctl_d);
    cudaFree(ctx->queue);
    cudaFree(ctx->clampM);
    cudaFree(ctx->clampRef);
    cudaFree(ctx->clampCount);
    cudaFree(ctx->clampX);
    cudaFree(ctx->clampFro);
    cudaFree(ctx->clampBucket);
    cudaFree(ctx->clampBucketCount);
    delete ctx;
    return SX_OK;
}

const char* sx_last_error(sx_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int sx_inject_alloc_failure(sx_ctx* ctx, int n)
{
    if (!ctx || n < 0) return SX_EINVAL;
    ctx->fail_alloc_in = n;
    return SX_OK;
}

int sx_scene_create(sx_ctx* ctx, int64_t n_nodes, const double* X_rest, int64_t stride,
                    void* stream, sx_scene** out)
{
    if (!ctx || !out) return SX_EINVAL;
    *out = nullptr;
    if (n_nodes <= 0 || !X_rest || stride < 3)
        return fail(ctx, SX_EINVAL, "scene_create: need n_nodes > 0, X_rest, stride >= 3");
    if (n_nodes >= (int64_t)INT32_MAX / 4)
        return fail(ctx, SX_EINVAL, "scene_create: n_nodes too large for int32 node ids");
    cudaStream_t st = (cudaStream_t)stream;
    auto* s = new sx_scene();
    s->ctx = ctx;
    s->stream = st;
    s->N = n_nodes;
    const size_t n3 = 3 * (size_t)n_nodes;
    int rc = SX_OK;
    rc |= dalloc(s, &s->X, n3);
    rc |= dalloc(s, &s->x, n3);
    rc |= dalloc(s, &s->v, n3);
    rc |= dalloc(s, &s->x_start, n3);
    rc |= dalloc(s, &s->x_tilde, n3);
    rc |= dalloc(s, &s->x_trial, n3);
    rc |= dalloc(s, &s->dx, n3);
    rc |= dalloc(s, &s->mass, (size_t)n_nodes);
    rc |= dalloc(s, &s->extra_mass, (size_t)n_nodes);
    rc |= dalloc(s, &s->pinned, (size_t)n_nodes);
    rc |= dalloc(s, &s->sc, 1);
    if (rc != SX_OK) {
        sx_scene_destroy(s);
        return fail(ctx, SX_ENOMEM, "scene_create: device allocation failed");
    }
    cudaError_t e = cudaMemcpy2DAsync(s->X, 3 * sizeof(double), X_rest, stride * sizeof(double),
                                      3 * sizeof(double), (size_t)n_nodes, cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->x, s->X, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->v, 0, n3 * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->extra_mass, 0, n_nodes * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->pinned, 0, (size_t)n_nodes, st);
    if (e == cudaSuccess) {
        SceneScal init{};
        init.active = 1;
        e = cudaMemcpyAsync(s->sc, &init, sizeof(init), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) {
        sx_scene_destroy(s);
        return cuda_fail(ctx, e, "scene_create");
    }
    *out = s;
    return SX_OK;
}

int sx_scene_destroy(sx_scene* s)
{
    if (!s) return SX_EINVAL;
    if (s->ctx) drop_batches_with(s->ctx, s);
    // the work of the scene's latest stream ends before its memory goes back
    // to the pool; only that stream is waited for, not the device
    cudaStreamSynchronize(s->stream);
    for (void* p : s->allocs) cudaFreeAsync(p, s->stream);
    cudaStreamSynchronize(s->stream);
    delete s;
    return SX_OK;
}

namespace {

__global__ void k_identity_rotations(int64_t n, double* R)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
#pragma unroll
    for (int k = 0; k < 9; ++k) R[(int64_t)k * n + e] = (k % 4 == 0) ? 1.0 : 0.0;
}

// [rows][n] layout -> n records of `rows` values
__global__ void k_rows_to_records(const double* __restrict__ in, int64_t n, int rows,
                                  double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= rows * n) return;
    const int64_t e = i / rows, k = i % rows;
    out[i] = in[k * n + e];
}

// row-major 3x3 per tet (n x 9) <-> the block's [9][n] layout
__global__ void k_rot_transpose(const double* __restrict__ in, int64_t n, int to_soa,
                                double* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= 9 * n) return;
    const int64_t e = i / 9, k = i % 9;
    if (to_soa) out[k * n + e] = in[i];
    else out[i] = in[k * n + e];
}

int add_tet_block(sx_scene* s, int model, const int32_t* tets, int64_t n, const double* young,
                  const double* poisson, double density, int literal_params, void* stream,
                  int* energy_id, const char* what)
{
    int rc = add_block_common(s, what);
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (n < 0 || (n > 0 && (!tets || !young || !poisson)) || !(density >= 0.0))
        return fail(ctx, SX_EINVAL, std::string(what) + ": bad arguments");
    if (model < SX_MODEL_SNH || model > SX_MODEL_ARAP)
        return fail(ctx, SX_EINVAL, std::string(what) + ": unknown model");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    BlockHost b;
    b.kind = SX_KIND_SNH_TET4;
    b.model = model;
    b.n = n;
    b.rho = density;
    if ((rc = copy_conn(ctx, s, tets, n, &b.conn, st)) != SX_OK) return rc;
    if (dalloc(s, &b.Dminv, 9 * (size_t)n) || dalloc(s, &b.V, (size_t)n) ||
        dalloc(s, &b.mu, (size_t)n) || dalloc(s, &b.lam, (size_t)n))
        return fail(ctx, SX_ENOMEM, std::string(what) + ": allocation failed");
    if (lagged_model(b)) {
        if (dalloc(s, &b.Rot, 9 * (size_t)std::max<int64_t>(n, 1)))
            return fail(ctx, SX_ENOMEM, std::string(what) + ": allocation failed");
        if (n) k_identity_rotations<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, b.Rot);
    }
    double *dy = nullptr, *dp = nullptr;
    int* bad = nullptr;
    CK(cudaMallocAsync((void**)&dy, std::max<int64_t>(n, 1) * sizeof(double), st));
    CK(cudaMallocAsync((void**)&dp, std::max<int64_t>(n, 1) * sizeof(double), st));
    CK(cudaMallocAsync((void**)&bad, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
    if (n) {
        CK(cudaMemcpyAsync(dy, young, n * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(dp, poisson, n * sizeof(double), cudaMemcpyDefault, st));
    }
    CK(launch_snh_rest(s->X, s->N, b.conn, n, dy, dp, density,
                       model == SX_MODEL_SNH ? literal_params : 1, b.Dminv, b.V,
                       b.mu, b.lam, bad, st));
    int h_bad2[2] = {0, 0};
    CK(cudaMemcpyAsync(h_bad2, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(dy, st));
    CK(cudaFreeAsync(dp, st));
    CK(cudaFreeAsync(bad, st));
    CK(cudaStreamSynchronize(st));
    if (h_bad2[1])
        return fail(ctx, SX_EINVAL, std::string(what) + ": node id out of range");
    if (h_bad2[0])
        return fail(ctx, SX_EDEGENERATE,
                    std::string(what) + ": " + std::to_string(h_bad2[0]) +
                        " tets with det(Dm) <= 0");
    register_block(s, std::move(b), energy_id);
    return SX_OK;
}

// the lagged-rotation block `energy_id` of a scene, or null
BlockHost* lagged_block(sx_scene* s, int energy_id)
{
    if (!s || energy_id < 0 || energy_id >= (int)s->blocks.size()) return nullptr;
    BlockHost& b = s->blocks[energy_id];
    return lagged_model(b) ? &b : nullptr;
}

// friction lag of every friction block at the current state with step dt
// (a changed dt changes the block descriptors: new scene version)
cudaError_t update_friction(sx_scene* s, double dt, cudaStream_t st)
{
    for (auto& b : s->blocks)
        if (b.kind == SX_KIND_PT_FRICTION) {
            if (b.dt_f != dt) {
                b.dt_f = dt;
                s->version++;
            }
            cudaError_t e = launch_friction_lag(s->x, b.conn, b.n, b.dhat, b.kappa, b.flag, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

// R of every lagged block of the scene at its current state
cudaError_t update_rotations(sx_scene* s, cudaStream_t st)
{
    for (auto& b : s->blocks)
        if (lagged_model(b) && b.n) {
            cudaError_t e = launch_tet_rotations(b.conn, s->x, b.Dminv, b.n, b.Rot, st);
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

}  // namespace

int sx_add_snh_tet4(sx_scene* s, const int32_t* tets, int64_t n, const double* young,
                    const double* poisson, double density, int literal_params, void* stream,
                    int* energy_id)
{
    return add_tet_block(s, SX_MODEL_SNH, tets, n, young, poisson, density, literal_params,
                         stream, energy_id, "add_snh_tet4");
}

int sx_add_tet4(sx_scene* s, int model, const int32_t* tets, int64_t n, const double* young,
                const double* poisson, double density, void* stream, int* energy_id)
{
    return add_tet_block(s, model, tets, n, young, poisson, density, 0, stream, energy_id,
                         "add_tet4");
}

int sx_update_rotations(sx_scene* s, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    CK(update_rotations(s, st));
    return SX_OK;
}

int sx_update_friction(sx_scene* s, double dt, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    if (!(dt > 0.0)) return fail(ctx, SX_EINVAL, "update_friction: dt must be > 0");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    CK(update_friction(s, dt, st));
    return SX_OK;
}

int sx_get_friction_lag(sx_scene* s, int energy_id, double* beta, double* T, double* fn,
                        double* dx_lag, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    if (energy_id < 0 || energy_id >= (int)s->blocks.size() ||
        s->blocks[energy_id].kind != SX_KIND_PT_FRICTION)
        return fail(ctx, SX_EINVAL, "get_friction_lag: not a friction block");
    const BlockHost& b = s->blocks[energy_id];
    cudaStream_t st = (cudaStream_t)stream;
    if (!b.n) return SX_OK;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, 13 * b.n * sizeof(double), st));
    k_rows_to_records<<<(unsigned)((13 * b.n + 255) / 256), 256, 0, st>>>(b.flag, b.n, 13, tmp);
    CK(cudaGetLastError());
    std::vector<double> h(13 * (size_t)b.n);
    CK(cudaMemcpyAsync(h.data(), tmp, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(tmp, st));
    CK(cudaStreamSynchronize(st));
    std::vector<double> ob(3 * (size_t)b.n), oT(6 * (size_t)b.n), of((size_t)b.n),
        od(3 * (size_t)b.n);
    for (int64_t e = 0; e < b.n; ++e) {
        const double* r = h.data() + 13 * e;
        for (int k = 0; k < 3; ++k) ob[3 * e + k] = r[k];
        for (int k = 0; k < 6; ++k) oT[6 * e + k] = r[3 + k];
        of[e] = r[9];
        for (int k = 0; k < 3; ++k) od[3 * e + k] = r[10 + k];
    }
    // stream-ordered copies (no synchronization with other streams)
    if (beta) CK(cudaMemcpyAsync(beta, ob.data(), ob.size() * sizeof(double), cudaMemcpyDefault, st));
    if (T) CK(cudaMemcpyAsync(T, oT.data(), oT.size() * sizeof(double), cudaMemcpyDefault, st));
    if (fn) CK(cudaMemcpyAsync(fn, of.data(), of.size() * sizeof(double), cudaMemcpyDefault, st));
    if (dx_lag)
        CK(cudaMemcpyAsync(dx_lag, od.data(), od.size() * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaStreamSynchronize(st));
    return SX_OK;
}

int sx_get_rotations(sx_scene* s, int energy_id, double* R, void* stream)
{
    BlockHost* b = lagged_block(s, energy_id);
    if (!b || (!R && b->n)) return s ? fail(s->ctx, SX_EINVAL, "get_rotations: not a COROT / ARAP block") : SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    if (!b->n) return SX_OK;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, 9 * b->n * sizeof(double), st));
    k_rot_transpose<<<(unsigned)((9 * b->n + 255) / 256), 256, 0, st>>>(b->Rot, b->n, 0, tmp);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(R, tmp, 9 * b->n * sizeof(double), cudaMemcpyDefault, st));
    CK(cudaFreeAsync(tmp, st));
    CK(cudaStreamSynchronize(st));
    return SX_OK;
}

int sx_set_rotations(sx_scene* s, int energy_id, const double* R, void* stream)
{
    BlockHost* b = lagged_block(s, energy_id);
    if (!b || (!R && b->n)) return s ? fail(s->ctx, SX_EINVAL, "set_rotations: not a COROT / ARAP block") : SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    if (!b->n) return SX_OK;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, 9 * b->n * sizeof(double), st));
    CK(cudaMemcpyAsync(tmp, R, 9 * b->n * sizeof(double), cudaMemcpyDefault, st));
    k_rot_transpose<<<(unsigned)((9 * b->n + 255) / 256), 256, 0, st>>>(tmp, b->n, 1, b->Rot);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(tmp, st));
    return SX_OK;
}

int sx_add_hinge4(sx_scene* s, const int32_t* stencils, int64_t n, const double* q,
                  const double* c, double k_b, void* stream, int* energy_id)
{
    int rc = add_block_common(s, "add_hinge4");
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (n < 0 || (n > 0 && (!stencils || !q || !c)))
        return fail(ctx, SX_EINVAL, "add_hinge4: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    BlockHost b;
    b.kind = SX_KIND_HINGE4;
    b.n = n;
    b.kb = k_b;
    if ((rc = copy_conn(ctx, s, stencils, n, &b.conn, st)) != SX_OK) return rc;
    if (dalloc(s, &b.q, 4 * (size_t)n) || dalloc(s, &b.c, (size_t)n))
        return fail(ctx, SX_ENOMEM, "add_hinge4: allocation failed");
    double* tq = nullptr;
    CK(cudaMallocAsync((void**)&tq, std::max<int64_t>(n, 1) * 4 * sizeof(double), st));
    if (n) {
        CK(cudaMemcpyAsync(tq, q, n * 4 * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(b.c, c, n * sizeof(double), cudaMemcpyDefault, st));
        k_soa4<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tq, n, b.q);
        CK(cudaGetLastError());
    }
    CK(cudaFreeAsync(tq, st));
    CK(cudaStreamSynchronize(st));
    register_block(s, std::move(b), energy_id);
    return SX_OK;
}

int sx_add_pt_barrier(sx_scene* s, const int32_t* pairs, int64_t n, double dhat, double kappa,
                      void* stream, int* energy_id)
{
    int rc = add_block_common(s, "add_pt_barrier");
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (n < 0 || (n > 0 && !pairs) || !(dhat > 0.0) || !(kappa >= 0.0))
        return fail(ctx, SX_EINVAL, "add_pt_barrier: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    BlockHost b;
    b.kind = SX_KIND_PT_BARRIER;
    b.n = n;
    b.dhat = dhat;
    b.kappa = kappa;
    if ((rc = copy_conn(ctx, s, pairs, n, &b.conn, st)) != SX_OK) return rc;
    CK(cudaStreamSynchronize(st));
    register_block(s, std::move(b), energy_id);
    return SX_OK;
}

int sx_add_tet_ho(sx_scene* s, int order, const int32_t* tets, int64_t n, const double* young,
                  const double* poisson, double density, const double* rule, int nq,
                  void* stream, int* energy_id)
{
    int rc = add_block_common(s, "add_tet_ho");
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if ((order != 2 && order != 3) || n < 0 || (n > 0 && (!tets || !young || !poisson)) ||
        !rule || nq < 1 || nq > SX_HO_MAX_QP || !(density >= 0.0))
        return fail(ctx, SX_EINVAL, "add_tet_ho: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    const int K = order == 2 ? 10 : 20;
    std::vector<int> sub, own;
    const int S = tetho_cover(K, sub, own);
    // host copies of the element arrays (host or device input)
    std::vector<int32_t> ht((size_t)n * K);
    std::vector<double> hy((size_t)n), hp((size_t)n);
    if (n) {
        CK(cudaMemcpyAsync(ht.data(), tets, ht.size() * sizeof(int32_t), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(hy.data(), young, n * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaMemcpyAsync(hp.data(), poisson, n * sizeof(double), cudaMemcpyDefault, st));
        CK(cudaStreamSynchronize(st));
    }
    for (int32_t id : ht)
        if (id < 0 || id >= s->N) return fail(ctx, SX_EINVAL, "add_tet_ho: node id out of range");
    BlockHost b;
    b.kind = SX_KIND_TET_HO;
    b.n = n * S;
    b.rho = density;
    b.ho_K = K;
    b.ho_S = S;
    b.ho_nq = nq;
    b.ho_n = n;
    // a tile of whole elements: at most one thread per sub-stencil and one
    // per (element, point)
    b.ho_ept = kHoTileElems;
    // the sub-stencils as 4-node stencils for the pattern and the assembly
    {
        std::vector<int32_t> c4((size_t)n * S * 4);
        for (int64_t e = 0; e < n; ++e)
            for (int j = 0; j < S; ++j)
                for (int a = 0; a < 4; ++a)
                    c4[((size_t)e * S + j) * 4 + a] = ht[(size_t)e * K + sub[4 * j + a]];
        if ((rc = copy_conn(ctx, s, c4.data(), n * S, &b.conn, st)) != SX_OK) return rc;
        CK(cudaStreamSynchronize(st));
    }
    std::vector<int32_t> soa((size_t)n * K);
    for (int64_t e = 0; e < n; ++e)
        for (int a = 0; a < K; ++a) soa[(size_t)a * n + e] = ht[(size_t)e * K + a];
    std::vector<double> hdN((size_t)nq * K * 3), hw(nq);
    for (int q = 0; q < nq; ++q) {
        hw[q] = rule[4 * q];
        tetho_ref_grads(K, rule + 4 * q + 1, hdN.data() + (size_t)q * K * 3);
    }
    // Lame parameters of the SNH density (mu' = 4 mu / 3, lambda' = lambda + 5 mu / 6)
    std::vector<double> hmu((size_t)n), hlam((size_t)n);
    for (int64_t e = 0; e < n; ++e) {
        const double m = hy[e] / (2.0 * (1.0 + hp[e]));
        const double l = hy[e] * hp[e] / ((1.0 + hp[e]) * (1.0 - 2.0 * hp[e]));
        hmu[e] = m * (4.0 / 3.0);
        hlam[e] = l + m * (5.0 / 6.0);
    }
    if (dalloc(s, &b.ho_conn, (size_t)n * K) || dalloc(s, &b.ho_Jinv, (size_t)nq * 9 * n) ||
        dalloc(s, &b.ho_wdet, (size_t)nq * n) || dalloc(s, &b.ho_dN, hdN.size()) ||
        dalloc(s, &b.ho_sub, sub.size()) || dalloc(s, &b.ho_own, own.size()) ||
        dalloc(s, &b.mu, (size_t)n) || dalloc(s, &b.lam, (size_t)n) ||
        dalloc(s, &b.ho_modes, (size_t)n * nq * 91) ||
        dalloc(s, &b.ho_rec, (size_t)n * nq * kHoRec) || dalloc(s, &b.ho_flag, (size_t)n) ||
        dalloc(s, &b.ho_pair, (size_t)3 * K * (K + 1) / 2) || dalloc(s, &b.ho_gown, (size_t)K))
        return fail(ctx, SX_ENOMEM, "add_tet_ho: allocation failed");
    {
        // owned blocks (owner-local node pair, slot j * 10 + ab) and the
        // owner of each node's gradient (j * 4 + local node)
        std::vector<int> pr, gown(K, -1);
        for (int j = 0; j < S; ++j)
            for (int a = 0; a < 4; ++a) {
                if ((own[j] >> (10 + a)) & 1) gown[sub[4 * j + a]] = j * 4 + a;
                for (int c = a; c < 4; ++c) {
                    const int ab = a == 0 ? c : (a == 1 ? 3 + c : (a == 2 ? 5 + c : 9));
                    if ((own[j] >> ab) & 1) {
                        pr.push_back(sub[4 * j + a]);
                        pr.push_back(sub[4 * j + c]);
                        pr.push_back(j * 10 + ab);
                    }
                }
            }
        if ((int)pr.size() != 3 * K * (K + 1) / 2)
            return fail(ctx, SX_EINVAL, "add_tet_ho: sub-stencil cover does not own every pair once");
        CK(cudaMemcpyAsync(b.ho_pair, pr.data(), pr.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b.ho_gown, gown.data(), K * sizeof(int), cudaMemcpyHostToDevice, st));
        CK(cudaMemsetAsync(b.ho_flag, 0, std::max<int64_t>(n, 1) * sizeof(int), st));
        CK(cudaStreamSynchronize(st));
    }
    if (n) {
        CK(cudaMemcpyAsync(b.ho_conn, soa.data(), soa.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b.mu, hmu.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(b.lam, hlam.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    CK(cudaMemcpyAsync(b.ho_dN, hdN.data(), hdN.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.ho_sub, sub.data(), sub.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b.ho_own, own.data(), own.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    double *dw = nullptr, *vol = nullptr;
    int* bad = nullptr;
    CK(cudaMallocAsync((void**)&dw, nq * sizeof(double), st));
    CK(cudaMallocAsync((void**)&vol, std::max<int64_t>(n, 1) * sizeof(double), st));
    CK(cudaMallocAsync((void**)&bad, 2 * sizeof(int), st));
    CK(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
    CK(cudaMemcpyAsync(dw, hw.data(), nq * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(launch_tetho_rest(s->X, s->N, b.ho_conn, n, K, nq, dw, b.ho_dN, b.ho_Jinv, b.ho_wdet, vol,
                         bad, st));
    int hbad[2] = {0, 0};
    std::vector<double> hv((size_t)n);
    CK(cudaMemcpyAsync(hbad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    if (n) CK(cudaMemcpyAsync(hv.data(), vol, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(dw, st));
    CK(cudaFreeAsync(vol, st));
    CK(cudaFreeAsync(bad, st));
    CK(cudaStreamSynchronize(st));
    if (hbad[1]) return fail(ctx, SX_EINVAL, "add_tet_ho: node id out of range");
    if (hbad[0])
        return fail(ctx, SX_EDEGENERATE, "add_tet_ho: " + std::to_string(hbad[0]) +
                                              " elements with det J0 <= 0 at a point");
    // lumped mass rho V_e / K per node, in element order, into the extra mass
    if (n && density > 0.0) {
        std::vector<double> m((size_t)s->N, 0.0);
        for (int64_t e = 0; e < n; ++e)
            for (int a = 0; a < K; ++a) m[ht[(size_t)e * K + a]] += density * hv[e] / K;
        double* tmp = nullptr;
        CK(cudaMallocAsync((void**)&tmp, s->N * sizeof(double), st));
        CK(cudaMemcpyAsync(tmp, m.data(), s->N * sizeof(double), cudaMemcpyHostToDevice, st));
        k_add_vec<<<(unsigned)((s->N + 255) / 256), 256, 0, st>>>(s->extra_mass, tmp, s->N);
        if (s->finalized)
            k_add_vec<<<(unsigned)((s->N + 255) / 256), 256, 0, st>>>(s->mass, tmp, s->N);
        CK(cudaGetLastError());
        CK(cudaFreeAsync(tmp, st));
        CK(cudaStreamSynchronize(st));
    }
    register_block(s, std::move(b), energy_id);
    return SX_OK;
}

int sx_add_pt_friction(sx_scene* s, const int32_t* pairs, int64_t n, double mu, double yhat,
                       double dhat, double kappa, void* stream, int* energy_id)
{
    int rc = add_block_common(s, "add_pt_friction");
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (n < 0 || (n > 0 && !pairs) || !(mu >= 0.0) || !(yhat > 0.0) || !(dhat > 0.0) ||
        !(kappa >= 0.0))
        return fail(ctx, SX_EINVAL, "add_pt_friction: bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    BlockHost b;
    b.kind = SX_KIND_PT_FRICTION;
    b.n = n;
    b.dhat = dhat;
    b.kappa = kappa;
    b.mu_f = mu;
    b.yhat = yhat;
    if ((rc = copy_conn(ctx, s, pairs, n, &b.conn, st)) != SX_OK) return rc;
    if (dalloc(s, &b.flag, 13 * (size_t)std::max<int64_t>(n, 1)))
        return fail(ctx, SX_ENOMEM, "add_pt_friction: allocation failed");
    CK(cudaMemsetAsync(b.flag, 0, 13 * std::max<int64_t>(n, 1) * sizeof(double), st));
    CK(cudaStreamSynchronize(st));
    register_block(s, std::move(b), energy_id);
    return SX_OK;
}

int sx_add_node_mass(sx_scene* s, const double* mass, void* stream)
{
    if (!s || !mass) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    double* tmp = nullptr;
    CK(cudaMallocAsync((void**)&tmp, s->N * sizeof(double), st));
    CK(cudaMemcpyAsync(tmp, mass, s->N * sizeof(double), cudaMemcpyDefault, st));
    k_add_vec<<<(unsigned)((s->N + 255) / 256), 256, 0, st>>>(s->extra_mass, tmp, s->N);
    if (s->finalized)
        k_add_vec<<<(unsigned)((s->N + 255) / 256), 256, 0, st>>>(s->mass, tmp, s->N);
    CK(cudaGetLastError());
    CK(cudaFreeAsync(tmp, st));
    CK(cudaStreamSynchronize(st));
    return SX_OK;
}

int sx_set_pinned(sx_scene* s, const int32_t* nodes, int64_t n, void* stream)
{
    if (!s || n < 0 || (n > 0 && !nodes)) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    int* bad = nullptr;
    int32_t* tmp = nullptr;
    CK(cudaMallocAsync((void**)&bad, sizeof(int), st));
    CK(cudaMallocAsync((void**)&tmp, std::max<int64_t>(n, 1) * sizeof(int32_t), st));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), st));
    CK(cudaMemsetAsync(s->pinned, 0, (size_t)s->N, st));
    if (n) {
        CK(cudaMemcpyAsync(tmp, nodes, n * sizeof(int32_t), cudaMemcpyDefault, st));
        k_set_pinned<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(tmp, n, s->N, s->pinned, bad);
        CK(cudaGetLastError());
    }
    int h = 0;
    CK(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(bad, st));
    CK(cudaFreeAsync(tmp, st));
    CK(cudaStreamSynchronize(st));
    if (h) return fail(ctx, SX_EINVAL, "set_pinned: node id out of range");
    return SX_OK;
}

int sx_set_gravity(sx_scene* s, const double g[3])
{
    if (!s || !g) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    for (int i = 0; i < 3; ++i) s->gravity[i] = g[i];
    CK(cudaMemcpyAsync((char*)s->sc + offsetof(SceneScal, grav), s->gravity, 3 * sizeof(double),
                       cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return SX_OK;
}

}  // extern "C"

namespace {
void release_finalized(sx_scene* s);
}  // namespace

extern "C" {

int sx_finalize(sx_scene* s, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    if (s->finalized) return SX_OK;
    if (s->pat.row_ptr) return fail(ctx, SX_EORDER, "finalize: scene already finalized once");
    // concatenated stencils in registration order
    int4* conn = nullptr;
    CK(cudaMallocAsync((void**)&conn, std::max<int64_t>(s->nst, 1) * sizeof(int4), st));
    for (auto& b : s->blocks)
        if (b.n) CK(cudaMemcpyAsync(conn + b.base, b.conn, b.n * sizeof(int4),
                                    cudaMemcpyDeviceToDevice, st));
    std::string err;
    int rc = build_pattern(conn, s->nst, s->N, &s->pat, &err, st);
    cudaFreeAsync(conn, st);
    if (rc != SX_OK) return fail(ctx, rc, err);
    for (void* p : {(void*)s->pat.row_ptr, (void*)s->pat.col, (void*)s->pat.diag_slot,
                    (void*)s->pat.slots, (void*)s->pat.slot_ptr, (void*)s->pat.slot_src,
                    (void*)s->pat.slot_order, (void*)s->pat.node_ptr, (void*)s->pat.node_src}) {
        s->allocs.push_back(p);
        s->fin_allocs.push_back(p);
    }
    const int64_t pat_bytes = (int64_t)(s->N + 1) * 8 + s->pat.nnzb * 12 + s->N * 4 +
                              s->nst * 16 * 4 * 2 + s->nst * 4 * 4;
    s->bytes += pat_bytes;
    s->fin_bytes += pat_bytes;
    // lumped mass: extra + rho V / 4 of every SNH tet, in element order
    CK(cudaMemcpyAsync(s->mass, s->extra_mass, s->N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    for (auto& b : s->blocks)
        if (b.kind == SX_KIND_SNH_TET4)
            CK(launch_block_mass(s->pat.node_ptr, s->pat.node_src, s->N, b.base, b.n, b.V, b.rho,
                                 s->mass, st));
    const size_t n3 = 3 * (size_t)s->N;
    if (dalloc_fin(s, &s->Ee, (size_t)s->nst) || dalloc_fin(s, &s->ge, 12 * (size_t)s->nst) ||
        dalloc_fin(s, &s->He, 90 * (size_t)s->nst) ||
        dalloc_fin(s, &s->vals64, 9 * (size_t)s->pat.nnzb + 8) || dalloc_fin(s, &s->grad, n3) ||
        dalloc_fin(s, &s->r, n3) || dalloc_fin(s, &s->z, n3) || dalloc_fin(s, &s->p0, n3) ||
        dalloc_fin(s, &s->p1, n3) || dalloc_fin(s, &s->q, n3) ||
        dalloc_fin(s, &s->Minv, 9 * (size_t)s->N)) {
        // back to the registered, unfinalized form: finalize can be retried
        release_finalized(s);
        return fail(ctx, SX_ENOMEM, "finalize: device allocation failed");
    }
    CK(cudaMemsetAsync(s->grad, 0, n3 * sizeof(double), st));
    CK(cudaMemsetAsync(s->vals64, 0, 9 * (size_t)s->pat.nnzb * sizeof(double), st));
    if ((rc = build_sell(s, st)) != SX_OK) {
        const std::string why = ctx->err;
        release_finalized(s);
        return fail(ctx, rc, why);
    }
    CK(cudaStreamSynchronize(st));
    s->finalized = true;
    s->version++;
    drop_batches_with(ctx, s);
    return SX_OK;
}

}  // extern "C"

namespace {

// Releases everything the last finalize built (the scene is back to its
// registered, unfinalized form; state, masses and pins are kept).
void release_finalized(sx_scene* s)
{
    drop_batches_with(s->ctx, s);
    cudaStreamSynchronize(s->stream);
    for (void* p : s->fin_allocs) {
        auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
        if (it != s->allocs.end()) s->allocs.erase(it);
        cudaFreeAsync(p, s->stream);
    }
    cudaStreamSynchronize(s->stream);
    s->fin_allocs.clear();
    s->bytes -= s->fin_bytes;
    s->fin_bytes = 0;
    s->pat = PatternOut{};
    s->Ee = s->ge = s->He = s->vals64 = s->grad = nullptr;
    s->r = s->z = s->p0 = s->p1 = s->q = s->Minv = nullptr;
    s->vals32 = nullptr;
    s->p32 = nullptr;
    s->sell_ptr = s->sell_col = nullptr;
    s->sell_v64 = nullptr;
    s->sell_v32 = nullptr;
    s->sell_steps = 0;
    s->finalized = false;
    s->last_level = -1;
    s->version++;
}

// Puts `conn` (n pairs, device, owned by the scene) in place of barrier
// block b's pairs, re-bases the blocks and rebuilds the topology.
int replace_pairs(sx_scene* s, int b, int4* conn, int64_t n, cudaStream_t st)
{
    BlockHost& blk = s->blocks[b];
    if (blk.kind == SX_KIND_PT_FRICTION) {
        // a new lag array, zero (no friction until the next lag)
        double* nl = nullptr;
        if (dalloc(s, &nl, 13 * (size_t)std::max<int64_t>(n, 1))) return SX_ENOMEM;
        cudaError_t e = cudaMemsetAsync(nl, 0, 13 * std::max<int64_t>(n, 1) * sizeof(double), st);
        if (e != cudaSuccess) return SX_ECUDA;
        if (blk.flag)
            free_scene_alloc(s, blk.flag, 13 * std::max<int64_t>(blk.n, 1) * (int64_t)sizeof(double));
        blk.flag = nl;
    }
    if (blk.conn) free_scene_alloc(s, blk.conn, std::max<int64_t>(blk.n, 1) * (int64_t)sizeof(int4));
    blk.conn = conn;
    blk.n = n;
    int64_t base = 0;
    for (auto& bb : s->blocks) {
        bb.base = base;
        base += bb.n;
    }
    s->nst = base;
    const bool was = s->finalized;
    release_finalized(s);
    if (!was) return SX_OK;
    return sx_finalize(s, st);
}

}  // namespace

extern "C" {

int sx_set_pairs(sx_scene* s, int energy_id, const int32_t* pairs, int64_t n, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    if (energy_id < 0 || energy_id >= (int)s->blocks.size() ||
        (s->blocks[energy_id].kind != SX_KIND_PT_BARRIER &&
         s->blocks[energy_id].kind != SX_KIND_PT_FRICTION) ||
        n < 0 || (n > 0 && !pairs))
        return fail(ctx, SX_EINVAL, "set_pairs: needs a point-triangle block and n >= 0 pairs");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    int4* conn = nullptr;
    int rc = copy_conn(ctx, s, pairs, n, &conn, st);
    if (rc != SX_OK) return rc;
    CK(cudaStreamSynchronize(st));
    return replace_pairs(s, energy_id, conn, n, st);
}

int sx_compact_pairs(sx_scene* s, int energy_id, int64_t* n_active, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    if (energy_id < 0 || energy_id >= (int)s->blocks.size() ||
        s->blocks[energy_id].kind != SX_KIND_PT_BARRIER)
        return fail(ctx, SX_EINVAL, "compact_pairs: needs a point-triangle block");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    const BlockHost& blk = s->blocks[energy_id];
    const int64_t n = blk.n;
    int *keep = nullptr, *off = nullptr;
    CK(cudaMallocAsync((void**)&keep, std::max<int64_t>(n, 1) * sizeof(int), st));
    CK(cudaMallocAsync((void**)&off, (n + 1) * sizeof(int), st));
    CK(launch_pair_activity(s->x, blk.conn, n, blk.dhat, keep, st));
    std::string err;
    int rc = scan_counts(keep, n, off, st, &err);
    if (rc != SX_OK) return fail(ctx, rc, err);
    int cnt = 0;
    CK(cudaMemcpyAsync(&cnt, off + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int4* conn = nullptr;
    if (dalloc(s, &conn, (size_t)cnt) != SX_OK) return fail(ctx, SX_ENOMEM, "compact_pairs: allocation failed");
    CK(launch_gather_pairs(blk.conn, keep, off, n, conn, st));
    CK(cudaFreeAsync(keep, st));
    CK(cudaFreeAsync(off, st));
    CK(cudaStreamSynchronize(st));
    if (n_active) *n_active = cnt;
    return replace_pairs(s, energy_id, conn, cnt, st);
}

int sx_set_state(sx_scene* s, const double* x, const double* v, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    const size_t b = 3 * (size_t)s->N * sizeof(double);
    if (x) CK(cudaMemcpyAsync(s->x, x, b, cudaMemcpyDefault, st));
    if (v) CK(cudaMemcpyAsync(s->v, v, b, cudaMemcpyDefault, st));
    return SX_OK;
}

int sx_get_state(sx_scene* s, double* x, double* v, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    const size_t b = 3 * (size_t)s->N * sizeof(double);
    if (x) CK(cudaMemcpyAsync(x, s->x, b, cudaMemcpyDefault, st));
    if (v) CK(cudaMemcpyAsync(v, s->v, b, cudaMemcpyDefault, st));
    return SX_OK;
}

int sx_set_inertia(sx_scene* s, double dt, const double* x_tilde, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    if (!x_tilde) {
        if (s->inertia_on) s->version++;
        s->inertia_on = false;
        return SX_OK;
    }
    if (!(dt > 0.0)) return fail(ctx, SX_EINVAL, "set_inertia: dt must be > 0");
    CK(cudaMemcpyAsync(s->x_tilde, x_tilde, 3 * (size_t)s->N * sizeof(double), cudaMemcpyDefault,
                       st));
    if (!s->inertia_on || s->dt != dt || s->inertia_mode != 0) s->version++;
    s->inertia_on = true;
    s->inertia_mode = 0;
    s->dt = dt;
    return SX_OK;
}

static int status_from_scal(sx_ctx* ctx, const SceneScal& sc)
{
    if (sc.nonfinite) return fail(ctx, SX_ENAN, "eval: non-finite energy, gradient or Hessian");
    if (sc.bad_state)
        return fail(ctx, SX_ESTATE, "eval: " + std::to_string(sc.bad_state) +
                                        " barrier pairs at distance <= 0");
    return SX_OK;
}

int sx_eval_batch(sx_ctx* ctx, sx_scene* const* scenes, int n, int level, int project,
                  int precision, double* E_out, void* stream)
{
    if (!ctx || !scenes || n <= 0) return SX_EINVAL;
    if (level < SX_E || level > SX_EGH || (precision != SX_FP64 && precision != SX_FP32))
        return fail(ctx, SX_EINVAL, "eval: bad level or precision");
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        int rc = check_scene_ready(scenes[i]);
        if (rc != SX_OK) return rc;
        if (scenes[i]->ctx != ctx) return fail(ctx, SX_EINVAL, "eval: scene of another context");
        scenes[i]->stream = st;
        if (level >= 2 && precision == SX_FP32 && (rc = ensure_vals32(ctx, scenes[i])) != SX_OK)
            return rc;
    }
    Batch* B = get_batch(ctx, scenes, n);
    int rc = prepare_batch(ctx, B, st);
    if (rc != SX_OK) return rc;
    std::vector<int> act(n, 1);
    if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
    if ((rc = run_eval(ctx, B, level, project, precision, false, st)) != SX_OK) return rc;
    if (E_out) {
        if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
        int worst = SX_OK;
        for (int i = 0; i < n; ++i) {
            E_out[i] = B->h_scal[i].E;
            int r2 = status_from_scal(ctx, B->h_scal[i]);
            if (r2 != SX_OK) worst = r2;
        }
        return worst;
    }
    return SX_OK;
}

int sx_eval(sx_scene* s, int level, int project, int precision, double* E_out, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_scene* arr[1] = {s};
    return sx_eval_batch(s->ctx, arr, 1, level, project, precision, E_out, stream);
}

int sx_get_bsr(sx_scene* s, const int32_t** row_ptr, const int32_t** col, const void** vals,
               int64_t* nnzb, int* dtype)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    if (row_ptr) *row_ptr = s->pat.row_ptr;
    if (col) *col = s->pat.col;
    if (nnzb) *nnzb = s->pat.nnzb;
    if (dtype) *dtype = s->last_precision;
    if (vals) *vals = s->last_precision == SX_FP32 ? (const void*)s->vals32 : (const void*)s->vals64;
    return SX_OK;
}

int sx_get_grad(sx_scene* s, const double** grad)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    if (grad) *grad = s->grad;
    return SX_OK;
}

int sx_get_diag_slots(sx_scene* s, const int32_t** diag)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    if (diag) *diag = s->pat.diag_slot;
    return SX_OK;
}

int sx_copy_bsr(sx_scene* s, int32_t* row_ptr, int32_t* col, void* vals, int* dtype,
                void* stream)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    if (row_ptr)
        CK(cudaMemcpyAsync(row_ptr, s->pat.row_ptr, (s->N + 1) * sizeof(int32_t),
                           cudaMemcpyDefault, st));
    if (col)
        CK(cudaMemcpyAsync(col, s->pat.col, s->pat.nnzb * sizeof(int32_t), cudaMemcpyDefault, st));
    if (dtype) *dtype = s->last_precision;
    if (vals) {
        if (s->last_precision == SX_FP32)
            CK(cudaMemcpyAsync(vals, s->vals32, 9 * s->pat.nnzb * sizeof(float), cudaMemcpyDefault,
                               st));
        else
            CK(cudaMemcpyAsync(vals, s->vals64, 9 * s->pat.nnzb * sizeof(double),
                               cudaMemcpyDefault, st));
    }
    return SX_OK;
}

int sx_copy_grad(sx_scene* s, double* grad, void* stream)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (grad)
        CK(cudaMemcpyAsync(grad, s->grad, 3 * s->N * sizeof(double), cudaMemcpyDefault,
                           (cudaStream_t)stream));
    return SX_OK;
}

int sx_scene_info(sx_scene* s, int64_t* n_nodes, int64_t* nnzb, int64_t* n_stencils,
                  int* n_blocks)
{
    if (!s) return SX_EINVAL;
    if (n_nodes) *n_nodes = s->N;
    if (nnzb) *nnzb = s->finalized ? s->pat.nnzb : 0;
    if (n_stencils) *n_stencils = s->nst;
    if (n_blocks) *n_blocks = (int)s->blocks.size();
    return SX_OK;
}

int sx_block_info(sx_scene* s, int energy_id, int* kind, int64_t* n)
{
    if (!s || energy_id < 0 || energy_id >= (int)s->blocks.size()) return SX_EINVAL;
    if (kind) *kind = s->blocks[energy_id].kind;
    if (n) *n = s->blocks[energy_id].n;
    return SX_OK;
}

int sx_eval_stats(sx_scene* s, int* clamped, int* bad_state, int* nonfinite, void* stream)
{
    if (!s) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    SceneScal h{};
    CK(cudaMemcpyAsync(&h, s->sc, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    if (clamped) *clamped = h.clamped;
    if (bad_state) *bad_state = h.bad_state;
    if (nonfinite) *nonfinite = h.nonfinite;
    return SX_OK;
}

int sx_eval_elements(sx_scene* s, int energy_id, int project, int precision, double* E,
                     double* g, double* H, int32_t* slots, void* stream)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (energy_id < 0 || energy_id >= (int)s->blocks.size())
        return fail(ctx, SX_EINVAL, "eval_elements: bad energy id");
    if (precision != SX_FP64 && precision != SX_FP32)
        return fail(ctx, SX_EINVAL, "eval_elements: bad precision");
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    const BlockHost& b = s->blocks[energy_id];
    if (slots && b.n)
        CK(cudaMemcpyAsync(slots, s->pat.slots + 16 * b.base, b.n * 16 * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, st));
    if (!E && !g && !H) return SX_OK;
    sx_scene* arr[1] = {s};
    Batch* B = get_batch(ctx, arr, 1);
    if ((rc = prepare_batch(ctx, B, st)) != SX_OK) return rc;
    std::vector<int> act(1, 1);
    if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
    std::vector<Tile> tiles;
    const int et = elements_block_threads();
    const int64_t nu = tile_units(b), ts = tile_step(b, et);
    for (int64_t k = 0; k < nu; k += ts)
        tiles.push_back(Tile{0, energy_id, k, (int)std::min<int64_t>(ts, nu - k), 0});
    Tile* d_tiles = nullptr;
    if ((rc = upload(ctx, &d_tiles, tiles, st)) != SX_OK) return rc;
    double* tmpE = nullptr;
    if (!E) CK(cudaMallocAsync((void**)&tmpE, std::max<int64_t>(b.n, 1) * sizeof(double), st));
    ElemLaunch L{};
    L.scenes = B->d_desc;
    L.tiles = d_tiles;
    L.ntiles = (int)tiles.size();
    L.level = H ? 2 : (g ? 1 : 0);
    L.project = project;
    L.precision = precision;
    L.queue = ctx->queue;
    L.out_E = E ? E : tmpE;
    double* scratch_g = nullptr;
    if (!g && H) CK(cudaMallocAsync((void**)&scratch_g, std::max<int64_t>(b.n, 1) * 12 * sizeof(double), st));
    L.out_g = g ? g : scratch_g;
    L.out_H = H;
    double* qM = nullptr;
    ClampRef* qR = nullptr;
    int* qC = nullptr;
    // the same two-launch projection as an assembled evaluation: float
    // eigenvectors, norms and the bins by N-block size
    float* qX = nullptr;
    double* qF = nullptr;
    int* qB = nullptr;
    if (H && project) {
        const size_t cap = (size_t)std::max<int64_t>(b.n, 1);
        CK(cudaMallocAsync((void**)&qM, cap * 45 * sizeof(double), st));
        CK(cudaMallocAsync((void**)&qR, cap * sizeof(ClampRef), st));
        CK(cudaMallocAsync((void**)&qC, (2 + kClampBins) * sizeof(int), st));
        CK(cudaMemsetAsync(qC, 0, (2 + kClampBins) * sizeof(int), st));
        CK(cudaMallocAsync((void**)&qX, cap * kClampRec * sizeof(float), st));
        CK(cudaMallocAsync((void**)&qF, cap * sizeof(double), st));
        CK(cudaMallocAsync((void**)&qB, cap * kClampBins * sizeof(int), st));
    }
    L.clamp_X = qX;
    L.clamp_fro = qF;
    L.clamp_bucket = qB;
    L.clamp_bucket_count = qC ? qC + 2 : nullptr;
    L.clamp_M = qM;
    L.clamp_ref = qR;
    L.clamp_count = qC;
    L.clamp_failed = qC ? qC + 1 : nullptr;
    L.clamp_cap = (int)std::max<int64_t>(b.n, 1);
    L.clamp_threads = ctx->clamp_threads[precision == SX_FP32 ? 1 : 0];
    L.clamp_grid = clamp_grid_for(L.clamp_cap, L.clamp_threads);
    L.share_sms = ctx->share_sms;
    L.kinds = kind_bit(b);
    if (b.kind == SX_KIND_TET_HO && b.ho_n) {
        PL(SX_PH_ELEMENTS, 1, launch_tetho_points(L, 0, energy_id, b.ho_n, b.ho_nq, st));
        PL(SX_PH_ELEMENTS, 1, launch_tetho_blocks(L, 0, energy_id, b.ho_n, b.ho_K, b.ho_nq, st));
    }
    PL(SX_PH_ELEMENTS, 1, launch_elements(L, elem_grid(ctx, precision, L.kinds, H ? project : 0,
                                                         L.ntiles), st));
    if (H && project) PL(SX_PH_CLAMP, 1, launch_clamp(L, st));
    int qfail[2] = {0, 0};
    if (qC) CK(cudaMemcpyAsync(qfail, qC, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (qM) {
        cudaFreeAsync(qM, st);
        cudaFreeAsync(qR, st);
        cudaFreeAsync(qC, st);
        cudaFreeAsync(qX, st);
        cudaFreeAsync(qF, st);
        cudaFreeAsync(qB, st);
    }
    cudaFreeAsync(d_tiles, st);
    if (tmpE) cudaFreeAsync(tmpE, st);
    if (scratch_g) cudaFreeAsync(scratch_g, st);
    if (qfail[1]) return fail(ctx, SX_ENAN, "eval_elements: projection did not converge");
    return SX_OK;
}

int sx_profile(sx_ctx* ctx, int enable)
{
    if (!ctx) return SX_EINVAL;
    prof_drain(ctx);
    for (int i = 0; i < SX_PH_COUNT; ++i) ctx->prof_ms[i] = 0.0;
    ctx->prof_on = enable != 0;
    return SX_OK;
}

int sx_profile_read(sx_ctx* ctx, double* ms, int64_t* launches, int reset)
{
    if (!ctx) return SX_EINVAL;
    prof_drain(ctx);
    for (int i = 0; i < SX_PH_COUNT; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (launches) launches[i] = ctx->prof_launches[i];
        if (reset) {
            ctx->prof_ms[i] = 0.0;
            ctx->prof_launches[i] = 0;
        }
    }
    return SX_OK;
}

int sx_projection_bins(sx_ctx* ctx, int* counts, void* stream)
{
    if (!ctx || !counts) return SX_EINVAL;
    static_assert(SX_PROJ_BINS == kClampBins, "projection bins");
    for (int i = 0; i < SX_PROJ_BINS; ++i) counts[i] = 0;
    if (!ctx->clampBucketCount) return SX_OK;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(counts, ctx->clampBucketCount, SX_PROJ_BINS * sizeof(int),
                       cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return SX_OK;
}

void sx_newton_opts_default(sx_newton_opts* o)
{
    if (!o) return;
    o->newton_tol = 1e-8;
    o->pcg_tol = 1e-10;
    o->max_newton = 100;
    o->max_pcg = 10000;
    o->max_halvings = 30;
    o->project = 1;
    o->precision = SX_FP64;
    o->armijo_c = 1e-4;
    o->forcing = 0;
    o->graphs = 1;
}

}  // extern "C"

namespace {

int ensure_pcg_graph(sx_ctx* ctx, Batch* B, const sx_newton_opts& o)
{
    (void)ctx;
    const int pi = o.precision == SX_FP32 ? 1 : 0;
    if (B->pcg_graph_failed) return SX_ECUDA;
    if (B->pcg_graph[pi] && B->pcg_graph_tol[pi] == o.pcg_tol && B->pcg_graph_max[pi] == o.max_pcg)
        return SX_OK;
    if (B->pcg_graph[pi]) {
        cudaGraphExecDestroy(B->pcg_graph[pi]);
        B->pcg_graph[pi] = nullptr;
    }
    PcgChunkArgs a{};
    a.scenes = B->d_desc;
    a.n_scenes = (int)B->scenes.size();
    a.node_tiles = B->d_node;
    a.n_node_tiles = (int)B->node_tiles.size();
    a.row_tiles = B->d_row;
    a.n_row_tiles = (int)B->row_tiles.size();
    a.precision = o.precision;
    a.part_row = B->d_part_row;
    a.row_beg = B->d_row_beg;
    a.row_end = B->d_row_end;
    a.part_node = B->d_part_node;
    a.node_beg = B->d_node_beg;
    a.node_end = B->d_node_end;
    a.tol = o.pcg_tol;
    a.max_iter = o.max_pcg;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
    if (ok) ok = add_pcg_chunk_nodes(g, a) == cudaSuccess;
    if (ok) ok = cudaGraphInstantiate(&ex, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
        cudaGetLastError();
        B->pcg_graph_failed = true;   // plain launches from now on
        return SX_ECUDA;
    }
    B->pcg_graph[pi] = ex;
    B->pcg_graph_tol[pi] = o.pcg_tol;
    B->pcg_graph_max[pi] = o.max_pcg;
    return SX_OK;
}

}  // namespace

extern "C" {

int sx_newton_step_batch(sx_ctx* ctx, sx_scene* const* scenes, int n, double dt,
                         const sx_newton_opts* opts_in, sx_step_report* reports, void* stream)
{
    if (!ctx || !scenes || n <= 0 || !(dt > 0.0)) return SX_EINVAL;
    sx_newton_opts o;
    if (opts_in) o = *opts_in;
    else sx_newton_opts_default(&o);
    cudaStream_t st = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < n; ++i) {
        int rc = check_scene_ready(scenes[i]);
        if (rc != SX_OK) return rc;
        scenes[i]->stream = st;
        if (o.precision == SX_FP32 && (rc = ensure_vals32(ctx, scenes[i])) != SX_OK) return rc;
        sx_scene* s = scenes[i];
        if (!s->inertia_on || s->dt != dt || s->inertia_mode != 1) s->version++;
        s->inertia_on = true;
        s->inertia_mode = 1;
        s->dt = dt;
        // friction lag at the start-of-step state with this step's dt (before
        // the batch's descriptors are prepared: dt is part of them)
        CK(update_friction(s, dt, st));
    }
    Batch* B = get_batch(ctx, scenes, n);
    int rc = prepare_batch(ctx, B, st);
    if (rc != SX_OK) return rc;
    const int nnt = (int)B->node_tiles.size();
    std::vector<int> done(n, 0), status(n, SX_OK), iters(n, 0), pcg_it(n, 0), halv(n, 0);
    std::string why;   // the first failure's reason
    std::vector<double> g0(n, 0.0), gl(n, 0.0), E(n, 0.0);
    std::vector<int> act(n, 1);
    if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
    // lagged rotations (COROT, ARAP): taken at the start-of-step state and
    // held for the step (§6.1)
    for (int i = 0; i < n; ++i) CK(update_rotations(scenes[i], st));
    PL(SX_PH_NEWTON, 1, launch_predict(B->d_desc, B->d_node, nnt, B->d_part_node, st));
    PL(SX_PH_REDUCE, 1, launch_scene_reduce(B->d_part_node, 1, 0, B->d_node_beg, B->d_node_end,
                                            n, B->d_desc, F_FEXT2, 0, st));
    std::vector<double> fext(n, 0.0);
    for (int it = 0; it <= o.max_newton; ++it) {
        // The convergence test needs E and g only. A scene whose previous
        // residual was within 10 sqrt(tol) of its reference will likely pass
        // it now (Newton converges quadratically): it is evaluated to E + g
        // first, and only a scene that does not pass takes the E + g + H
        // evaluation below, at the same state (the same E and g: level 1 runs
        // the same kernels without the Hessian). This saves the last
        // iteration's Hessian, projection and assembly.
        if (it > 0) {
            std::vector<int> likely(n, 0);
            int nl = 0;
            for (int i = 0; i < n; ++i) {
                const double ref = std::max(std::max(g0[i], fext[i]), 1e-30);
                likely[i] = !done[i] && gl[i] <= 10.0 * std::sqrt(o.newton_tol) * ref;
                nl += likely[i];
            }
            if (nl > 0) {
                if ((rc = set_active(ctx, B, likely, st)) != SX_OK) return rc;
                if ((rc = run_eval(ctx, B, SX_EG, 0, o.precision, false, st)) != SX_OK) return rc;
                if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
                for (int i = 0; i < n; ++i) {
                    if (!likely[i]) continue;
                    const SceneScal& sc = B->h_scal[i];
                    if (sc.nonfinite || !std::isfinite(sc.E) || sc.bad_state) continue;
                    const double gn = std::sqrt(sc.gnorm2);
                    if (gn <= o.newton_tol * std::max(std::max(g0[i], fext[i]), 1e-30)) {
                        E[i] = sc.E;
                        gl[i] = gn;
                        done[i] = 1;
                    }
                }
            }
        }
        for (int i = 0; i < n; ++i) act[i] = !done[i];
        {
            bool any = false;
            for (int i = 0; i < n; ++i) any = any || act[i];
            if (!any) break;
        }
        if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
        if ((rc = run_eval(ctx, B, SX_EGH, o.project, o.precision, false, st)) != SX_OK) return rc;
        if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
        int live = 0;
        for (int i = 0; i < n; ++i) {
            if (done[i]) continue;
            const SceneScal& sc = B->h_scal[i];
            E[i] = sc.E;
            if (sc.nonfinite || !std::isfinite(sc.E)) {
                status[i] = SX_ENAN;
                done[i] = 1;
                if (why.empty()) why = "non-finite energy, gradient, Hessian or projection";
                continue;
            }
            if (sc.bad_state) {
                status[i] = SX_ESTATE;
                done[i] = 1;
                if (why.empty())
                    why = "a stencil in an invalid state (barrier pair at d <= 0, "
                          "Neo-Hookean tet at J <= 0)";
                continue;
            }
            double gn = std::sqrt(sc.gnorm2);
            gl[i] = gn;
            if (it == 0) {
                g0[i] = gn;
                fext[i] = std::sqrt(sc.fext2);
            }
            // residual against the larger of the initial residual and the
            // external force on the free DOFs
            if (gn <= o.newton_tol * std::max(std::max(g0[i], fext[i]), 1e-30)) {
                done[i] = 1;
                continue;
            }
            if (it == o.max_newton) {
                status[i] = SX_ENOTCONV;
                done[i] = 1;
                if (why.empty()) why = "Newton iteration cap reached";
                continue;
            }
            iters[i] = it + 1;
            ++live;
        }
        if (!live) break;
        for (int i = 0; i < n; ++i) act[i] = !done[i];
        if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
        // ---- PCG on H dx = -g (fixed tolerance or forcing sequence)
        {
            std::vector<double> tl(n, o.pcg_tol);
            if (o.forcing)
                for (int i = 0; i < n; ++i)
                    if (act[i])
                        tl[i] = std::max(o.pcg_tol,
                                         std::min(0.5, std::sqrt(gl[i] / std::max(g0[i], 1e-300))));
            if ((rc = set_pcg_tol(ctx, B, tl, st)) != SX_OK) return rc;
        }
        PL(SX_PH_PCG, 1, launch_pcg_setup_p(B->d_desc, B->d_node, nnt, o.precision,
                                            B->d_part_node, st));
        PL(SX_PH_PCG, 1, launch_pcg_reduce(B->d_part_node, 2, B->d_node_beg, B->d_node_end, n,
                                           B->d_desc, 0, o.pcg_tol, o.max_pcg, st));
        const bool graph = o.graphs && !ctx->prof_on && ensure_pcg_graph(ctx, B, o) == SX_OK;
        // the PCG runs over the full tile lists until at most half of the
        // scenes they cover are still iterating; then over lists compacted
        // to those scenes (plain launches), compacting again at each halving
        bool compacted = false;
        int included = n;
        const Tile *cn = B->d_node, *cr = B->d_row;
        const int *cnb = B->d_node_beg, *cne = B->d_node_end, *crb = B->d_row_beg,
                  *cre = B->d_row_end;
        int cnnt = nnt, cnrt = (int)B->row_tiles.size();
        for (int k = 0;; k += 8) {
            if (graph && !compacted) {
                const int pi = o.precision == SX_FP32 ? 1 : 0;
                CK(cudaGraphLaunch(B->pcg_graph[pi], st));
                ctx->prof_launches[SX_PH_SPMV] += 8;
                ctx->prof_launches[SX_PH_PCG] += 16;
            } else {
                int par = 0;
                for (int j = 0; j < 8; ++j) {
                    PL(SX_PH_PCG, 1, launch_pcg_pdir(B->d_desc, cn, cnnt, o.precision, par, st));
                    PL(SX_PH_SPMV, 1, launch_spmv_pq(B->d_desc, cr, cnrt, o.precision, par,
                                                     B->d_part_row, crb, cre, st));
                    PL(SX_PH_PCG, 1, launch_pcg_update(B->d_desc, cn, cnnt, par, B->d_part_node,
                                                       cnb, cne, o.pcg_tol, o.max_pcg, st));
                    par ^= 1;
                }
            }
            if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
            std::vector<int> running(n, 0);
            int nrun = 0;
            for (int i = 0; i < n; ++i)
                if (act[i] && !B->h_scal[i].pcg_done) {
                    running[i] = 1;
                    ++nrun;
                }
            if (nrun == 0) break;
            if (n > 1 && 2 * nrun <= included) {
                if ((rc = compact_pcg_tiles(ctx, B, running, &cnnt, &cnrt, st)) != SX_OK) return rc;
                compacted = true;
                included = nrun;
                cn = B->d_node_c;
                cr = B->d_row_c;
                cnb = B->d_nb_c;
                cne = B->d_ne_c;
                crb = B->d_rb_c;
                cre = B->d_re_c;
            }
        }
        for (int i = 0; i < n; ++i) {
            if (!act[i]) continue;
            pcg_it[i] += B->h_scal[i].pcg_iters;
            if (B->h_scal[i].pcg_status != 0) {
                const int ps = B->h_scal[i].pcg_status;
                status[i] = SX_ENOTCONV;
                if (why.empty())
                    why = ps == 1 ? "PCG: p.q <= 0 (the system is not positive definite)"
                                  : "PCG: iteration cap reached";
                done[i] = 1;
                act[i] = 0;
            }
        }
        if ((rc = set_active(ctx, B, act, st)) != SX_OK) return rc;
        // ---- Armijo backtracking on E_BE
        PL(SX_PH_NEWTON, 1, launch_gdx(B->d_desc, B->d_node, nnt, B->d_part_node, st));
        PL(SX_PH_REDUCE, 1, launch_scene_reduce(B->d_part_node, 1, 0, B->d_node_beg,
                                                B->d_node_end, n, B->d_desc, F_GDX, 0, st));
        if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
        std::vector<double> gdx(n), alpha(n, 1.0);
        for (int i = 0; i < n; ++i) gdx[i] = B->h_scal[i].gdx;
        std::vector<int> search = act;
        for (int h = 0; h <= o.max_halvings; ++h) {
            bool any = false;
            for (int i = 0; i < n; ++i) any |= search[i] != 0;
            if (!any) break;
            if ((rc = set_active(ctx, B, search, st)) != SX_OK) return rc;
            if ((rc = set_alpha(ctx, B, alpha, st)) != SX_OK) return rc;
            PL(SX_PH_NEWTON, 1, launch_trial(B->d_desc, B->d_node, nnt, st));
            if ((rc = run_eval(ctx, B, SX_E, 0, o.precision, true, st)) != SX_OK) return rc;
            if ((rc = read_scal(ctx, B, st)) != SX_OK) return rc;
            std::vector<int> acc(n, 0);
            for (int i = 0; i < n; ++i) {
                if (!search[i]) continue;
                const SceneScal& sc = B->h_scal[i];
                // below the resolution of double energies (|g.dx| < 1e-12 |E|)
                // the Armijo comparison is noise: take the full Newton step
                const bool tiny = std::fabs(gdx[i]) < 1e-12 * std::fabs(E[i]);
                bool ok = sc.bad_state == 0 && sc.nonfinite == 0 && std::isfinite(sc.E) &&
                          (tiny || sc.E <= E[i] + o.armijo_c * alpha[i] * gdx[i]);
                if (ok) {
                    acc[i] = 1;
                    search[i] = 0;
                } else {
                    alpha[i] *= 0.5;
                    halv[i] += 1;
                }
            }
            if ((rc = set_active(ctx, B, acc, st)) != SX_OK) return rc;
            PL(SX_PH_NEWTON, 1, launch_accept(B->d_desc, B->d_node, nnt, st));
        }
        for (int i = 0; i < n; ++i)
            if (search[i]) {
                status[i] = SX_ELINESEARCH;
                done[i] = 1;
                if (why.empty()) why = "line search: no sufficient decrease";
            }
    }
    // a scene whose step failed keeps the state it had at the call (x back
    // to the start of the step, v untouched); the others take
    // v = (x - x_t) / dt
    std::vector<int> okv(n), badv(n);
    bool any_bad = false;
    for (int i = 0; i < n; ++i) {
        okv[i] = status[i] == SX_OK;
        badv[i] = !okv[i];
        any_bad = any_bad || badv[i];
    }
    if (any_bad) {
        if ((rc = set_active(ctx, B, badv, st)) != SX_OK) return rc;
        PL(SX_PH_NEWTON, 1, launch_restore(B->d_desc, B->d_node, nnt, st));
    }
    if ((rc = set_active(ctx, B, okv, st)) != SX_OK) return rc;
    PL(SX_PH_NEWTON, 1, launch_velocity(B->d_desc, B->d_node, nnt, st));
    CK(cudaStreamSynchronize(st));
    double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    int worst = SX_OK;
    for (int i = 0; i < n; ++i) {
        if (reports) {
            sx_step_report& r = reports[i];
            r.status = status[i];
            r.newton_iters = iters[i];
            r.pcg_iters = pcg_it[i];
            r.ls_halvings = halv[i];
            r.g0_norm = g0[i];
            r.g_norm = gl[i];
            r.energy = E[i];
            r.ms = ms;
        }
        if (status[i] != SX_OK) worst = status[i];
    }
    if (worst != SX_OK)
        fail(ctx, worst, "newton_step: at least one scene failed" + (why.empty() ? std::string() : " (" + why + ")"));
    return worst;
}

int sx_newton_step(sx_scene* s, double dt, const sx_newton_opts* opts, sx_step_report* report,
                   void* stream)
{
    if (!s) return SX_EINVAL;
    sx_scene* arr[1] = {s};
    return sx_newton_step_batch(s->ctx, arr, 1, dt, opts, report, stream);
}

int sx_advance(sx_scene* s, double dt, const sx_newton_opts* opts, int max_dt_halvings,
               sx_step_report* report, int* substeps, void* stream)
{
    if (!s || !(dt > 0.0) || max_dt_halvings < 0 || max_dt_halvings > 30) return SX_EINVAL;
    sx_ctx* ctx = s->ctx;
    cudaStream_t st = (cudaStream_t)stream;
    const auto t0 = std::chrono::steady_clock::now();
    const size_t n3 = 3 * (size_t)s->N;
    double *xs = nullptr, *vs = nullptr;
    {
        // both snapshots or neither (no buffer left behind on failure)
        const cudaError_t ex = cudaMallocAsync((void**)&xs, n3 * sizeof(double), st);
        const cudaError_t ev = ex == cudaSuccess
                                   ? cudaMallocAsync((void**)&vs, n3 * sizeof(double), st)
                                   : cudaSuccess;
        if (ex != cudaSuccess || ev != cudaSuccess) {
            if (xs) cudaFreeAsync(xs, st);
            return cuda_fail(ctx, ex != cudaSuccess ? ex : ev, "advance: state snapshot");
        }
    }
    sx_step_report agg{};
    int taken = 0, rc_final = SX_OK;
    // intervals still to cover, the next one at the back: (size, depth)
    std::vector<std::pair<double, int>> todo{{dt, 0}};
    while (!todo.empty()) {
        const std::pair<double, int> cur = todo.back();
        todo.pop_back();
        cudaError_t e = cudaMemcpyAsync(xs, s->x, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(vs, s->v, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            rc_final = cuda_fail(ctx, e, "advance: state copy");
            break;
        }
        sx_step_report r{};
        const int rc = sx_newton_step(s, cur.first, opts, &r, stream);
        if (rc == SX_OK) {
            if (taken == 0) agg.g0_norm = r.g0_norm;
            agg.newton_iters += r.newton_iters;
            agg.pcg_iters += r.pcg_iters;
            agg.ls_halvings += r.ls_halvings;
            agg.g_norm = r.g_norm;
            agg.energy = r.energy;
            ++taken;
            continue;
        }
        const bool retry = rc == SX_ENOTCONV || rc == SX_ELINESEARCH || rc == SX_ENAN ||
                           rc == SX_ESTATE;
        // back to the start of this substep, whatever the failure (a retried
        // substep starts there; any other failure returns with that state)
        e = cudaMemcpyAsync(s->x, xs, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s->v, vs, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) {
            rc_final = cuda_fail(ctx, e, "advance: state restore after a failed substep");
            break;
        }
        if (!retry || cur.second >= max_dt_halvings) {
            rc_final = rc;
            break;
        }
        // two halves, the first one next
        todo.push_back({0.5 * cur.first, cur.second + 1});
        todo.push_back({0.5 * cur.first, cur.second + 1});
    }
    cudaFreeAsync(xs, st);
    cudaFreeAsync(vs, st);
    CK(cudaStreamSynchronize(st));
    // substeps that failed and were covered by halves left their reason in
    // the context's error text; a successful call clears it
    if (rc_final == SX_OK) ctx->err.clear();
    agg.status = rc_final;
    agg.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (report) *report = agg;
    if (substeps) *substeps = taken;
    return rc_final;
}

int sx_scene_footprint(const sx_scene_desc* d, int64_t* bytes)
{
    if (!d || !bytes) return SX_EINVAL;
    const int64_t N = d->n_nodes, nst = d->n_tets + d->n_hinges + d->n_pairs;
    int64_t nnzb = d->nnzb_hint > 0 ? d->nnzb_hint : N + 16 * nst;
    int64_t b = 0;
    b += N * (3 * 8 * 13 + 8 * 2 + 1 + 9 * 8 + 8 * 2);    // node vectors, mass, pins, Minv, ptrs
    b += d->n_tets * (16 + 12 * 8);                         // conn + rest params
    b += d->n_hinges * (16 + 5 * 8);
    b += d->n_pairs * 16;
    b += nst * (8 + 12 * 8 + 90 * 8 + 16 * 4 * 2 + 4 * 4); // staging, slots, lists
    // the context's projection scratch for the scene's projectable stencils
    // (tets and pairs): 9x9 matrix, reference, float eigenvectors, norm, bins
    b += (d->n_tets + d->n_pairs) * (45 * 8 + 16 + kClampRec * 4 + 8 + kClampBins * 4);
    b += nnzb * (4 + 4 + 4 + 9 * 8);                        // col, slot_ptr, order, values
    b += (nnzb + nnzb / 4 + 64) * (4 + 9 * 8) + N / 8;      // SpMV sliced copy (padded)
    b += 1 << 20;
    *bytes = b;
    return SX_OK;
}

int sx_scene_bytes(sx_scene* s, int64_t* bytes)
{
    if (!s || !bytes) return SX_EINVAL;
    *bytes = s->bytes;
    return SX_OK;
}

int sx_set_launch_shape(sx_ctx* ctx, int precision, int clamp_threads, int elem_blocks_per_sm)
{
    if (!ctx || (precision != SX_FP64 && precision != SX_FP32) ||
        (clamp_threads != 32 && clamp_threads != 64 && clamp_threads != 128 &&
         clamp_threads != 256) ||
        elem_blocks_per_sm < -1)
        return SX_EINVAL;
    const int p = precision == SX_FP32 ? 1 : 0;
    ctx->clamp_threads[p] = clamp_threads;
    ctx->elem_bps[p] = elem_blocks_per_sm;   // capped at what fits when launched
    return SX_OK;
}

int sx_get_launch_shape(sx_ctx* ctx, int precision, int* clamp_threads, int* elem_blocks_per_sm)
{
    if (!ctx || (precision != SX_FP64 && precision != SX_FP32)) return SX_EINVAL;
    const int p = precision == SX_FP32 ? 1 : 0;
    if (clamp_threads) *clamp_threads = ctx->clamp_threads[p];
    if (elem_blocks_per_sm) *elem_blocks_per_sm = ctx->elem_bps[p];
    return SX_OK;
}

// Launch-shape autotuner: times E + g + projected H + assembly of this batch
// (CUDA events on the caller's stream, best of 3 after a warm-up pass) for
// the default shape, then for each other projection block size, then for
// each element-grid choice with the best block size, and keeps the fastest
// for `precision` in the context. Every shape computes the same result (the
// per-element work and every sum are independent of the grid).
int sx_autotune(sx_ctx* ctx, sx_scene* const* scenes, int n, int precision,
                sx_tune_report* report, void* stream)
{
    if (!ctx || !scenes || n <= 0 || (precision != SX_FP64 && precision != SX_FP32))
        return SX_EINVAL;
    const int p = precision == SX_FP32 ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    int cand = 0;
    auto timed = [&](int ct, int bps, double* ms) -> int {
        ctx->clamp_threads[p] = ct;
        ctx->elem_bps[p] = bps;
        int rc = sx_eval_batch(ctx, scenes, n, SX_EGH, 1, precision, nullptr, stream);
        if (rc != SX_OK) return rc;
        double best = 1e300;
        for (int r = 0; r < 3; ++r) {
            CK(cudaEventRecord(a, st));
            rc = sx_eval_batch(ctx, scenes, n, SX_EGH, 1, precision, nullptr, stream);
            if (rc != SX_OK) return rc;
            CK(cudaEventRecord(b, st));
            CK(cudaEventSynchronize(b));
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, a, b));
            best = std::min(best, (double)t);
        }
        ++cand;
        *ms = best;
        return SX_OK;
    };
    int best_ct = 128, best_bps = -1;
    double def_ms = 0.0, best_ms = 0.0, ms = 0.0;
    int rc = timed(best_ct, best_bps, &def_ms);
    best_ms = def_ms;
    for (int ct : {32, 64, 256}) {
        if (rc != SX_OK) break;
        rc = timed(ct, best_bps, &ms);
        if (rc == SX_OK && ms < best_ms) {
            best_ms = ms;
            best_ct = ct;
        }
    }
    // element grid: as many blocks as fit (default), one per SM, one tile
    // per block
    for (int bps : {1, 0}) {
        if (rc != SX_OK) break;
        rc = timed(best_ct, bps, &ms);
        if (rc == SX_OK && ms < best_ms) {
            best_ms = ms;
            best_bps = bps;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->clamp_threads[p] = best_ct;
    ctx->elem_bps[p] = best_bps;
    if (rc != SX_OK) return rc;
    if (report) {
        report->clamp_threads = best_ct;
        report->elem_blocks_per_sm = best_bps;
        report->default_ms = def_ms;
        report->tuned_ms = best_ms;
        report->candidates = cand;
    }
    return SX_OK;
}

}  // extern "C"

// ==================================================================== no-alloc
// Scratch of sx_eval_elements_noalloc: file-scope device arrays, so that
// the call never allocates. In host code these names are only stand-ins
// for the device symbols; their device addresses come from
// cudaGetSymbolAddress, looked up once per device.
namespace {

constexpr int kNaMaxTiles = (SX_NOALLOC_MAX_ELEMENTS + 127) / 128;

static __device__ __align__(256) SceneDev g_na_desc[1];
static __device__ __align__(256) Tile g_na_tiles[kNaMaxTiles];
static __device__ __align__(256) int g_na_counters[4];   // queue, clamp count, clamp failures
static __device__ __align__(256) double g_na_clampM[(size_t)SX_NOALLOC_MAX_ELEMENTS * 45];
static __device__ __align__(256) ClampRef g_na_clampRef[SX_NOALLOC_MAX_ELEMENTS];

struct NaPtrs {
    bool ready = false;
    SceneDev* desc = nullptr;
    Tile* tiles = nullptr;
    int* counters = nullptr;
    double* clampM = nullptr;
    ClampRef* clampRef = nullptr;
};

constexpr int kNaMaxDevices = 64;
NaPtrs g_na_ptrs[kNaMaxDevices];
std::mutex g_na_mutex;

// once per device, with that device current
int na_setup(sx_ctx* ctx, NaPtrs** out)
{
    const int dev = ctx->device;
    if (dev < 0 || dev >= kNaMaxDevices) return fail(ctx, SX_EINVAL, "noalloc: device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    NaPtrs& P = g_na_ptrs[dev];
    if (!P.ready) {
        int prev = -1;
        CK(cudaGetDevice(&prev));
        if (prev != dev) CK(cudaSetDevice(dev));
        cudaError_t e = cudaGetSymbolAddress((void**)&P.desc, g_na_desc);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&P.tiles, g_na_tiles);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&P.counters, g_na_counters);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&P.clampM, g_na_clampM);
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&P.clampRef, g_na_clampRef);
        if (prev != dev) cudaSetDevice(prev);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "noalloc: cudaGetSymbolAddress");
        P.ready = true;
    }
    *out = &P;
    return SX_OK;
}

}  // namespace

extern "C" int sx_eval_elements_noalloc(sx_scene* s, int energy_id, int project, int precision,
                                        double* E, double* g, double* H, void* stream)
{
    int rc = check_scene_ready(s);
    if (rc != SX_OK) return rc;
    sx_ctx* ctx = s->ctx;
    if (energy_id < 0 || energy_id >= (int)s->blocks.size())
        return fail(ctx, SX_EINVAL, "eval_elements_noalloc: bad energy id");
    if (precision != SX_FP64 && precision != SX_FP32)
        return fail(ctx, SX_EINVAL, "eval_elements_noalloc: bad precision");
    const BlockHost& b = s->blocks[energy_id];
    if (b.n > SX_NOALLOC_MAX_ELEMENTS)
        return fail(ctx, SX_EINVAL,
                    "eval_elements_noalloc: block has " + std::to_string(b.n) +
                        " elements, more than the static scratch holds (" +
                        std::to_string(SX_NOALLOC_MAX_ELEMENTS) + ")");
    if (b.n == 0) return SX_OK;
    {
        // the static tile table holds kNaMaxTiles tiles (shorter high-order
        // tiles may need more than the 128-stencil ones it is sized for)
        const int64_t ts = tile_step(b, elements_block_threads());
        if ((b.n + ts - 1) / ts > kNaMaxTiles)
            return fail(ctx, SX_EINVAL, "eval_elements_noalloc: block needs more tiles than the "
                                        "static scratch holds");
    }
    NaPtrs* P = nullptr;
    if ((rc = na_setup(ctx, &P)) != SX_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    s->stream = st;
    // scene descriptor and tile table into the static arrays (pageable
    // sources: each copy returns once the source has been consumed)
    const SceneDev desc = make_desc(s, false);
    CK(cudaMemcpyAsync(P->desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, st));
    Tile tiles[kNaMaxTiles];
    const int et = elements_block_threads();
    int nt = 0;
    const int64_t nu = tile_units(b), ts = tile_step(b, et);
    for (int64_t k = 0; k < nu; k += ts)
        tiles[nt++] = Tile{0, energy_id, k, (int)std::min<int64_t>(ts, nu - k), 0};
    CK(cudaMemcpyAsync(P->tiles, tiles, nt * sizeof(Tile), cudaMemcpyHostToDevice, st));
    static const int one = 1;
    CK(cudaMemcpyAsync((char*)s->sc + offsetof(SceneScal, active), &one, sizeof(int),
                       cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(P->counters, 0, 4 * sizeof(int), st));
    ElemLaunch L{};
    L.scenes = P->desc;
    L.tiles = P->tiles;
    L.ntiles = nt;
    L.level = H ? 2 : (g ? 1 : 0);
    L.project = project;
    L.precision = precision;
    L.queue = P->counters;
    L.out_E = E;
    L.out_g = g;
    L.out_H = H;
    L.clamp_M = P->clampM;
    L.clamp_ref = P->clampRef;
    L.clamp_count = P->counters + 1;
    L.clamp_failed = P->counters + 2;
    L.clamp_cap = SX_NOALLOC_MAX_ELEMENTS;
    L.clamp_threads = ctx->clamp_threads[precision == SX_FP32 ? 1 : 0];
    L.clamp_grid = clamp_grid_for(L.clamp_cap, L.clamp_threads);
    L.share_sms = ctx->share_sms;
    L.kinds = kind_bit(b);
    const int grid = elem_grid(ctx, precision, L.kinds, H ? project : 0, nt);
    if (b.kind == SX_KIND_TET_HO && b.ho_n) {
        PL(SX_PH_ELEMENTS, 1, launch_tetho_points(L, 0, energy_id, b.ho_n, b.ho_nq, st));
        PL(SX_PH_ELEMENTS, 1, launch_tetho_blocks(L, 0, energy_id, b.ho_n, b.ho_K, b.ho_nq, st));
    }
    PL(SX_PH_ELEMENTS, 1, launch_elements(L, grid, st));
    if (H && project) PL(SX_PH_CLAMP, 1, launch_clamp(L, st));
    int failed = 0;
    CK(cudaMemcpyAsync(&failed, P->counters + 2, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (failed) return fail(ctx, SX_ENAN, "eval_elements_noalloc: projection did not converge");
    return SX_OK;
}
