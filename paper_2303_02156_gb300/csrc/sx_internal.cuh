// sx_internal.cuh -- internal types shared by the libsx translation units.
//
// Data model (device, per scene; AoS xyz per node, SoA per-element params):
//   x, v, x_start, x_tilde, x_trial, dx, grad, r, z, p0, p1, q : double[3N]
//   mass : double[N];  pinned : uint8[N];  Minv : double[9N]
//   energy blocks: conn int4[n]; SNH Dm^-1 double[9][n], V, mu', lambda'
//                  double[n]; hinge q double[4][n], c double[n]
//   staged element outputs: E_e double[nst]; g_e double[nst][12];
//                           H_e (double|float)[nst][90] = 10 upper 3x3 blocks
//   pattern: row_ptr int[N+1], col int[nnzb], diag_slot int[N],
//            slots int[nst][16]
//   assembly lists (element-id ordered): slot_ptr int[nnzb+1],
//            slot_src int[nst*16] (code 16*stencil + 4a + b),
//            node_ptr int[N+1], node_src int[nst*4] (code 4*stencil + a)
//   BSR values: double[nnzb][9] (FP64) and float[nnzb][9] (FP32 form)
//   SpMV copy of the values, sliced ELLPACK (32-row slices padded to their
//   longest row): sell_ptr int[N/32+1], sell_col int[32 steps],
//   sell_v64 double[9 x 32 steps] (+ sell_v32 float in the FP32 form)
//
// Kernels are written over "tiles" (scene, block, start, count) so that a
// single scene, a batch of scenes and the server's mixes all run through
// the same launches; per-tile partial sums are reduced per scene in a fixed
// order, so every result is deterministic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/sx.h"

#define SX_MAX_BLOCKS 8

namespace sx {

// upper 3x3 blocks of a 4-node stencil Hessian, in staging order
// non-finite test on the exponent bits: an integer-pipe operation (a
// floating compare would take an issue slot of the FP64 pipe, and a float
// value would first be converted there)
__device__ __forceinline__ bool nonfinite_bits(double x)
{
    return (__double2hiint(x) & 0x7ff00000) == 0x7ff00000;
}
__device__ __forceinline__ bool nonfinite_bits(float x)
{
    return (__float_as_int(x) & 0x7f800000) == 0x7f800000;
}

__host__ __device__ constexpr int up_index(int a, int b)
{
    // (0,0)=0 (0,1)=1 (0,2)=2 (0,3)=3 (1,1)=4 (1,2)=5 (1,3)=6 (2,2)=7 (2,3)=8 (3,3)=9
    return a == 0 ? b : (a == 1 ? 3 + b : (a == 2 ? 5 + b : 9));
}

struct ElemBlock {
    int kind;            // SX_KIND_*
    int model;           // SX_MODEL_* of a tet4 block
    int64_t n;           // stencils in this block
    int64_t base;        // first scene-global stencil id of this block
    const int4* conn;
    // SNH tet4
    const double* Dminv;  // [9][n] row-major Dm^-1 entries
    const double* V;
    const double* mu;
    const double* lam;
    const double* R;      // [9][n] lagged rotations (COROT, ARAP)
    // hinge
    const double* q;      // [4][n]
    const double* c;
    double kb;
    // barrier, friction (the friction's fn comes from this barrier)
    double dhat, kappa;
    // friction: lag [13][n] = beta (3), T (6), fn, dx_lag (3); mu, yhat, dt
    const double* flag;
    double mu_f, yhat, dt_f;
    // high-order tets: ho_n elements of ho_K nodes, ho_S sub-stencils each
    // (n = ho_n ho_S), ho_nq quadrature points
    int ho_K, ho_S, ho_nq;
    int64_t ho_n;
    const int* ho_conn;      // [K][ho_n] node ids
    const double* ho_Jinv;   // [nq][9][ho_n] J0^-1 at the points
    const double* ho_wdet;   // [nq][ho_n] w_q det J0
    const double* ho_dN;     // [nq][K][3] reference gradients
    const int* ho_sub;       // [S][4] local nodes of the sub-stencils
    const int* ho_own;       // [S] bits 0-9: owned upper blocks, 10-13: owned nodes
    double* ho_modes;        // [ho_n][nq][91] negative modes per point (projection scratch)
    double* ho_rec;          // [ho_n][nq][kHoRec] per-point records (scratch)
    int* ho_flag;            // [ho_n] non-finite output seen (scratch)
    const int* ho_pair;      // [K(K+1)/2][3] owned blocks: owner-local node pair, slot j*10+ab
    const int* ho_gown;      // [K] owner of each node's gradient: j*4 + local node
};

// per-scene scalars the device loops read and write
struct SceneScal {
    double E;          // energy of the last evaluation
    double gnorm2;     // ||g_free||^2 of the last EG/EGH evaluation
    double bnorm2;     // PCG: ||b||^2
    double rz;         // PCG: r.z
    double rz_new;
    double pq;         // PCG: p.Aq
    double rr;         // PCG: ||r||^2
    double gdx;        // Newton: g.dx
    double pcg_alpha;
    double pcg_beta;
    double ls_alpha;   // line-search step
    double pcg_tol;    // relative PCG tolerance of the current solve
    double fext2;      // ||M g_ext||^2 over the free DOFs (Newton residual scale)
    double grav[3];    // external acceleration (M^-1 f_ext)
    int pcg_done;      // 1 once converged or stopped (kernels skip the scene)
    int pcg_iters;
    int pcg_status;    // 0 ok, 1 breakdown (p.Ap <= 0), 2 iteration cap
    int active;        // scene takes part in the current batched phase
    int bad_state;     // barrier pairs with d <= 0 in the last evaluation
    int nonfinite;     // non-finite values seen in the last evaluation
    int clamped;       // elements projected in the last EGH evaluation
    int clamp_fail;    // set by the projection kernel if QL did not converge
    int cnt_spmv;      // PCG: row tiles of this scene done in the current SpMV
    int cnt_update;    // PCG: node tiles of this scene done in the current update
};

struct SceneDev {
    int64_t N;
    int64_t nst;
    int64_t nnzb;
    int nblocks;
    int inertia_on;
    int inertia_mode;   // 0: residual x - x_tilde; 1: (x - x_start) - (dt v + dt^2 g)
    int pad0;
    double dt;
    double inv_dt2;
    ElemBlock blk[SX_MAX_BLOCKS];
    double* x;
    double* v;
    double* x_start;
    double* x_tilde;
    double* x_trial;
    double* dx;
    double* mass;
    const uint8_t* pinned;
    double* grad;
    double* Ee;
    double* ge;
    void* He;
    const int* row_ptr;
    const int* col;
    const int* diag_slot;
    const int* slots;
    const int* slot_ptr;
    const int* slot_src;
    const int* slot_order;
    const int* node_ptr;
    const int* node_src;
    double* vals64;
    float* vals32;
    // the PCG's sliced-ELLPACK copy of the values: 32-row slices, slice s
    // spans steps sell_ptr[s] .. sell_ptr[s+1]; columns [step][lane],
    // values [step][9][lane] (pad entries: value 0, the row's own column)
    const int* sell_ptr;
    const int* sell_col;
    double* sell_v64;
    float* sell_v32;
    double* r;
    double* z;
    double* p0;
    double* p1;
    float* p32;     // FP32 form: float copy of the current direction
    double* q;
    double* Minv;
    SceneScal* sc;
};

struct Tile {
    int scene;   // index into the batch's SceneDev array
    int blk;     // energy block (element tiles) or unused
    int64_t start;
    int count;
    int pad;
};

// ---------------------------------------------------------------- kernels
// element evaluation (sx_elements.cu)
struct ClampRef {
    int scene;
    int blk;
    int64_t e;   // element index inside its energy block
};

// per queued stencil record of the split projection (floats): the float
// eigenvectors as the Jacobi left them (column c at 9 c), their 9
// eigenvalues (81 + c), the column of each ascending-eigenvalue slot
// (4 bits per slot in the two words at 90), the N-block size k (an int in
// word 92), pad
constexpr int kClampRec = 96;
constexpr int kClampBins = 20;
constexpr int kClampPass2 = 10;   // bins 11..13: second refinement pass, k = 1..3
constexpr int kClampDefl = 16;    // bins 17..19: deflation of k' = 1..3 negative modes

struct ElemLaunch {
    const SceneDev* scenes;
    const Tile* tiles;
    int ntiles;
    int level;
    int project;
    int precision;
    double* tile_E;       // per tile energy partial
    int* tile_bad;        // per tile barrier d<=0 count
    int* tile_nonfinite;
    int* tile_clamped;    // per tile number of projected elements
    int* queue;           // work counter for the persistent launch
    // element-level output mode (sx_eval_elements): when non-null the
    // kernel writes E, g (12) and the full 12x12 H per element of the
    // block (indexed by the element's position in its block) instead of
    // the staged assembly buffers
    double* out_E;
    double* out_g;
    double* out_H;
    // projection queue: translation-free 9x9 Hessians (45 packed doubles)
    // of the stencils that failed the PSD test, and where their blocks live
    double* clamp_M;
    ClampRef* clamp_ref;
    int* clamp_count;
    int* clamp_failed;
    int clamp_cap;
    int clamp_grid;
    // split projection (batched evaluations; null: one fused launch): a
    // record of kClampRec floats per queued stencil (its float eigenvectors,
    // their eigenvalues and their order),
    // ||M||_F per queued stencil, and the queue positions binned
    // (kClampBins bins of clamp_cap: 0..9 by N-block size k, kClampPass2 + k
    // for the second refinement pass of k = 1..3, kClampDefl + k' for the
    // deflation of the k' negative modes of a stencil with k >= 4)
    float* clamp_X;
    double* clamp_fro;
    int* clamp_bucket;
    int* clamp_bucket_count;
    int clamp_threads;    // projection block size: 32, 64, 128 (default) or 256
    int kinds;            // stencil kinds present (1 SNH, 2 hinge, 4 barrier)
    int share_sms;        // leave one projection block per SM for other work
};
cudaError_t launch_elements(const ElemLaunch& L, int grid, cudaStream_t s);
cudaError_t launch_clamp(const ElemLaunch& L, cudaStream_t s);
int elements_block_threads();
int clamp_block_threads();
// the element kernel instantiations: variant 0 every kind, 1 SNH only, 2
// every kind with the F-space projection, 3 SNH only with it
const void* elements_kernel(int precision, int variant);
constexpr int kElemVariants = 8;
// the element-kernel instantiations of each translation unit (KINDS values)
const void* elements_kernel_snh(int kinds, bool f32);      // 1, 7
const void* elements_kernel_fproj(int kinds, bool f32);    // 9, 15
const void* elements_kernel_models(int kinds, bool f32);   // 25, 63
cudaError_t launch_elements_snh(int kinds, bool f32, const ElemLaunch& L, int grid,
                                cudaStream_t s);
cudaError_t launch_elements_fproj(int kinds, bool f32, const ElemLaunch& L, int grid,
                                  cudaStream_t s);
cudaError_t launch_elements_models(int kinds, bool f32, const ElemLaunch& L, int grid,
                                   cudaStream_t s);
// high-order tets (sx_tetho.cu)
constexpr int kHoMaxK = 20;
int tetho_cover(int K, std::vector<int>& sub, std::vector<int>& own);
void tetho_ref_grads(int K, const double* xi, double* dN);
cudaError_t launch_tetho_rest(const double* X, int64_t N, const int* conn, int64_t n, int K,
                              int nq, const double* rule_w, const double* dN, double* Jinv,
                              double* wdet, double* vol, int* bad, cudaStream_t s);
const void* elements_kernel_ho(int kinds, bool f32);       // 64, 127
// phase 1 of the high-order tets: one thread per (element, point) of block
// `blk` of scene `scene` (F, psi, P, the Hessian coefficients -> ho_rec;
// with projection the negative modes -> ho_modes), before the element kernel
cudaError_t launch_tetho_points(const ElemLaunch& L, int scene, int blk, int64_t n_el, int nq,
                                cudaStream_t s);
// then the blocks, gradients and energies of the block's sub-stencils
// (one element per group of threads; K, nq as registered)
cudaError_t launch_tetho_blocks(const ElemLaunch& L, int scene, int blk, int64_t n_el, int K,
                                int nq, cudaStream_t s);
// shared memory one element of k_tetho_blocks needs (bytes), with projection
int tetho_block_smem(int K, int nq);
constexpr int kHoRec = 42;   // wd, psi, Ji (9), F (9), C (9), P (9), cI cF cC cS
constexpr int kHoTileElems = 32;   // whole elements per element-kernel tile
cudaError_t launch_elements_ho(int kinds, bool f32, const ElemLaunch& L, int grid,
                               cudaStream_t s);
cudaError_t launch_friction_lag(const double* x, const int4* conn, int64_t n, double dhat,
                                double kappa, double* lag, cudaStream_t s);
cudaError_t launch_tet_rotations(const int4* conn, const double* x, const double* Dminv,
                                 int64_t n, double* R, cudaStream_t s);
int elements_variant(int kinds, int project);

// point-triangle pair activation and order-preserving compaction
// (sx_elements.cu)
cudaError_t launch_pair_activity(const double* x, const int4* conn, int64_t n, double dhat,
                                 int* keep, cudaStream_t s);
cudaError_t launch_gather_pairs(const int4* conn, const int* keep, const int* offsets, int64_t n,
                                int4* out, cudaStream_t s);

// registration and pattern (sx_graph.cu)
cudaError_t launch_snh_rest(const double* X, int64_t N, const int4* tets, int64_t n,
                            const double* young, const double* poisson, double rho,
                            int literal, double* Dminv, double* V, double* mu,
                            double* lam, int* bad, cudaStream_t s);
cudaError_t launch_block_mass(const int* node_ptr, const int* node_src, int64_t N,
                              int64_t base, int64_t cnt, const double* V, double rho,
                              double* mass, cudaStream_t s);
struct PatternOut {
    int* row_ptr;
    int* col;
    int64_t nnzb;
    int* diag_slot;
    int* slots;
    int* slot_ptr;
    int* slot_src;
    int* slot_order;   // per tile of kSlotTile blocks: the blocks by ascending list length
    int* node_ptr;
    int* node_src;
};
// BSR blocks per assembly tile (the unit of slot_order)
constexpr int kSlotTile = 256;
int build_pattern(const int4* conn, int64_t nst, int64_t N, PatternOut* out,
                  std::string* err, cudaStream_t s);
// exclusive prefix sum of n int32 counts into out[0..n] (out[n] = total)
int scan_counts(const int* in, int64_t n, int* out, cudaStream_t s, std::string* err);

// assembly and reductions (sx_assemble.cu)
struct AsmLaunch {
    const SceneDev* scenes;
    const Tile* tiles;
    int ntiles;
    int precision;
};
cudaError_t launch_assemble_vals(const AsmLaunch& L, cudaStream_t s);
cudaError_t launch_inertia_diag(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                int precision, cudaStream_t s);
cudaError_t launch_assemble_grad(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                 double* tile_part, cudaStream_t s);
cudaError_t launch_inertia_energy(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                                  const double* unused, double* tile_part, int use_trial,
                                  cudaStream_t s);
enum ScalField { F_E = 0, F_GNORM2 = 1, F_GDX = 2, F_FEXT2 = 3 };
cudaError_t launch_scene_reduce(const double* part, int stride, int off, const int* tbeg,
                                const int* tend, int nscenes, const SceneDev* scenes,
                                int field, int accumulate, cudaStream_t s);
cudaError_t launch_scene_reduce_flags(const int* bad, const int* nonfin, const int* clamped,
                                      const int* tbeg, const int* tend, int nscenes,
                                      const SceneDev* scenes, cudaStream_t s);
cudaError_t launch_gather_scal(const SceneDev* scenes, int n, SceneScal* out, cudaStream_t s);
cudaError_t launch_set_scal(const SceneDev* scenes, int n, const int* active,
                            const double* ls_alpha, const double* pcg_tol, cudaStream_t s);

// solver (sx_solve.cu)
cudaError_t launch_predict(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                           double* part, cudaStream_t s);
cudaError_t launch_pcg_setup_p(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                               int precision, double* part, cudaStream_t s);
// q = A p with the p.q partials per row tile; the last tile of each scene
// to finish also forms that scene's p.q and alpha (tbeg/tend: the scene's
// tile range in `row_tiles`)
cudaError_t launch_spmv_pq(const SceneDev* scenes, const Tile* row_tiles, int ntiles,
                           int precision, int parity, double* part, const int* tbeg,
                           const int* tend, cudaStream_t s);
cudaError_t launch_pcg_pdir(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                            int precision, int parity, cudaStream_t s);
int spmv_rows_per_tile();
// the SpMV's sliced copy of a pattern: per 32-row slice its longest row
// (widths[(N + 31) / 32]), then, from their exclusive prefix sum sell_ptr,
// the padded column array
cudaError_t launch_sell_widths(const int* row_ptr, int64_t N, int* widths, cudaStream_t s);
cudaError_t launch_sell_cols(const int* row_ptr, const int* col, int64_t N, const int* sell_ptr,
                             int* sell_col, cudaStream_t s);
// eight PCG iterations as a chain of kernel nodes appended to `graph`
struct PcgChunkArgs {   // (the fused kernels take the scenes' tile ranges)
    const SceneDev* scenes;
    int n_scenes;
    const Tile* node_tiles;
    int n_node_tiles;
    const Tile* row_tiles;
    int n_row_tiles;
    int precision;
    double* part_row;
    const int* row_beg;
    const int* row_end;
    double* part_node;
    const int* node_beg;
    const int* node_end;
    double tol;
    int max_iter;
};
cudaError_t add_pcg_chunk_nodes(cudaGraph_t graph, const PcgChunkArgs& a);
// dx += alpha p, r -= alpha q, z = Minv r with the r.z and r.r partials;
// the last tile of each scene forms its convergence test and beta
cudaError_t launch_pcg_update(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                              int parity, double* part, const int* tbeg, const int* tend,
                              double tol, int max_iter, cudaStream_t s);
cudaError_t launch_pcg_reduce(const double* part, int nv, const int* tbeg, const int* tend,
                              int nscenes, const SceneDev* scenes, int stage, double tol,
                              int max_iter, cudaStream_t s);
cudaError_t launch_gdx(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                       double* part, cudaStream_t s);
cudaError_t launch_trial(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                         cudaStream_t s);
cudaError_t launch_accept(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                          cudaStream_t s);
cudaError_t launch_velocity(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                            cudaStream_t s);
// x = x_start (the state at the start of the step) for the active scenes
cudaError_t launch_restore(const SceneDev* scenes, const Tile* node_tiles, int ntiles,
                           cudaStream_t s);

}  // namespace sx
