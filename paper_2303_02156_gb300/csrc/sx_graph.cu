// sx_graph.cu -- scene registration and the fixed sparsity structure.
//
// Rest precompute of the Stable Neo-Hookean tets (App. A linear tet4;
// App. B density parameters) and the 3x3 block CRS pattern of §5.3
// (Eq. 11): the union of every stencil's node pairs plus every diagonal,
// columns ascending, full storage; the per-stencil slot maps (BSR block of
// local pair (a, b)); and the element-id-ordered lists that let the
// assembly kernels gather instead of scatter (no atomics in the per-step
// path). Every output here is an exact integer function of the
// connectivity, so it is bit-identical from run to run even though
// atomics are used while counting.
#include <cuda_runtime.h>

#include <string>

#include "sx_internal.cuh"

namespace sx {

static inline int nblk(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ------------------------------------------------------------------ rest
__global__ void k_snh_rest(const double* X, int64_t N, const int4* tets, int64_t n,
                           const double* young,
                           const double* poisson, int literal, double* Dminv, double* V,
                           double* mu, double* lam, int* bad)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    int4 t = tets[e];
    const int id[4] = {t.x, t.y, t.z, t.w};
    for (int a = 0; a < 4; ++a)
        if (id[a] < 0 || id[a] >= N) {
            atomicAdd(bad + 1, 1);
            return;
        }
    double D[3][3];   // D[i][k] = X_{k+1,i} - X_{0,i}
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 3; ++i) D[i][k] = X[3 * (int64_t)id[k + 1] + i] - X[3 * (int64_t)id[0] + i];
    // inverse through the adjugate: rows of D^-1 are cross products of the
    // columns of D divided by det D
    double c0[3] = {D[0][0], D[1][0], D[2][0]};
    double c1[3] = {D[0][1], D[1][1], D[2][1]};
    double c2[3] = {D[0][2], D[1][2], D[2][2]};
    double r0[3] = {c1[1] * c2[2] - c1[2] * c2[1], c1[2] * c2[0] - c1[0] * c2[2],
                    c1[0] * c2[1] - c1[1] * c2[0]};
    double r1[3] = {c2[1] * c0[2] - c2[2] * c0[1], c2[2] * c0[0] - c2[0] * c0[2],
                    c2[0] * c0[1] - c2[1] * c0[0]};
    double r2[3] = {c0[1] * c1[2] - c0[2] * c1[1], c0[2] * c1[0] - c0[0] * c1[2],
                    c0[0] * c1[1] - c0[1] * c1[0]};
    double det = c0[0] * r0[0] + c0[1] * r0[1] + c0[2] * r0[2];
    if (!(det > 0.0)) atomicAdd(bad, 1);
    double id_ = 1.0 / det;
    for (int j = 0; j < 3; ++j) {
        Dminv[(int64_t)(0 * 3 + j) * n + e] = r0[j] * id_;
        Dminv[(int64_t)(1 * 3 + j) * n + e] = r1[j] * id_;
        Dminv[(int64_t)(2 * 3 + j) * n + e] = r2[j] * id_;
    }
    V[e] = det / 6.0;
    double Ey = young[e], nu = poisson[e];
    double m = Ey / (2.0 * (1.0 + nu));
    double l = Ey * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    if (literal) {
        mu[e] = m;
        lam[e] = l;
    } else {
        mu[e] = m * (4.0 / 3.0);
        lam[e] = l + m * (5.0 / 6.0);
    }
}

cudaError_t launch_snh_rest(const double* X, int64_t N, const int4* tets, int64_t n,
                            const double* young, const double* poisson, double rho,
                            int literal, double* Dminv, double* V, double* mu,
                            double* lam, int* bad, cudaStream_t s)
{
    (void)rho;
    if (n == 0) return cudaSuccess;
    k_snh_rest<<<nblk(n, 256), 256, 0, s>>>(X, N, tets, n, young, poisson, literal, Dminv, V,
                                            mu, lam, bad);
    return cudaGetLastError();
}

// mass[n] += sum over incident tets (element order) of rho V / 4
__global__ void k_tet_mass(const int* node_ptr, const int* node_src, int64_t N,
                           int64_t base, int64_t cnt, const double* V, double rho,
                           double* mass)
{
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= N) return;
    double s = 0.0;
    for (int k = node_ptr[n]; k < node_ptr[n + 1]; ++k) {
        int64_t st = node_src[k] >> 2;
        if (st >= base && st < base + cnt) s += rho * V[st - base] * 0.25;
    }
    mass[n] += s;
}

cudaError_t launch_block_mass(const int* node_ptr, const int* node_src, int64_t N,
                              int64_t base, int64_t cnt, const double* V, double rho,
                              double* mass, cudaStream_t s)
{
    if (N == 0) return cudaSuccess;
    k_tet_mass<<<nblk(N, 256), 256, 0, s>>>(node_ptr, node_src, N, base, cnt, V, rho, mass);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ scan
// exclusive prefix sum of int32 counts into int32 offsets (total < 2^31),
// out has n+1 entries. Three-phase: tile scans, recursive scan of tile
// sums, add-back.
static constexpr int kScanT = 512;

__global__ void k_scan_tiles(const int* in, int64_t n, int* out, int* tile_sums)
{
    __shared__ int sh[kScanT];
    int64_t i = blockIdx.x * (int64_t)kScanT + threadIdx.x;
    int v = (i < n) ? in[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int off = 1; off < kScanT; off <<= 1) {
        int t = (threadIdx.x >= (unsigned)off) ? sh[threadIdx.x - off] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = sh[threadIdx.x] - v;   // exclusive
    if (threadIdx.x == kScanT - 1) tile_sums[blockIdx.x] = sh[threadIdx.x];
}

__global__ void k_scan_add(int* out, int64_t n, const int* tile_off)
{
    int64_t i = blockIdx.x * (int64_t)kScanT + threadIdx.x;
    if (i < n) out[i] += tile_off[blockIdx.x];
}

__global__ void k_set_last(int* out, int64_t n, const int* in)
{
    // out[n] = out[n-1] + in[n-1]
    if (n == 0) out[0] = 0;
    else out[n] = out[n - 1] + in[n - 1];
}

static int exclusive_scan(const int* in, int64_t n, int* out, cudaStream_t s,
                          std::string* err)
{
    if (n == 0) {
        cudaMemsetAsync(out, 0, sizeof(int), s);
        return SX_OK;
    }
    int64_t nt = (n + kScanT - 1) / kScanT;
    int* sums = nullptr;
    int* offs = nullptr;
    if (cudaMallocAsync((void**)&sums, nt * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&offs, (nt + 1) * sizeof(int), s) != cudaSuccess) {
        *err = "scan: device allocation failed";
        return SX_ENOMEM;
    }
    k_scan_tiles<<<(unsigned)nt, kScanT, 0, s>>>(in, n, out, sums);
    if (nt > 1) {
        int rc = exclusive_scan(sums, nt, offs, s, err);
        if (rc != SX_OK) return rc;
        k_scan_add<<<(unsigned)nt, kScanT, 0, s>>>(out, n, offs);
    }
    k_set_last<<<1, 1, 0, s>>>(out, n, in);
    cudaFreeAsync(sums, s);
    cudaFreeAsync(offs, s);
    return cudaGetLastError() == cudaSuccess ? SX_OK : SX_ECUDA;
}

int scan_counts(const int* in, int64_t n, int* out, cudaStream_t s, std::string* err)
{
    return exclusive_scan(in, n, out, s, err);
}

// ------------------------------------------------------------------ incidence
__global__ void k_count_nodes(const int4* conn, int64_t nst, int* deg)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nst) return;
    int4 t = conn[e];
    atomicAdd(&deg[t.x], 1);
    atomicAdd(&deg[t.y], 1);
    atomicAdd(&deg[t.z], 1);
    atomicAdd(&deg[t.w], 1);
}

__global__ void k_fill_nodes(const int4* conn, int64_t nst, const int* ptr, int* fill, int* src)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nst) return;
    int4 t = conn[e];
    const int id[4] = {t.x, t.y, t.z, t.w};
    for (int a = 0; a < 4; ++a) {
        int p = atomicAdd(&fill[id[a]], 1);
        src[ptr[id[a]] + p] = (int)(4 * e + a);
    }
}

// sort each segment ascending (insertion sort; segments are short)
__global__ void k_sort_segments(const int* ptr, int64_t nseg, int* v)
{
    int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int b = ptr[s], e = ptr[s + 1];
    for (int i = b + 1; i < e; ++i) {
        int key = v[i];
        int j = i - 1;
        while (j >= b && v[j] > key) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = key;
    }
}

__global__ void k_check_ids(const int4* conn, int64_t nst, int64_t N, int* bad)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nst) return;
    int4 t = conn[e];
    if (t.x < 0 || t.x >= N || t.y < 0 || t.y >= N || t.z < 0 || t.z >= N || t.w < 0 ||
        t.w >= N)
        atomicAdd(bad, 1);
}

int build_incidence(const int4* conn, int64_t nst, int64_t N, int** ptr_out, int** src_out,
                    std::string* err, cudaStream_t s)
{
    int *deg = nullptr, *ptr = nullptr, *src = nullptr, *fill = nullptr;
    if (cudaMallocAsync((void**)&deg, N * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&ptr, (N + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&src, (4 * nst + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&fill, N * sizeof(int), s) != cudaSuccess) {
        *err = "incidence: device allocation failed";
        for (void* p : {(void*)deg, (void*)ptr, (void*)src, (void*)fill})
            if (p) cudaFreeAsync(p, s);
        return SX_ENOMEM;
    }
    cudaMemsetAsync(deg, 0, N * sizeof(int), s);
    cudaMemsetAsync(fill, 0, N * sizeof(int), s);
    if (nst) k_count_nodes<<<nblk(nst, 256), 256, 0, s>>>(conn, nst, deg);
    int rc = exclusive_scan(deg, N, ptr, s, err);
    if (rc != SX_OK) return rc;
    if (nst) k_fill_nodes<<<nblk(nst, 256), 256, 0, s>>>(conn, nst, ptr, fill, src);
    if (N) k_sort_segments<<<nblk(N, 128), 128, 0, s>>>(ptr, N, src);
    cudaFreeAsync(deg, s);
    cudaFreeAsync(fill, s);
    *ptr_out = ptr;
    *src_out = src;
    return cudaGetLastError() == cudaSuccess ? SX_OK : SX_ECUDA;
}

// ------------------------------------------------------------------ pattern
// candidate columns of row n: n itself and every node of every incident
// stencil; sorted and deduplicated in place, row_len[n] = unique count
__global__ void k_row_candidates(const int4* conn, const int* node_ptr, const int* node_src,
                                 int64_t N, int* cand, int* row_len)
{
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= N) return;
    int b = node_ptr[n], e = node_ptr[n + 1];
    int64_t off = 4 * (int64_t)b + n;
    int len = 0;
    cand[off + len++] = (int)n;
    for (int k = b; k < e; ++k) {
        int st = node_src[k] >> 2;
        int4 t = conn[st];
        cand[off + len++] = t.x;
        cand[off + len++] = t.y;
        cand[off + len++] = t.z;
        cand[off + len++] = t.w;
    }
    int* v = cand + off;
    for (int i = 1; i < len; ++i) {
        int key = v[i];
        int j = i - 1;
        while (j >= 0 && v[j] > key) {
            v[j + 1] = v[j];
            --j;
        }
        v[j + 1] = key;
    }
    int u = 0;
    for (int i = 0; i < len; ++i)
        if (i == 0 || v[i] != v[i - 1]) v[u++] = v[i];
    row_len[n] = u;
}

__global__ void k_row_copy(const int* node_ptr, int64_t N, const int* cand, const int* row_ptr,
                           int* col)
{
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= N) return;
    int64_t off = 4 * (int64_t)node_ptr[n] + n;
    int b = row_ptr[n], e = row_ptr[n + 1];
    for (int k = b; k < e; ++k) col[k] = cand[off + (k - b)];
}

__device__ __forceinline__ int find_col(const int* row_ptr, const int* col, int r, int c)
{
    int lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int mid = (lo + hi) >> 1;
        int v = col[mid];
        if (v == c) return mid;
        if (v < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

__global__ void k_slots(const int4* conn, int64_t nst, const int* row_ptr, const int* col,
                        int* slots, int* slot_deg)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nst) return;
    int4 t = conn[e];
    const int id[4] = {t.x, t.y, t.z, t.w};
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
            int s = find_col(row_ptr, col, id[a], id[b]);
            slots[16 * e + 4 * a + b] = s;
            if (s >= 0) atomicAdd(&slot_deg[s], 1);
        }
}

__global__ void k_diag_slots(const int* row_ptr, const int* col, int64_t N, int* diag)
{
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= N) return;
    diag[n] = find_col(row_ptr, col, (int)n, (int)n);
}

__global__ void k_fill_slots(const int* slots, int64_t nst, const int* slot_ptr, int* fill,
                             int* src)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= nst) return;
    for (int k = 0; k < 16; ++k) {
        int s = slots[16 * e + k];
        if (s < 0) continue;
        int p = atomicAdd(&fill[s], 1);
        src[slot_ptr[s] + p] = (int)(16 * e + k);
    }
}

// Within each tile of kSlotTile consecutive blocks, the blocks ordered by
// ascending contributor count (ties by block index): the assembly threads
// of a warp then walk lists of similar length. Only which thread sums a
// block changes; each block's own summation order stays element order.
__global__ void __launch_bounds__(kSlotTile)
k_slot_order(const int* slot_ptr, int64_t nnz, int* order)
{
    __shared__ int len[kSlotTile];
    const int64_t t0 = (int64_t)blockIdx.x * kSlotTile;
    const int cnt = (nnz - t0 < (int64_t)kSlotTile) ? (int)(nnz - t0) : kSlotTile;
    const int i = threadIdx.x;
    len[i] = i < cnt ? slot_ptr[t0 + i + 1] - slot_ptr[t0 + i] : 0;
    __syncthreads();
    if (i >= cnt) return;
    const int li = len[i];
    int rank = 0;
    for (int j = 0; j < cnt; ++j) {
        const int lj = len[j];
        rank += (lj < li || (lj == li && j < i)) ? 1 : 0;
    }
    order[t0 + rank] = (int)(t0 + i);
}

int build_pattern(const int4* conn, int64_t nst, int64_t N, PatternOut* out,
                  std::string* err, cudaStream_t s)
{
    PatternOut P{};
    int rc;
    {
        int* bad = nullptr;
        cudaMallocAsync((void**)&bad, sizeof(int), s);
        cudaMemsetAsync(bad, 0, sizeof(int), s);
        if (nst) k_check_ids<<<nblk(nst, 256), 256, 0, s>>>(conn, nst, N, bad);
        int h = 0;
        cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        cudaFreeAsync(bad, s);
        if (h) {
            *err = "finalize: a stencil references a node id outside [0, n_nodes)";
            return SX_EINVAL;
        }
    }
    if (16 * nst + N >= (int64_t)INT32_MAX) {
        *err = "finalize: scene too large for int32 assembly lists";
        return SX_EINVAL;
    }
    rc = build_incidence(conn, nst, N, &P.node_ptr, &P.node_src, err, s);
    if (rc != SX_OK) return rc;
    // candidate rows
    int *cand = nullptr, *row_len = nullptr;
    if (cudaMallocAsync((void**)&cand, (16 * nst + N) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&row_len, N * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P.row_ptr, (N + 1) * sizeof(int), s) != cudaSuccess) {
        *err = "finalize: device allocation failed (pattern)";
        return SX_ENOMEM;
    }
    if (N) k_row_candidates<<<nblk(N, 128), 128, 0, s>>>(conn, P.node_ptr, P.node_src, N, cand,
                                                         row_len);
    rc = exclusive_scan(row_len, N, P.row_ptr, s, err);
    if (rc != SX_OK) return rc;
    int nnz = 0;
    cudaMemcpyAsync(&nnz, P.row_ptr + N, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    P.nnzb = nnz;
    // padded: staged SpMV tiles read 16-byte aligned windows
    if (cudaMallocAsync((void**)&P.col, (nnz + 16) * sizeof(int), s) != cudaSuccess) {
        *err = "finalize: device allocation failed (col)";
        return SX_ENOMEM;
    }
    if (N) k_row_copy<<<nblk(N, 256), 256, 0, s>>>(P.node_ptr, N, cand, P.row_ptr, P.col);
    cudaFreeAsync(cand, s);
    cudaFreeAsync(row_len, s);
    // slots, diagonal slots, slot contributor lists
    int *slot_deg = nullptr, *fill = nullptr;
    if (cudaMallocAsync((void**)&P.slots, (16 * nst + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P.diag_slot, N * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&slot_deg, (nnz + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&fill, (nnz + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P.slot_ptr, (nnz + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P.slot_src, (16 * nst + 1) * sizeof(int), s) != cudaSuccess ||
        cudaMallocAsync((void**)&P.slot_order, (nnz + 1) * sizeof(int), s) != cudaSuccess) {
        *err = "finalize: device allocation failed (slots)";
        return SX_ENOMEM;
    }
    cudaMemsetAsync(slot_deg, 0, (nnz + 1) * sizeof(int), s);
    cudaMemsetAsync(fill, 0, (nnz + 1) * sizeof(int), s);
    if (nst) k_slots<<<nblk(nst, 256), 256, 0, s>>>(conn, nst, P.row_ptr, P.col, P.slots, slot_deg);
    if (N) k_diag_slots<<<nblk(N, 256), 256, 0, s>>>(P.row_ptr, P.col, N, P.diag_slot);
    rc = exclusive_scan(slot_deg, nnz, P.slot_ptr, s, err);
    if (rc != SX_OK) return rc;
    if (nst) k_fill_slots<<<nblk(nst, 256), 256, 0, s>>>(P.slots, nst, P.slot_ptr, fill, P.slot_src);
    if (nnz) k_sort_segments<<<nblk(nnz, 128), 128, 0, s>>>(P.slot_ptr, nnz, P.slot_src);
    if (nnz) k_slot_order<<<nblk(nnz, kSlotTile), kSlotTile, 0, s>>>(P.slot_ptr, nnz, P.slot_order);
    cudaFreeAsync(slot_deg, s);
    cudaFreeAsync(fill, s);
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        *err = "finalize: kernel failure while building the pattern";
        return SX_ECUDA;
    }
    *out = P;
    return SX_OK;
}

}  // namespace sx
