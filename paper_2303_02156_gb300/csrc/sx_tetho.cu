// sx_tetho.cu -- rest precompute and host tables of the high-order Lagrange
// tets (§6.2 Eq. 12; App. A shape functions): reference shape
// gradients at the quadrature points, J0^-1 and w det J0 per element and
// point, and the cover of an element's node pairs by 4-node sub-stencils
// through which the fixed-pattern assembly takes its blocks.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "sx_internal.cuh"

namespace sx {

namespace {

// edges and faces of the reference tet in the local node order
constexpr int kEdge[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};
constexpr int kFace[4][3] = {{0, 1, 2}, {0, 1, 3}, {1, 2, 3}, {0, 2, 3}};

}  // namespace

// Reference gradients dN (K x 3) at xi of the Lagrange tet of K = 4, 10 or
// 20 nodes, through the barycentric coordinates L = (1 - xi0 - xi1 - xi2,
// xi0, xi1, xi2): dN_a/dxi_m = sum_v (dN_a/dL_v) (dL_v/dxi_m), with
// dL_0/dxi = (-1, -1, -1) and dL_v/dxi = e_{v-1} otherwise. The shape
// functions: order 1 L_v; order 2 L_v (2 L_v - 1) at the vertices and
// 4 L_i L_j at the edge nodes; order 3 (1/2) L_v (3 L_v - 1)(3 L_v - 2) at
// the vertices, (9/2) L_i L_j (3 L_i - 1) at the edge node nearer i, and
// 27 L_i L_j L_k at the face nodes.
void tetho_ref_grads(int K, const double* xi, double* dN)
{
    const double L[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
    double dl[kHoMaxK][4] = {};
    int a = 0;
    if (K == 4) {
        for (int v = 0; v < 4; ++v) dl[a++][v] = 1.0;
    } else if (K == 10) {
        for (int v = 0; v < 4; ++v) dl[a++][v] = 4.0 * L[v] - 1.0;
        for (int e = 0; e < 6; ++e, ++a) {
            dl[a][kEdge[e][0]] = 4.0 * L[kEdge[e][1]];
            dl[a][kEdge[e][1]] = 4.0 * L[kEdge[e][0]];
        }
    } else {
        for (int v = 0; v < 4; ++v) dl[a++][v] = 13.5 * L[v] * L[v] - 9.0 * L[v] + 1.0;
        for (int e = 0; e < 6; ++e)
            for (int side = 0; side < 2; ++side, ++a) {
                const int i = kEdge[e][side], j = kEdge[e][1 - side];
                dl[a][i] = 4.5 * L[j] * (6.0 * L[i] - 1.0);
                dl[a][j] = 4.5 * L[i] * (3.0 * L[i] - 1.0);
            }
        for (int f = 0; f < 4; ++f, ++a) {
            const int i = kFace[f][0], j = kFace[f][1], k = kFace[f][2];
            dl[a][i] = 27.0 * L[j] * L[k];
            dl[a][j] = 27.0 * L[i] * L[k];
            dl[a][k] = 27.0 * L[i] * L[j];
        }
    }
    for (int b = 0; b < K; ++b)
        for (int m = 0; m < 3; ++m) dN[3 * b + m] = dl[b][m + 1] - dl[b][0];
}

// Greedy cover of the K (K - 1)/2 node pairs of an element by 4-node
// sub-stencils: take the first uncovered pair, add the two nodes that
// cover the most further uncovered pairs (lowest id on ties). own[s]:
// bit up_index(a, b) when sub-stencil s is the first to hold the pair of
// its local nodes (a, b) (for a = b: the first to hold the node), bit
// 10 + a when it is the first to hold node a. Returns S.
int tetho_cover(int K, std::vector<int>& sub, std::vector<int>& own)
{
    std::vector<char> cov(K * K, 0);
    sub.clear();
    own.clear();
    for (;;) {
        int p = -1, q = -1;
        for (int i = 0; i < K && p < 0; ++i)
            for (int j = i + 1; j < K; ++j)
                if (!cov[i * K + j]) {
                    p = i;
                    q = j;
                    break;
                }
        if (p < 0) break;
        int ch[4] = {p, q, -1, -1};
        for (int c = 2; c < 4; ++c) {
            int best = -1, bs = -1;
            for (int r = 0; r < K; ++r) {
                bool used = false;
                for (int t = 0; t < c; ++t) used |= ch[t] == r;
                if (used) continue;
                int sc = 0;
                for (int t = 0; t < c; ++t) {
                    const int lo = std::min(r, ch[t]), hi = std::max(r, ch[t]);
                    sc += !cov[lo * K + hi];
                }
                if (sc > bs) {
                    bs = sc;
                    best = r;
                }
            }
            ch[c] = best;
        }
        for (int t = 0; t < 4; ++t)
            for (int u = t + 1; u < 4; ++u) {
                const int lo = std::min(ch[t], ch[u]), hi = std::max(ch[t], ch[u]);
                cov[lo * K + hi] = 1;
            }
        for (int t = 0; t < 4; ++t) sub.push_back(ch[t]);
    }
    const int S = (int)sub.size() / 4;
    std::vector<char> pair_done(K * K, 0), node_done(K, 0);
    for (int s = 0; s < S; ++s) {
        int bits = 0;
        const int* l = &sub[4 * s];
        for (int a = 0; a < 4; ++a) {
            if (!node_done[l[a]]) {
                node_done[l[a]] = 1;
                bits |= 1 << (10 + a);
                bits |= 1 << up_index(a, a);
            }
            for (int b = a + 1; b < 4; ++b) {
                const int lo = std::min(l[a], l[b]), hi = std::max(l[a], l[b]);
                if (!pair_done[lo * K + hi]) {
                    pair_done[lo * K + hi] = 1;
                    bits |= 1 << up_index(a, b);
                }
            }
        }
        own.push_back(bits);
    }
    return S;
}

// per element: node-id check, then at every point J0 = sum_a X_a dN_a^T,
// its inverse (adjugate / det), w det J0, and the volume sum_q w det J0
__global__ void k_tetho_rest(const double* __restrict__ X, int64_t N, const int* __restrict__ conn,
                             int64_t n, int K, int nq, const double* __restrict__ rule_w,
                             const double* __restrict__ dN, double* __restrict__ Jinv,
                             double* __restrict__ wdet, double* __restrict__ vol, int* bad)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    for (int a = 0; a < K; ++a) {
        const int id = conn[(int64_t)a * n + e];
        if (id < 0 || id >= N) {
            atomicAdd(bad + 1, 1);
            return;
        }
    }
    double V = 0.0;
    bool ok = true;
    for (int q = 0; q < nq; ++q) {
        double J[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int a = 0; a < K; ++a) {
            const double* p = X + 3 * (int64_t)conn[(int64_t)a * n + e];
            const double* d = dN + (q * K + a) * 3;
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) J[3 * i + j] = fma(p[i], d[j], J[3 * i + j]);
        }
        const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8],
                     c02 = J[3] * J[7] - J[4] * J[6];
        const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
        if (!(det > 0.0)) ok = false;
        const double id = 1.0 / det;
        const double inv[9] = {c00 * id, (J[2] * J[7] - J[1] * J[8]) * id,
                               (J[1] * J[5] - J[2] * J[4]) * id, c01 * id,
                               (J[0] * J[8] - J[2] * J[6]) * id, (J[2] * J[3] - J[0] * J[5]) * id,
                               c02 * id, (J[1] * J[6] - J[0] * J[7]) * id,
                               (J[0] * J[4] - J[1] * J[3]) * id};
        for (int k = 0; k < 9; ++k) Jinv[((int64_t)q * 9 + k) * n + e] = inv[k];
        wdet[(int64_t)q * n + e] = rule_w[q] * det;
        V += rule_w[q] * det;
    }
    vol[e] = V;
    if (!ok) atomicAdd(bad, 1);
}

cudaError_t launch_tetho_rest(const double* X, int64_t N, const int* conn, int64_t n, int K,
                              int nq, const double* rule_w, const double* dN, double* Jinv,
                              double* wdet, double* vol, int* bad, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_tetho_rest<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(X, N, conn, n, K, nq, rule_w, dN,
                                                             Jinv, wdet, vol, bad);
    return cudaGetLastError();
}

}  // namespace sx
