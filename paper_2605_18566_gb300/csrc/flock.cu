// flock.cu -- neighbour structure of the murmuration game: for every agent the k = 7
// nearest other agents (exact, by brute force over shared-memory tiles of positions) and
// the circular mean of their headings, psibar = atan2(sum sin psi_j, sum cos psi_j).  The
// agent game's target and Hamiltonian are built from these (games.cuh, Flock4): the
// topological interaction with a fixed number of neighbours (Appendix D.5) and the
// heading average <w>_r of Eq. DubinsJadbabaie, read as the neighbours' mean heading.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/hjg.h"
#include "dispatch.h"

namespace hjg {

constexpr int kKnnThreads = 256;
constexpr int kKnnTile = 1024;

// Exact k nearest neighbours (k = K) of each agent among all others, ordered by squared
// distance (FP32) and then by index.  One thread per query agent.  A NaN distance (a
// non-finite position on either side) never enters the list, so a slot can stay empty;
// it is written as -1.
template <int K>
__global__ void __launch_bounds__(kKnnThreads) knn_kernel(const float* __restrict__ x, int64_t ldx,
                                                          int64_t M, int32_t* __restrict__ idx) {
    __shared__ float4 tile[kKnnTile];
    const int64_t i = (int64_t)blockIdx.x * kKnnThreads + threadIdx.x;
    const bool active = i < M;
    float qx = 0.f, qy = 0.f, qz = 0.f;
    if (active) { qx = x[i * ldx]; qy = x[i * ldx + 1]; qz = x[i * ldx + 2]; }
    float bd[K];
    int32_t bi[K];
#pragma unroll
    for (int t = 0; t < K; ++t) { bd[t] = INFINITY; bi[t] = 0x7FFFFFFF; }
    for (int64_t base = 0; base < M; base += kKnnTile) {
        __syncthreads();
        for (int t = threadIdx.x; t < kKnnTile; t += kKnnThreads) {
            const int64_t j = base + t;
            tile[t] = j < M ? make_float4(x[j * ldx], x[j * ldx + 1], x[j * ldx + 2], 0.f)
                            : make_float4(INFINITY, INFINITY, INFINITY, 0.f);
        }
        __syncthreads();
        if (!active) continue;
        const int lim = (int)((M - base) < kKnnTile ? (M - base) : kKnnTile);
        for (int t = 0; t < lim; ++t) {
            const float4 p = tile[t];
            const float dx = p.x - qx, dy = p.y - qy, dz = p.z - qz;
            const float d = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const int32_t j = (int32_t)(base + t);
            if (d < bd[K - 1] || (d == bd[K - 1] && j < bi[K - 1])) {
                if (j == (int32_t)i) continue;
                float cd = d;
                int32_t cj = j;
#pragma unroll
                for (int s = 0; s < K; ++s) {   // insertion keeping (distance, index) order
                    const bool before = cd < bd[s] || (cd == bd[s] && cj < bi[s]);
                    const float td = bd[s];
                    const int32_t tj = bi[s];
                    bd[s] = before ? cd : td;
                    bi[s] = before ? cj : tj;
                    cd = before ? td : cd;
                    cj = before ? tj : cj;
                }
            }
        }
    }
    if (active)
#pragma unroll
        for (int t = 0; t < K; ++t) idx[i * K + t] = bi[t] < M ? bi[t] : -1;
}

// psibar (FP64 circular mean of the neighbours' headings, state component 3) and the
// per-agent game data: the K neighbour positions followed by psibar.  An empty slot (-1)
// gives NaN there and in psibar, so the agent's solve is reported as non-finite.
template <int K>
__global__ void flock_aux_kernel(const float* __restrict__ x, int64_t ldx, int64_t M,
                                 const int32_t* __restrict__ idx, float* __restrict__ psibar,
                                 float* __restrict__ aux, int64_t ldaux) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M) return;
    double ss = 0.0, cs = 0.0;
    bool empty = false;
    for (int t = 0; t < K; ++t) {
        const int64_t j = idx[i * K + t];
        if (j < 0 || j >= M) {
            empty = true;
            if (aux)
                for (int a = 0; a < 3; ++a) aux[i * ldaux + 3 * t + a] = NAN;
            continue;
        }
        double s, c;
        sincos((double)x[j * ldx + 3], &s, &c);
        ss += s;
        cs += c;
        if (aux)
            for (int a = 0; a < 3; ++a) aux[i * ldaux + 3 * t + a] = x[j * ldx + a];
    }
    const float pb = empty ? NAN : (float)atan2(ss, cs);
    if (psibar) psibar[i] = pb;
    if (aux) aux[i * ldaux + 3 * K] = pb;
}

cudaError_t flock_neighbours(const float* x, int64_t ldx, int64_t M, int32_t* idx, float* psibar,
                             float* aux, int64_t ldaux, cudaStream_t st) {
    if (M <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((M + kKnnThreads - 1) / kKnnThreads);
    knn_kernel<7><<<grid, kKnnThreads, 0, st>>>(x, ldx, M, idx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    flock_aux_kernel<7><<<grid, kKnnThreads, 0, st>>>(x, ldx, M, idx, psibar, aux, ldaux);
    return cudaGetLastError();
}

}  // namespace hjg

extern "C" hjg_status hjg_flock_neighbours(const float* states, int64_t M, int64_t ld, int k,
                                           int32_t* idx_out, float* psibar_out, void* stream) {
    if (k != 7 || M < 0 || M > 0x7FFFFFFFll || ld < 4) return HJG_EINVAL;
    if (M == 0) return HJG_OK;
    if (M < 8 || !states || !idx_out) return HJG_EINVAL;
    return hjg::flock_neighbours(states, ld, M, idx_out, psibar_out, nullptr, 0, (cudaStream_t)stream) ==
                   cudaSuccess
               ? HJG_OK
               : HJG_ECUDA;
}
