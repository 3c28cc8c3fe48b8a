// topology.cu -- topology markers of the zero sublevel set {v <= 0} on 2-D slices of the
// value function (the phase-transition markers of the murmuration study, Appendix D):
// for each slice, the number of connected components n_comp of the set, the number beta_1
// of holes (components of the complement that do not reach the slice border) and the Euler
// characteristic chi = n_comp - beta_1, plus the event flags of consecutive slices.
//
// The set is taken 4-connected and its complement 8-connected (the dual pair for which
// chi = n_comp - beta_1 holds on a square grid).  Before thresholding, each slice may be
// smoothed by a separable Gaussian filter (weights exp(-k^2 / (2 s^2)), |k| <= int(4 s +
// 0.5), normalised; half-sample-symmetric reflection at the border) to remove sampling
// speckle.  Connected components: union-find over all slices at once with atomicMin
// hooking (every pass is bounded: parents only decrease, and each loop has an iteration
// cap that raises an error flag instead of spinning), then path compression and counting.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/hjg.h"

namespace {

constexpr int kTopoThreads = 256;
constexpr int kFindCap = 1 << 24;   // bound on any parent walk (paths are far shorter)

__device__ __forceinline__ int reflect_index(int i, int m) {
    if (i < 0) return -i - 1;
    if (i >= m) return 2 * m - 1 - i;
    return i;
}

// One pass of the separable filter along rows (dir 0) or columns (dir 1).
__global__ void smooth_pass(const double* __restrict__ in, double* __restrict__ out, int H, int m,
                            const double* __restrict__ w, int r, int dir) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cells = (int64_t)m * m;
    if (c >= (int64_t)H * cells) return;
    const int64_t h = c / cells;
    const int i = (int)((c % cells) / m), j = (int)(c % m);
    const double* s = in + h * cells;
    double acc = 0.0;
    for (int k = -r; k <= r; ++k) {
        const int ii = dir ? reflect_index(i + k, m) : i;
        const int jj = dir ? j : reflect_index(j + k, m);
        acc = fma(w[k + r], s[(int64_t)ii * m + jj], acc);
    }
    out[c] = acc;
}

__device__ __forceinline__ int find_root(const int* __restrict__ L, int i, int* err) {
    for (int it = 0; it < kFindCap; ++it) {
        const int p = L[i];
        if (p == i) return i;
        i = p;
    }
    atomicExch(err, 1);
    return i;
}

// Hook the trees of a and b: the larger root points to the smaller.
__device__ void unite(int* L, int a, int b, int* err) {
    for (int it = 0; it < kFindCap; ++it) {
        a = find_root(L, a, err);
        b = find_root(L, b, err);
        if (a == b) return;
        if (a > b) { const int t = a; a = b; b = t; }
        const int old = atomicMin(&L[b], a);
        if (old == b) return;   // b was a root and now hangs below a
        b = old;                // b got another parent meanwhile: retry from there
    }
    atomicExch(err, 1);
}

__global__ void ccl_init(const double* __restrict__ f, int64_t n, int* __restrict__ L, uint8_t* __restrict__ fg) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    L[c] = (int)c;
    fg[c] = f[c] <= 0.0 ? 1 : 0;
}

// Set cells join their right and lower set neighbours (4-connectivity); complement cells
// join their right, lower, lower-left and lower-right complement neighbours (8).
__global__ void ccl_merge(const uint8_t* __restrict__ fg, int H, int m, int* L, int* err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cells = (int64_t)m * m;
    if (c >= (int64_t)H * cells) return;
    const int i = (int)((c % cells) / m), j = (int)(c % m);
    const uint8_t k = fg[c];
    if (j + 1 < m && fg[c + 1] == k) unite(L, (int)c, (int)(c + 1), err);
    if (i + 1 < m) {
        if (fg[c + m] == k) unite(L, (int)c, (int)(c + m), err);
        if (!k) {
            if (j > 0 && fg[c + m - 1] == 0) unite(L, (int)c, (int)(c + m - 1), err);
            if (j + 1 < m && fg[c + m + 1] == 0) unite(L, (int)c, (int)(c + m + 1), err);
        }
    }
}

__global__ void ccl_compress(int* L, int64_t n, int* err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    L[c] = find_root(L, (int)c, err);
}

// Complement components that reach the border are not holes: flag their roots.
__global__ void mark_border(const uint8_t* __restrict__ fg, const int* __restrict__ L, int H, int m,
                            uint8_t* __restrict__ border) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = 4 * (int64_t)m;
    if (t >= (int64_t)H * per) return;
    const int64_t h = t / per;
    const int e = (int)(t % per), side = e / m, q = e % m;
    const int i = side == 0 ? 0 : side == 1 ? m - 1 : q;
    const int j = side == 0 || side == 1 ? q : side == 2 ? 0 : m - 1;
    const int64_t c = h * (int64_t)m * m + (int64_t)i * m + j;
    if (!fg[c]) border[L[c]] = 1;
}

__global__ void count_roots(const uint8_t* __restrict__ fg, const int* __restrict__ L,
                            const uint8_t* __restrict__ border, int H, int m, int* __restrict__ ncomp,
                            int* __restrict__ holes) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t cells = (int64_t)m * m;
    if (c >= (int64_t)H * cells || L[c] != (int)c) return;
    const int64_t h = c / cells;
    if (fg[c]) atomicAdd(&ncomp[h], 1);
    else if (!border[c]) atomicAdd(&holes[h], 1);
}

unsigned blocks(int64_t n) { return (unsigned)((n + kTopoThreads - 1) / kTopoThreads); }

}  // namespace

extern "C" hjg_status hjg_topology(const double* v, int H, int m, double smooth_cells, double* smoothed_out,
                                   int32_t* markers_out, int32_t* events_out, int32_t* labels_out, void* stream) {
    if (H < 0 || m < 0 || (H > 0 && m > 0 && (!v || !markers_out)) || !(smooth_cells >= 0.0) ||
        (int64_t)H * m * m > 0x7FFFFFFFll)
        return HJG_EINVAL;
    const int r = smooth_cells > 0.0 ? (int)(4.0 * smooth_cells + 0.5) : 0;
    if (r >= m && smooth_cells > 0.0) return HJG_EINVAL;   // reflection needs a radius below the slice width
    if (H == 0 || m == 0) return HJG_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = (int64_t)H * m * m;
    double *f = nullptr, *tmp = nullptr, *w = nullptr;
    int *L = nullptr, *cnt = nullptr, *err = nullptr;
    uint8_t *fg = nullptr, *border = nullptr;
    hjg_status status = HJG_OK;
    auto ok = [&](cudaError_t e) {
        if (e != cudaSuccess && status == HJG_OK) status = (e == cudaErrorMemoryAllocation) ? HJG_ENOMEM : HJG_ECUDA;
        return status == HJG_OK;
    };
    if (ok(cudaMallocAsync((void**)&f, n * sizeof(double), st)) && ok(cudaMallocAsync((void**)&L, n * sizeof(int), st)) &&
        ok(cudaMallocAsync((void**)&fg, n, st)) && ok(cudaMallocAsync((void**)&border, n, st)) &&
        ok(cudaMallocAsync((void**)&cnt, 2 * (size_t)H * sizeof(int), st)) &&
        ok(cudaMallocAsync((void**)&err, sizeof(int), st)) && ok(cudaMemsetAsync(border, 0, n, st)) &&
        ok(cudaMemsetAsync(cnt, 0, 2 * (size_t)H * sizeof(int), st)) && ok(cudaMemsetAsync(err, 0, sizeof(int), st))) {
        if (r > 0) {
            std::vector<double> hw(2 * r + 1);
            double sum = 0.0;
            for (int k = -r; k <= r; ++k) sum += (hw[k + r] = std::exp(-0.5 * (double)k * k / (smooth_cells * smooth_cells)));
            for (double& x : hw) x /= sum;
            if (ok(cudaMallocAsync((void**)&tmp, n * sizeof(double), st)) &&
                ok(cudaMallocAsync((void**)&w, hw.size() * sizeof(double), st)) &&
                ok(cudaMemcpyAsync(w, hw.data(), hw.size() * sizeof(double), cudaMemcpyHostToDevice, st))) {
                smooth_pass<<<blocks(n), kTopoThreads, 0, st>>>(v, tmp, H, m, w, r, 0);
                smooth_pass<<<blocks(n), kTopoThreads, 0, st>>>(tmp, f, H, m, w, r, 1);
                ok(cudaGetLastError());
            }
        } else {
            ok(cudaMemcpyAsync(f, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        }
        if (status == HJG_OK) {
            ccl_init<<<blocks(n), kTopoThreads, 0, st>>>(f, n, L, fg);
            ccl_merge<<<blocks(n), kTopoThreads, 0, st>>>(fg, H, m, L, err);
            ccl_compress<<<blocks(n), kTopoThreads, 0, st>>>(L, n, err);
            mark_border<<<blocks(4 * (int64_t)H * m), kTopoThreads, 0, st>>>(fg, L, H, m, border);
            count_roots<<<blocks(n), kTopoThreads, 0, st>>>(fg, L, border, H, m, cnt, cnt + H);
            ok(cudaGetLastError());
        }
        std::vector<int> hc(2 * (size_t)H);
        int herr = 0;
        if (status == HJG_OK && ok(cudaMemcpyAsync(hc.data(), cnt, hc.size() * sizeof(int), cudaMemcpyDeviceToHost, st)) &&
            ok(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st))) {
            if (smoothed_out) ok(cudaMemcpyAsync(smoothed_out, f, n * sizeof(double), cudaMemcpyDefault, st));
            if (labels_out) ok(cudaMemcpyAsync(labels_out, L, n * sizeof(int), cudaMemcpyDefault, st));
            if (ok(cudaStreamSynchronize(st))) {
                if (herr) {
                    status = HJG_ETIMEOUT;
                } else {
                    for (int h = 0; h < H; ++h) {
                        markers_out[3 * h] = hc[h];                       // n_comp
                        markers_out[3 * h + 1] = hc[H + h];               // beta_1
                        markers_out[3 * h + 2] = hc[h] - hc[H + h];       // chi
                    }
                    if (events_out) {
                        for (int h = 0; h < H; ++h) {
                            int e = 0;
                            if (h > 0) {
                                const int* a = markers_out + 3 * (h - 1);
                                const int* b = markers_out + 3 * h;
                                if ((double)(b[2] - a[2]) < -0.5) e |= HJG_EVENT_VACUOLE;
                                if (b[1] >= 1 && a[1] == 0) e |= HJG_EVENT_CORDON;
                                if (b[0] > a[0]) e |= HJG_EVENT_FRAGMENTATION;
                            }
                            events_out[h] = e;
                        }
                    }
                }
            }
        }
    }
    for (void* p : {(void*)f, (void*)tmp, (void*)w, (void*)L, (void*)cnt, (void*)err, (void*)fg, (void*)border})
        if (p) cudaFreeAsync(p, st);
    return status;
}
