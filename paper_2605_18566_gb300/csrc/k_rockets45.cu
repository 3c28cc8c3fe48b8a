// Sweep kernels for the 15-agent multi-rocket game (Section 3.2), n = 45,
// two lanes per sample stream, and its control-variate kernel (tilted frame).
#include "dispatch.h"

namespace hjg {
namespace {
// KIND bit 1: the software-pipelined sampler; bits 2-3: the Philox multiply form (0 separate
// high and low multiplies, 1 widening, 2 one of each per round).
template <int KIND, int T, int B>
cudaError_t launch(const SweepArgs& A, bool tilt, int grid, cudaStream_t st) {
    constexpr bool P = (KIND & 2) != 0;
    constexpr int F = (KIND >> 2) & 3;
    if (tilt) sweep_kernel_r45<T, B, true, false, P, F><<<grid, T, 0, st>>>(A);
    else sweep_kernel_r45<T, B, false, false, P, F><<<grid, T, 0, st>>>(A);
    return cudaGetLastError();
}
template <int KIND, int T, int B>
int occupancy(bool tilt) {
    constexpr bool P = (KIND & 2) != 0;
    constexpr int F = (KIND >> 2) & 3;
    int nb = 0;
    if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_r45<T, B, true, false, P, F>, T, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_r45<T, B, false, false, P, F>, T, 0);
    return nb;
}
#define R45_LAUNCH(i, KIND, T, B) case i: return launch<KIND, T, B>(A, tilt, grid, st);
#define R45_OCC(i, KIND, T, B) case i: return occupancy<KIND, T, B>(tilt);
// The control-variate kernel (tilted frame only): 128 threads, 3 CTAs per SM (its ~166
// registers fit the 170 that bound allows; at 256 threads and one CTA per SM only 8 warps
// were resident).
cudaError_t sweep(const SweepArgs& A, bool tilt, int v, int grid, cudaStream_t st) {
    if (v == kCvVariant) {
        if (!tilt) return cudaErrorInvalidValue;
        sweep_kernel_r45<128, 3, true, true><<<grid, 128, 0, st>>>(A);
        return cudaGetLastError();
    }
    switch (v) { HJG_R45_VARIANTS(R45_LAUNCH) }
    return cudaErrorInvalidValue;
}
int occ(bool tilt, int v) {
    if (v == kCvVariant) {
        int nb = 0;
        if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_r45<128, 3, true, true>, 128, 0);
        return nb;
    }
    switch (v) { HJG_R45_VARIANTS(R45_OCC) }
    return 0;
}
}  // namespace
static_assert(kNumR45Variants <= kCvVariant, "the 45-D launch variants must not reach the control-variate slot");
GameKernels kernels_rockets45() {
    GameKernels k{};
    k.n = 45;
    k.nvariants = kNumR45Variants;
    HJG_R45_VARIANTS(HJG_FILL)
    k.threads[kCvVariant] = 128; k.minb[kCvVariant] = 3; k.per_warp[kCvVariant] = 0;
    k.has_cv = true;
    k.cv_tilt_only = true;
    k.sweep = sweep;
    k.occupancy = occ;
    k.init = launch_init<Rockets45>;
    k.coef = launch_coef<Rockets45>;
    k.delta = launch_delta<Rockets45>;
    return k;
}
}  // namespace hjg
