// Sweep kernels for the quadratic test problems (H = +-|p|^2/2 or H = 0, quadratic
// target), n in {1, 2, 3, 4, 6, 8}: the exact Cole-Hopf case of Corollary B.2 and the
// pure heat equation, used to check the estimator against closed forms.  One launch
// variant (128 threads) and the control-variate kernel.
#include "dispatch.h"

namespace hjg {
namespace {
template <class G>
cudaError_t sweep(const SweepArgs& A, bool tilt, int v, int grid, cudaStream_t st) {
    if (v == kCvVariant) return launch_sweep_cv<G>(A, tilt, grid, st);
    if (v == kF64Variant) return launch_sweep_f64<G>(A, tilt, grid, st);
    if (v != 0) return cudaErrorInvalidValue;
    return launch_sweep_generic<G, 0, 128, 1>(A, tilt, grid, st);
}
template <class G>
int occ(bool tilt, int v) {
    if (v == kCvVariant) return occupancy_cv<G>(tilt);
    if (v == kF64Variant) return occupancy_f64<G>(tilt);
    return v == 0 ? occupancy_generic<G, 0, 128, 1>(tilt) : 0;
}
template <int N, bool Z>
GameKernels make() {
    using G = Quadratic<N, Z>;
    GameKernels k{};
    k.n = N;
    k.nvariants = 1;
    k.threads[0] = 128;
    k.minb[0] = 1;
    k.threads[kCvVariant] = 256;   // the control-variate kernel
    k.minb[kCvVariant] = 4;
    k.has_cv = true;
    k.threads[kF64Variant] = kF64Threads;   // the FP64-throughout kernel
    k.minb[kF64Variant] = 1;
    k.has_f64 = true;
    k.sweep = sweep<G>;
    k.occupancy = occ<G>;
    k.init = launch_init<G>;
    k.coef = launch_coef<G>;
    k.delta = launch_delta<G>;
    return k;
}
}  // namespace

bool kernels_quadratic(int n, bool zero_h, GameKernels* out) {
#define HJG_Q(N) case N: *out = zero_h ? make<N, true>() : make<N, false>(); return true;
    switch (n) { HJG_Q(1) HJG_Q(2) HJG_Q(3) HJG_Q(4) HJG_Q(6) HJG_Q(8) }
#undef HJG_Q
    return false;
}
}  // namespace hjg
