// Sweep kernels for the 15-agent multi-rocket game (Section 3.2), n = 45,
// four lanes per sample stream.
#include "dispatch.h"

namespace hjg {
namespace {
template <int T>
cudaError_t launch(const SweepArgs& A, bool tilt, int grid, cudaStream_t st) {
    if (tilt) sweep_kernel_r45<T, true><<<grid, T, 0, st>>>(A);
    else sweep_kernel_r45<T, false><<<grid, T, 0, st>>>(A);
    return cudaGetLastError();
}
template <int T>
int occupancy(bool tilt) {
    int nb = 0;
    if (tilt) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_r45<T, true>, T, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_kernel_r45<T, false>, T, 0);
    return nb;
}
cudaError_t sweep(const SweepArgs& A, bool tilt, int threads, int grid, cudaStream_t st) {
    switch (threads) {
    case 128: return launch<128>(A, tilt, grid, st);
    case 256: return launch<256>(A, tilt, grid, st);
    case 512: return launch<512>(A, tilt, grid, st);
    }
    return cudaErrorInvalidValue;
}
int occ(bool tilt, int threads) {
    switch (threads) {
    case 128: return occupancy<128>(tilt);
    case 256: return occupancy<256>(tilt);
    case 512: return occupancy<512>(tilt);
    }
    return 0;
}
}  // namespace
GameKernels kernels_rockets45() { return {45, sweep, occ, launch_init<Rockets45>, 256}; }
}  // namespace hjg
