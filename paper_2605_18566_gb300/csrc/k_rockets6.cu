// Sweep kernels for the two-rocket planar game, n = 6.
#include "dispatch.h"

namespace hjg {
namespace {
cudaError_t sweep(const SweepArgs& A, bool tilt, int threads, int grid, cudaStream_t st) {
    switch (threads) {
    case 128: return launch_sweep_generic<Rockets6, 128>(A, tilt, grid, st);
    case 256: return launch_sweep_generic<Rockets6, 256>(A, tilt, grid, st);
    case 512: return launch_sweep_generic<Rockets6, 512>(A, tilt, grid, st);
    }
    return cudaErrorInvalidValue;
}
int occ(bool tilt, int threads) {
    switch (threads) {
    case 128: return occupancy_generic<Rockets6, 128>(tilt);
    case 256: return occupancy_generic<Rockets6, 256>(tilt);
    case 512: return occupancy_generic<Rockets6, 512>(tilt);
    }
    return 0;
}
}  // namespace
GameKernels kernels_rockets6() { return {6, sweep, occ, launch_init<Rockets6>, 256}; }
}  // namespace hjg
