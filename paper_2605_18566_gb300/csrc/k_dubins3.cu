// Sweep kernels for the relative Dubins game (Appendix D.2), n = 3.
#include "dispatch.h"

namespace hjg {
namespace {
cudaError_t sweep(const SweepArgs& A, bool tilt, int threads, int grid, cudaStream_t st) {
    switch (threads) {
    case 128: return launch_sweep_generic<Dubins3, 128>(A, tilt, grid, st);
    case 256: return launch_sweep_generic<Dubins3, 256>(A, tilt, grid, st);
    case 512: return launch_sweep_generic<Dubins3, 512>(A, tilt, grid, st);
    }
    return cudaErrorInvalidValue;
}
int occ(bool tilt, int threads) {
    switch (threads) {
    case 128: return occupancy_generic<Dubins3, 128>(tilt);
    case 256: return occupancy_generic<Dubins3, 256>(tilt);
    case 512: return occupancy_generic<Dubins3, 512>(tilt);
    }
    return 0;
}
}  // namespace
GameKernels kernels_dubins3() { return {3, sweep, occ, launch_init<Dubins3>, 256}; }
}  // namespace hjg
