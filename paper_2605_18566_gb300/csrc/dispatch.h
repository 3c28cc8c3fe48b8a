// dispatch.h -- per-game kernel tables; each game's kernels live in their own
// translation unit so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "sweep_impl.cuh"

namespace hjg {

struct GameKernels {
    int n;  // state dimension
    // Launch the fused sweep with `threads` per CTA (0 if unsupported) on `grid` CTAs.
    cudaError_t (*sweep)(const SweepArgs& A, bool tilt, int threads, int grid, cudaStream_t st);
    // Resident CTAs per SM for the given variant (0 if unsupported).
    int (*occupancy)(bool tilt, int threads);
    cudaError_t (*init)(const float* x, int64_t ldx, int64_t M, const GameParams& g, double delta,
                        double eta, double c_min, double c_max, double* v, float* p, int64_t ldp,
                        float* c, float* ess, cudaStream_t st);
    int default_threads;
};

bool kernels_for(int game, int n, GameKernels* out);

GameKernels kernels_dubins3();
GameKernels kernels_rockets6();
GameKernels kernels_rockets45();
bool kernels_quadratic(int n, bool zero_h, GameKernels* out);

}  // namespace hjg
