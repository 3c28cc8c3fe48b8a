// dispatch.h -- per-game kernel tables; each game's kernels live in their own
// translation unit so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include "../../include/hjg.h"
#include "sweep_impl.cuh"
#include "sweep_f64.cuh"

namespace hjg {

struct GameKernels {
    int n;            // state dimension
    int nvariants;    // launch variants (CTA size x register budget) available
    int threads[16];   // CTA size of each variant
    int minb[16];      // minimum resident CTAs per SM each variant was compiled for
    int per_warp[16];  // 1: one warp per state (the grid is counted in CTAs of threads/32 warps)
    bool has_cv;       // the control-variate kernel exists (launch slot kCvVariant)
    bool cv_tilt_only; //   and runs only in the tilted frame
    bool has_f64;      // the FP64-throughout kernel exists (launch slot kF64Variant)
    // Launch the fused sweep, variant v, on `grid` CTAs.
    cudaError_t (*sweep)(const SweepArgs& A, bool tilt, int v, int grid, cudaStream_t st);
    // Resident CTAs per SM of variant v (0 if it cannot launch).
    int (*occupancy)(bool tilt, int v);
    cudaError_t (*init)(const float* x, int64_t ldx, int64_t M, const GameParams& g, double delta,
                        double eta, double c_min, double c_max, double* v, float* p, int64_t ldp,
                        float* c, float* ess, cudaStream_t st, const float* aux, int64_t ldaux);
    cudaError_t (*coef)(const float* x, int64_t ldx, int64_t M, const float* p, int64_t ldp,
                        const GameParams& g, double delta, double eta, double c_min, double c_max, float* c,
                        const float* aux, int64_t ldaux, cudaStream_t st);
    // The iterate relative to the initial one (delta_kernel): read it out, or warm start.
    cudaError_t (*delta)(const float* x, int64_t ldx, int64_t M, const GameParams& g, double delta, double eta,
                         double c_min, double c_max, double* v, float* p, int64_t ldp, float* c, float* d,
                         int64_t ldd, bool warm, const float* aux, int64_t ldaux, cudaStream_t st);
};

GameKernels kernels_dubins3();
GameKernels kernels_rockets6();
GameKernels kernels_rockets45();
GameKernels kernels_flock4();
GameKernels kernels_rockets_rel3();
GameKernels kernels_double_int2();
bool kernels_quadratic(int n, bool zero_h, GameKernels* out);

// Whether the target's reach-avoid obstacle (if any) is valid for the game (hjg_api.cu).
bool obstacle_ok(const hjg_dynamics* dyn, const hjg_target* t);

// Flock neighbour structure (flock.cu): 7 nearest agents, their mean heading, and the
// per-agent game data [M][kFlockAux] (neighbour positions, then the mean heading).
constexpr int kFlockAux = 22;
cudaError_t flock_neighbours(const float* x, int64_t ldx, int64_t M, int32_t* idx, float* psibar,
                             float* aux, int64_t ldaux, cudaStream_t st);

}  // namespace hjg

// Body of a game translation unit for the one-lane-per-sample kernel.
#define HJG_GENERIC_GAME_TU(GAME, FN)                                                      \
    namespace hjg {                                                                        \
    namespace {                                                                            \
    cudaError_t sweep(const SweepArgs& A, bool tilt, int v, int grid, cudaStream_t st) {   \
        switch (v) {                                                                       \
            HJG_SWEEP_VARIANTS(HJG_CASE_LAUNCH)                                            \
            case kCvVariant: return launch_sweep_cv<HJG_GAME>(A, tilt, grid, st);          \
            case kF64Variant: return launch_sweep_f64<HJG_GAME>(A, tilt, grid, st);        \
        }                                                                                  \
        return cudaErrorInvalidValue;                                                      \
    }                                                                                      \
    int occ(bool tilt, int v) {                                                            \
        switch (v) {                                                                       \
            HJG_SWEEP_VARIANTS(HJG_CASE_OCC)                                               \
            case kCvVariant: return occupancy_cv<HJG_GAME>(tilt);                          \
            case kF64Variant: return occupancy_f64<HJG_GAME>(tilt);                        \
        }                                                                                  \
        return 0;                                                                          \
    }                                                                                      \
    }                                                                                      \
    GameKernels FN() {                                                                     \
        GameKernels k{};                                                                   \
        k.n = GAME::kN;                                                                    \
        k.nvariants = kNumVariants;                                                        \
        HJG_SWEEP_VARIANTS(HJG_FILL)                                                       \
        k.threads[kCvVariant] = 256; k.minb[kCvVariant] = 4; k.per_warp[kCvVariant] = 0;   \
        k.has_cv = true;                                                                   \
        k.threads[kF64Variant] = kF64Threads; k.minb[kF64Variant] = 1;                     \
        k.per_warp[kF64Variant] = 0; k.has_f64 = true;                                     \
        k.sweep = sweep;                                                                   \
        k.occupancy = occ;                                                                 \
        k.init = launch_init<GAME>;                                                        \
        k.coef = launch_coef<GAME>;                                                        \
        k.delta = launch_delta<GAME>;                                                      \
        return k;                                                                          \
    }                                                                                      \
    }
#define HJG_CASE_LAUNCH(i, KIND, T, B) case i: return launch_sweep_generic<HJG_GAME, KIND, T, B>(A, tilt, grid, st);
#define HJG_CASE_OCC(i, KIND, T, B) case i: return occupancy_generic<HJG_GAME, KIND, T, B>(tilt);
#define HJG_FILL(i, KIND, T, B) k.threads[i] = T; k.minb[i] = B; k.per_warp[i] = (KIND) & 1;
