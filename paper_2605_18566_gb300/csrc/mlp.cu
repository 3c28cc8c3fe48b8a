// mlp.cu -- the surrogate network: an MLP n_in -> W -> W -> W -> n_out with SiLU
// activations, BF16 weights and activations, FP32 accumulation on the tensor cores, FP32
// master weights and Adam.  It is trained on the (x, v, Dv) tuples the Picard sweeps
// produce (loss: mean squared error of v plus the mean squared error of Dv averaged over
// its n components) and supplies a warm start (v, Dv, hence c = Gamma(Dv) and the tilt
// theta = -sigma^2 c Dv) for the sweep, whose own estimate stays the measure of its accuracy.
//
// Layout: parameters are one FP32 array [W1 | b1 | W2 | b2 | W3 | b3 | W4 | b4] with each
// W_l stored [out][in] row-major; a BF16 copy of the W_l feeds the tensor cores.  Inputs
// and outputs are padded to multiples of 16 (45 -> 48, 46 -> 48).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hjg.h"

namespace {

constexpr int kLayers = 4;

__host__ __device__ inline int pad16(int n) { return (n + 15) / 16 * 16; }

// ------------------------------------------------------------------------------------
// Strided BF16 GEMM: C(m, n) = sum_k A(m, k) B(k, n), with A(m, k) = A[m*sam + k*sak],
// B(k, n) = B[k*sbk + n*sbn] (BF16), FP32 accumulation, and an epilogue (bias, SiLU,
// BF16 activation copy).  gridDim.z splits K (each split writes its own partial for a
// later reduction).
enum Epi { kEpiStore = 0, kEpiBiasSilu = 1, kEpiBias = 2, kEpiSiluBwd = 3 };

struct GemmArgs {
    const __nv_bfloat16* A;
    const __nv_bfloat16* B;
    int64_t sam, sak, sbk, sbn;
    int M, N, K;
    float* C;          // FP32 output (z or partial), [M][ldc] (+ split * M * ldc)
    int64_t ldc;
    __nv_bfloat16* H;  // BF16 activation output (kEpiBiasSilu, kEpiSiluBwd), [M][ldh]
    int64_t ldh;
    __nv_bfloat16* Ht; // the same BF16 output transposed, [N][ldht] (or null)
    int64_t ldht;
    const float* Zin;  // kEpiSiluBwd: pre-activations [M][ldz]; H = C * silu'(Zin)
    int64_t ldz;
    const float* bias; // [N]
    int kper;          // K values per split (a multiple of 64 when split)
};

// Logistic sigmoid and SiLU through one hardware tanh (sigma(z) = (1 + tanh(z / 2)) / 2):
// one MUFU operation per element instead of an exponential and a reciprocal; its relative
// error (about 2^-11) is below the BF16 rounding of the activations it produces.
__device__ __forceinline__ float tanh_hw(float x) {
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sigmoid_t(float z) { return fmaf(0.5f, tanh_hw(0.5f * z), 0.5f); }
__device__ __forceinline__ float silu_t(float z) { return z * sigmoid_t(z); }
__device__ __forceinline__ float silu(float z) { return silu_t(z); }


// ------------------------------------------------------------------------------------
// The GEMM runs on the 5th-generation tensor cores (tcgen05, sm_100 family):
// a CTA of 4 warps owns a 128 x 64 tile of C, accumulated in tensor memory (TMEM, 128
// lanes x 64 FP32 columns; the narrow tile doubles the CTAs of the width-256 layers, which
// measured 11-13 % faster than 128 x 128 tiles).  Per K chunk of 64 the operands are copied
// by the tensor memory accelerator into shared memory in the canonical K-major no-swizzle
// layout (8-row x 16-byte core matrices), and thread 0 issues four tcgen05.mma (M = 128,
// N = 64, K = 16) and commits them to an
// mbarrier; every wait on a barrier is bounded and records a time-out in *err.  The
// epilogue reads TMEM with tcgen05.ld (warp w owns lanes 32w..32w+31 = rows).
constexpr int kTcM = 128, kTcN = 64, kTcK = 64;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start address, leading (K-direction) and stride
// (row-direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Descriptor of a K-major operand in the 128-byte swizzled layout that a SWIZZLE_128B
// tensor-map copy of a 64-wide BF16 K chunk produces: one 128-byte row per M/N index (its
// eight 16-byte pieces permuted by the row index mod 8), 8-row groups 1,024 bytes apart
// (SBO), the leading offset unused; swizzle mode 2 in bits 61-63.  The tile must start on a
// 1,024-byte boundary; the K steps of 16 within the chunk advance the start address by 32
// bytes (base offset 0: the start stays within the first 128 bytes of the pattern).
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, int* err, uint32_t limit = 1u << 24) {
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done) : "r"(bar), "r"(phase) : "memory");
        if (done) return true;
    }
    atomicExch(err, 1);
    return false;
}

// S-stage TMA pipeline: one thread issues, per K chunk of 64, the tensor-memory-accelerator
// copies of both operand tiles (cp.async.bulk.tensor, completion counted in bytes on the
// stage's "full" mbarrier) and, once a stage is full, the four tcgen05.mma of that chunk,
// whose commit arrives on the stage's "empty" mbarrier; a stage is refilled only after that
// arrival.  Up to S chunks are in flight.  The operands are K-major in global memory (A(m, k)
// = A[m lda + k], B(k, n) = Bt[n ldb + k], lda and ldb multiples of 8, 16-byte aligned
// bases; gemm() packs other layouts first) and are described by 2-D tensor maps (K
// innermost); each copy moves one 8-element K slice of 128 (A) or 64 (B) rows, so a chunk
// lands in shared memory as [8 K slices][rows][16 B]: the canonical K-major no-swizzle
// layout with core matrices 128 B apart along the rows and rows x 16 B apart along K.  Rows
// and K beyond the tensor read as zero.  S = 4 when a CTA's K range has at most four chunks
// and the grid fits in one wave at two CTAs per SM (every GEMM of the width-256 network at
// batch 8,192 then issues all its copies at once), else S = 2 (four CTAs per SM for long K
// ranges and multi-wave grids).
constexpr int kTcStage = (kTcM + kTcN) * kTcK * 2;   // bytes of one stage (A then B)
constexpr int tc_smem(int stages) { return stages * kTcStage; }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* tm, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        :: "r"(dst), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(bar) : "memory");
}

// The copies of one K chunk (k0 = its first K index, a multiple of 64) into stage `st`.
__device__ __forceinline__ void tma_chunk(uint32_t st, const CUtensorMap* tmA, const CUtensorMap* tmB, int m0,
                                          int n0, int k0, uint32_t bar) {
    mbar_expect_tx(bar, (uint32_t)kTcStage);
#pragma unroll
    for (int o = 0; o < kTcK / 8; ++o) {
        tma_load_2d(st + (uint32_t)(o * kTcM * 16), tmA, k0 + 8 * o, m0, bar);
        tma_load_2d(st + (uint32_t)(kTcM * kTcK * 2 + o * kTcN * 16), tmB, k0 + 8 * o, n0, bar);
    }
}

template <int EPI, int kTcStages>
__global__ void __launch_bounds__(128) gemm_tc_kernel(const GemmArgs g, const __grid_constant__ CUtensorMap tmA,
                                                      const __grid_constant__ CUtensorMap tmB, int* err) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kTcStages], empty[kTcStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTcM, n0 = blockIdx.x * kTcN;
    const int kbeg = blockIdx.z * g.kper, kend = min(g.K, kbeg + g.kper);
    const int nch = kend > kbeg ? (kend - kbeg + kTcK - 1) / kTcK : 0;
    const uint32_t s0 = smem_u32(smem);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kTcN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kTcStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t idesc = umma_idesc_bf16(kTcM, kTcN);
    bool ok = true;
    if (tid == 0 && nch > 0) {
        // parities of the next completion to wait for on each stage's barriers
        uint32_t ph_full[kTcStages] = {}, ph_empty[kTcStages] = {};
        int issued = 0, landed = 0;
        for (; issued < nch && issued < kTcStages; ++issued)
            tma_chunk(s0 + (uint32_t)(issued * kTcStage), &tmA, &tmB, m0, n0, kbeg + issued * kTcK,
                      smem_u32(&full[issued]));
        for (int c = 0; c < nch; ++c) {
            const int s = c % kTcStages;
            if (!mbar_wait(smem_u32(&full[s]), ph_full[s], err)) { ok = false; break; }
            ph_full[s] ^= 1u;
            landed = c + 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + (uint32_t)(s * kTcStage), sb = sa + kTcM * kTcK * 2;
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks) {
                const uint64_t da = umma_desc(sa + ks * (kTcM * 32), kTcM * 16, 128);
                const uint64_t db = umma_desc(sb + ks * (kTcN * 32), kTcN * 16, 128);
                const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(smem_u32(&empty[s])) : "memory");
            if (issued < nch) {   // refill this stage once its MMAs are done
                if (!mbar_wait(smem_u32(&empty[s]), ph_empty[s], err)) { ok = false; break; }
                ph_empty[s] ^= 1u;
                tma_chunk(sa, &tmA, &tmB, m0, n0, kbeg + issued * kTcK, smem_u32(&full[s]));
                ++issued;
            }
        }
        if (ok) {   // the last commit covers every earlier MMA of this thread
            const int s = (nch - 1) % kTcStages;
            ok = mbar_wait(smem_u32(&empty[s]), ph_empty[s], err);
        } else {    // a wait ran out: let the copies still in flight land (bounded) before leaving
            for (int c = landed; c < issued; ++c) {
                const int s = c % kTcStages;
                mbar_wait(smem_u32(&full[s]), ph_full[s], err);
                ph_full[s] ^= 1u;
            }
        }
    }
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // epilogue: row r = 32 warp + lane; per pass of 32 columns the bias and (kEpiSiluBwd)
    // pre-activation loads are issued first, then four tcgen05.ld of 8 columns and one
    // wait, so the global-memory and TMEM latencies overlap instead of adding up per
    // 8 columns.
    const int r = warp * 32 + lane;
    const int m = m0 + r;
    float* C = g.C ? g.C + (int64_t)blockIdx.z * g.M * g.ldc : nullptr;
    const bool vecC = C && (g.ldc % 4) == 0 && ((uintptr_t)C & 15) == 0;
    const bool vecH = (g.ldh % 8) == 0 && ((uintptr_t)g.H & 15) == 0;
    const bool vecZ = EPI == kEpiSiluBwd && (g.ldz % 4) == 0 && ((uintptr_t)g.Zin & 15) == 0;
    constexpr bool kH = EPI == kEpiBiasSilu || EPI == kEpiSiluBwd;
    constexpr bool kBias = EPI == kEpiBiasSilu || EPI == kEpiBias;
    constexpr int kPass = 32;
    // One pass's outputs are staged in the operand stages' shared memory (the finished MMAs
    // no longer read it) and written out cooperatively, so that every global store is a
    // 16-byte piece of a contiguous row run: the FP32 output [128][kCsLd], the BF16
    // activation [128][kHsLd] and its transpose [kPass][kHtLd] (the rows of a column
    // contiguous).  The paddings keep the shared-memory accesses free of bank conflicts.
    constexpr int kCsLd = kPass + 4, kHsLd = kPass + 8, kHtLd = kTcM + 8;
    constexpr int kCsBytes = kTcM * kCsLd * 4, kHsBytes = kTcM * kHsLd * 2;
    static_assert(kCsBytes + kHsBytes + kPass * kHtLd * 2 <= 2 * kTcStage, "staging must fit the operand stages");
    float* cs = reinterpret_cast<float*>(smem);
    __nv_bfloat16* hs = reinterpret_cast<__nv_bfloat16*>(smem + kCsBytes);
    __nv_bfloat16* hs_t = reinterpret_cast<__nv_bfloat16*>(smem + kCsBytes + kHsBytes);
    if (ok && nch > 0) {
#pragma unroll 1
        for (int p0 = 0; p0 < kTcN; p0 += kPass) {
            const int np = n0 + p0;
            float pre[kPass];   // bias (kBias) or pre-activation Z (kEpiSiluBwd) of the pass
            if (kBias) {
#pragma unroll
                for (int j = 0; j < kPass; ++j) pre[j] = np + j < g.N ? g.bias[np + j] : 0.0f;
            } else if (EPI == kEpiSiluBwd) {
                if (m < g.M && np + kPass <= g.N && vecZ) {
                    const float4* zp = reinterpret_cast<const float4*>(g.Zin + (int64_t)m * g.ldz + np);
#pragma unroll
                    for (int q = 0; q < kPass / 4; ++q) {
                        const float4 t = zp[q];
                        pre[4 * q] = t.x; pre[4 * q + 1] = t.y; pre[4 * q + 2] = t.z; pre[4 * q + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < kPass; ++j)
                        pre[j] = (m < g.M && np + j < g.N) ? g.Zin[(int64_t)m * g.ldz + np + j] : 0.0f;
                }
            }
            uint32_t v[kPass];
#pragma unroll
            for (int q = 0; q < kPass / 8; ++q)
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                    : "=r"(v[8 * q]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]),
                      "=r"(v[8 * q + 4]), "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(p0 + 8 * q)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < kPass / 8; ++q) {   // stage row r of the pass
                float x[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    x[j] = __uint_as_float(v[8 * q + j]);
                    if (kBias) x[j] += pre[8 * q + j];
                }
                if (EPI == kEpiSiluBwd) {   // dZ = dH silu'(Z), silu'(z) = s (1 + z (1 - s)), s = sigmoid(z)
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float z = pre[8 * q + j];
                        const float sg = sigmoid_t(z);
                        x[j] = x[j] * sg * (1.0f + z * (1.0f - sg));
                    }
                }
                if (C) {
                    float4* d = reinterpret_cast<float4*>(cs + r * kCsLd + 8 * q);
                    d[0] = make_float4(x[0], x[1], x[2], x[3]);
                    d[1] = make_float4(x[4], x[5], x[6], x[7]);
                }
                if (kH) {
                    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16(EPI == kEpiBiasSilu ? silu(x[j]) : x[j]);
                    *reinterpret_cast<uint4*>(hs + r * kHsLd + 8 * q) = *reinterpret_cast<const uint4*>(h);
                    if (g.Ht) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) hs_t[(8 * q + j) * kHtLd + r] = h[j];
                    }
                }
            }
            __syncthreads();
            if (C) {   // 128 rows x kPass FP32: 16-byte pieces, a warp covering four rows
#pragma unroll
                for (int i = 0; i < kTcM * kPass / 4 / 128; ++i) {
                    const int idx = tid + 128 * i;
                    const int rr = idx / (kPass / 4), c4 = 4 * (idx % (kPass / 4));
                    const int mm = m0 + rr, n = np + c4;
                    if (mm >= g.M || n >= g.N) continue;
                    const float* src = cs + rr * kCsLd + c4;
                    float* dst = C + (int64_t)mm * g.ldc + n;
                    if (vecC && n + 4 <= g.N) *reinterpret_cast<float4*>(dst) = *reinterpret_cast<const float4*>(src);
                    else for (int t = 0; t < 4 && n + t < g.N; ++t) dst[t] = src[t];
                }
            }
            if (kH) {   // 128 rows x kPass BF16, and the transpose: kPass columns x 128 rows
#pragma unroll
                for (int i = 0; i < kTcM * kPass / 8 / 128; ++i) {
                    const int idx = tid + 128 * i;
                    const int rr = idx / (kPass / 8), c8 = 8 * (idx % (kPass / 8));
                    const int mm = m0 + rr, n = np + c8;
                    if (mm >= g.M || n >= g.N) continue;
                    const __nv_bfloat16* src = hs + rr * kHsLd + c8;
                    __nv_bfloat16* dst = g.H + (int64_t)mm * g.ldh + n;
                    if (vecH && n + 8 <= g.N) *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
                    else for (int t = 0; t < 8 && n + t < g.N; ++t) dst[t] = src[t];
                }
                if (g.Ht) {
                    const bool vecT = (g.ldht % 8) == 0 && ((uintptr_t)g.Ht & 15) == 0;
#pragma unroll
                    for (int i = 0; i < kPass * kTcM / 8 / 128; ++i) {
                        const int idx = tid + 128 * i;
                        const int c = idx / (kTcM / 8), r8 = 8 * (idx % (kTcM / 8));
                        const int n = np + c, mm = m0 + r8;
                        if (n >= g.N || mm >= g.M) continue;
                        const __nv_bfloat16* src = hs_t + c * kHtLd + r8;
                        __nv_bfloat16* dst = g.Ht + (int64_t)n * g.ldht + mm;
                        if (vecT && mm + 8 <= g.M) *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(src);
                        else for (int t = 0; t < 8 && mm + t < g.M; ++t) dst[t] = src[t];
                    }
                }
            }
            __syncthreads();   // the next pass overwrites the staging
        }
    } else if (m < g.M) {   // empty K range (or a timed-out wait): C = 0 (+ bias)
        for (int n = n0; n < min(g.N, n0 + kTcN); ++n) {
            const float x = (EPI == kEpiBiasSilu || EPI == kEpiBias) ? g.bias[n] : 0.0f;
            if (C) C[(int64_t)m * g.ldc + n] = x;
            if (kH) {
                const __nv_bfloat16 hv = __float2bfloat16(EPI == kEpiBiasSilu ? silu(x) : 0.0f);
                g.H[(int64_t)m * g.ldh + n] = hv;
                if (g.Ht) g.Ht[(int64_t)n * g.ldht + m] = hv;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kTcN));
}

// Pack an operand into K-major form: dst[r][k] = src[r * s_r + k * s_k] for k < K, zero
// for K <= k < ldd (ldd a multiple of 8).  32 x 32 tiles through shared memory, so that
// both the reads (along whichever index of src is contiguous) and the writes (along k)
// are coalesced.
__global__ void pack_kmajor_kernel(const __nv_bfloat16* __restrict__ src, int64_t s_r, int64_t s_k, int R, int K,
                                   __nv_bfloat16* __restrict__ dst, int64_t ldd) {
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const bool r_fast = s_r == 1;   // src contiguous along r: let threadIdx.x run along r
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int a = r_fast ? k0 + i : r0 + i;                  // slow index
        const int b = r_fast ? r0 + threadIdx.x : k0 + threadIdx.x;   // fast index
        const int r = r_fast ? b : a, k = r_fast ? a : b;
        __nv_bfloat16 v = __float2bfloat16(0.0f);
        if (r < R && k < K) v = src[(int64_t)r * s_r + (int64_t)k * s_k];
        if (r_fast) tile[threadIdx.x][i] = v; else tile[i][threadIdx.x] = v;   // tile[r - r0][k - k0]
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, k = k0 + threadIdx.x;
        if (r < R && k < ldd) dst[(int64_t)r * ldd + k] = tile[i][threadIdx.x];
    }
}

int* g_tc_err = nullptr;   // device word set by a timed-out barrier wait

inline int64_t pad8(int64_t k) { return (k + 7) / 8 * 8; }

// Scratch (elements) gemm() needs to pack the operands of g into K-major form.
inline int64_t gemm_scratch_a(const GemmArgs& g) {
    const bool ok = g.sak == 1 && g.sam % 8 == 0 && g.K % 8 == 0 && ((uintptr_t)g.A & 15) == 0;
    return ok ? 0 : (int64_t)g.M * pad8(g.K);
}
inline int64_t gemm_scratch_b(const GemmArgs& g) {
    const bool ok = g.sbk == 1 && g.sbn % 8 == 0 && g.K % 8 == 0 && ((uintptr_t)g.B & 15) == 0;
    return ok ? 0 : (int64_t)g.N * pad8(g.K);
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime (no link
// against libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 2-D tensor map of a K-major BF16 operand [rows][ld] (K = the first k_extent columns of a
// row), box = one 8-element K slice of box_rows rows; out-of-range elements read as zero.
bool operand_map(CUtensorMap* tm, const __nv_bfloat16* base, int64_t rows, int64_t k_extent, int64_t ld,
                 int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || ((uintptr_t)base & 15) != 0 || (ld % 8) != 0 || rows < 1 || k_extent < 1) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k_extent, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {8u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The same operand as 64-wide K boxes of box_rows rows in the 128-byte swizzled layout (one
// copy per operand and K chunk; umma_desc_sw128 reads it).
bool operand_map_sw128(CUtensorMap* tm, const __nv_bfloat16* base, int64_t rows, int64_t k_extent, int64_t ld,
                       int box_rows) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn || ((uintptr_t)base & 15) != 0 || (ld % 8) != 0 || rows < 1 || k_extent < 1 || box_rows > 256)
        return false;
    const cuuint64_t dims[2] = {(cuuint64_t)k_extent, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1u, 1u};
    return fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int EPI, int S>
cudaError_t launch_tc_s(const GemmArgs& k, int splits, cudaStream_t st) {
    static bool attr = false;   // opt in to the dynamic shared memory once per process
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(gemm_tc_kernel<EPI, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             tc_smem(S));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap tmA, tmB;   // unused (zero) when K is empty: the kernel then writes C = 0 (+ bias)
    memset(&tmA, 0, sizeof tmA);
    memset(&tmB, 0, sizeof tmB);
    if (k.K > 0 &&
        (!operand_map(&tmA, k.A, k.M, k.K, k.sam, kTcM) || !operand_map(&tmB, k.B, k.N, k.K, k.sbn, kTcN)))
        return cudaErrorInvalidValue;
    dim3 grid((k.N + kTcN - 1) / kTcN, (k.M + kTcM - 1) / kTcM, splits);
    gemm_tc_kernel<EPI, S><<<grid, 128, tc_smem(S), st>>>(k, tmA, tmB, g_tc_err);
    return cudaGetLastError();
}

template <int EPI>
cudaError_t launch_tc(const GemmArgs& k, int splits, cudaStream_t st) {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
            sms = 1;
    }
    const int64_t ctas = (int64_t)((k.N + kTcN - 1) / kTcN) * ((k.M + kTcM - 1) / kTcM) * splits;
    const bool deep = k.kper <= 4 * kTcK && ctas <= 2 * (int64_t)sms;   // one wave at 2 CTAs per SM
    return deep ? launch_tc_s<EPI, 4>(k, splits, st) : launch_tc_s<EPI, 2>(k, splits, st);
}

// C = A B (+ epilogue) on the tensor cores.  Operands that are not K-major with aligned
// rows are packed into the caller's scratch (sizes gemm_scratch_a / _b) first.  With
// splits > 1 each split covers a multiple of 64 values of K and writes its own partial.
cudaError_t gemm(const GemmArgs& g, int epi, int splits, cudaStream_t st, __nv_bfloat16* scratch_a = nullptr,
                 __nv_bfloat16* scratch_b = nullptr) {
    if (!g_tc_err) {
        if (cudaMalloc(&g_tc_err, sizeof(int)) != cudaSuccess) return cudaErrorMemoryAllocation;
        if (cudaMemset(g_tc_err, 0, sizeof(int)) != cudaSuccess) return cudaErrorMemoryAllocation;
    }
    GemmArgs k = g;
    const int64_t Kp = pad8(g.K);
    if (gemm_scratch_a(g)) {
        if (!scratch_a) return cudaErrorInvalidValue;
        dim3 grid((unsigned)((Kp + 31) / 32), (unsigned)((g.M + 31) / 32));
        pack_kmajor_kernel<<<grid, dim3(32, 8), 0, st>>>(g.A, g.sam, g.sak, g.M, g.K, scratch_a, Kp);
        k.A = scratch_a; k.sam = Kp; k.sak = 1;
    }
    if (gemm_scratch_b(g)) {
        if (!scratch_b) return cudaErrorInvalidValue;
        dim3 grid((unsigned)((Kp + 31) / 32), (unsigned)((g.N + 31) / 32));
        pack_kmajor_kernel<<<grid, dim3(32, 8), 0, st>>>(g.B, g.sbn, g.sbk, g.N, g.K, scratch_b, Kp);
        k.B = scratch_b; k.sbn = Kp; k.sbk = 1;
    }
    k.K = (int)Kp;   // the padded columns hold zeros
    // split boundaries on chunk boundaries; a split left without K values writes zeros
    k.kper = splits > 1 ? ((int)((Kp + splits - 1) / splits) + kTcK - 1) / kTcK * kTcK : (int)Kp;
    switch (epi) {
    case kEpiStore: return launch_tc<kEpiStore>(k, splits, st);
    case kEpiBiasSilu: return launch_tc<kEpiBiasSilu>(k, splits, st);
    case kEpiBias: return launch_tc<kEpiBias>(k, splits, st);
    case kEpiSiluBwd: return launch_tc<kEpiSiluBwd>(k, splits, st);
    }
    return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------------------------
// Element-wise kernels.

// x [B][ldx] FP32 (n_in used) -> X [B][in_pad] BF16 (zero padding).
// Network input: the standardised features (x_j - shift_j) mul_j in BF16, zero padded.
__global__ void pack_input_kernel(const float* __restrict__ x, int64_t ldx, int64_t B, int n_in,
                                  int in_pad, const float* __restrict__ scal, __nv_bfloat16* __restrict__ X) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * in_pad) return;
    const int64_t b = e / in_pad;
    const int j = (int)(e % in_pad);
    X[e] = __float2bfloat16(j < n_in ? (x[b * ldx + j] - scal[j]) * scal[in_pad + j] : 0.0f);
}

// Network output in the targets' units: out_j = o_j mul_j + shift_j.
__global__ void unscale_output_kernel(const float* __restrict__ o, int out_pad, int64_t B, int n_out,
                                      const float* __restrict__ oscal, float* __restrict__ out, int64_t ldout) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * n_out) return;
    const int64_t b = e / n_out;
    const int j = (int)(e % n_out);
    out[b * ldout + j] = fmaf(o[b * out_pad + j], oscal[out_pad + j], oscal[j]);
}

// Input gradient in the inputs' units: d out_j / d x_i = (d o_j / d xs_i) mul_i^in mul_j^out.
__global__ void scale_input_grad_kernel(const float* __restrict__ g, int in_pad, int64_t B, int n_in,
                                        const float* __restrict__ iscal, const float* __restrict__ oscal,
                                        int out_pad, int j, float* __restrict__ gx, int64_t ldg) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= B * n_in) return;
    const int64_t b = e / n_in;
    const int i = (int)(e % n_in);
    gx[b * ldg + i] = g[b * in_pad + i] * iscal[in_pad + i] * oscal[out_pad + j];
}

// Per-feature mean and standard deviation of v [B][ld] (columns 0..n-1, FP64 sums, one
// CTA per column, fixed reduction order): shift_j = mean, mul_j = 1/std (inputs) or std
// (outputs); a column with std below 1e-12 (relative) gets std 1.
__global__ void feature_stats_kernel(const float* __restrict__ v, int64_t ld, int64_t B, int pad, int inverse,
                                     float* __restrict__ scal) {
    __shared__ double s1[256], s2[256];
    const int j = blockIdx.x;
    double a = 0.0, q = 0.0;
    for (int64_t b = threadIdx.x; b < B; b += 256) {
        const double x = (double)v[b * ld + j];
        a += x;
        q = fma(x, x, q);
    }
    s1[threadIdx.x] = a; s2[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) { s1[threadIdx.x] += s1[threadIdx.x + w]; s2[threadIdx.x] += s2[threadIdx.x + w]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mean = s1[0] / (double)B;
        const double var = fmax(s2[0] / (double)B - mean * mean, 0.0);
        double sd = sqrt(var);
        if (!(sd > 1e-12 * (1.0 + fabs(mean)))) sd = 1.0;
        scal[j] = (float)mean;
        scal[pad + j] = (float)(inverse ? 1.0 / sd : sd);
    }
}

// Loss and its gradient w.r.t. the outputs: L = mean_b[(o_0 - y_0)^2 + mean_j (o_j - y_j)^2]
// over j = 1..n_out-1, with the targets standardised like the outputs (y - shift) / mul.
// dO (BF16) is written for the backward GEMMs; each block sums its elements' loss terms in
// FP32 (warp shuffles, then the 8 warps) and writes the sum / B to partial[blockIdx.x]
// (added in a fixed order on the host).  Launched with 256 threads.
__global__ void __launch_bounds__(256) loss_grad_kernel(const float* __restrict__ out, int64_t ldo,
                                                         const float* __restrict__ y, int64_t ldy, int64_t B,
                                                         int n_out, int out_pad, const float* __restrict__ oscal,
                                                         __nv_bfloat16* __restrict__ dO, float* __restrict__ dOf,
                                                         double* __restrict__ partial) {
    __shared__ float red[8];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float l = 0.0f;   // w d^2 of this element; the block's sum is divided by B in FP64
    if (e < B * out_pad) {
        const int64_t b = e / out_pad;
        const int j = (int)(e % out_pad);
        float g = 0.0f;
        if (j < n_out) {
            const float d = out[b * ldo + j] - (y[b * ldy + j] - oscal[j]) / oscal[out_pad + j];
            const float w = j == 0 ? 1.0f : 1.0f / (float)(n_out - 1);
            l = w * d * d;
            g = 2.0f * w * d / (float)B;
        }
        dO[e] = __float2bfloat16(g);
        if (dOf) dOf[e] = g;
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) t += red[w];
        partial[blockIdx.x] = (double)t / (double)B;
    }
}

// dZ = dH * SiLU'(Z), SiLU'(z) = s (1 + z (1 - s)), s = sigmoid(z); BF16 out.
__global__ void silu_backward_kernel(const float* __restrict__ dH, const float* __restrict__ Z, int64_t n,
                                     __nv_bfloat16* __restrict__ dZ) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float z = Z[e];
    const float s = sigmoid_t(z);
    dZ[e] = __float2bfloat16(dH[e] * s * (1.0f + z * (1.0f - s)));
}

// Sum of `splits` partial weight gradients [splits][rows][cols] into grad (FP32), and the
// bias gradient (column sums of dZ over the batch) for this layer; the splits are added in
// order, one element per thread (a float4 form with a quarter of the threads measured 10 %
// slower over a training step).
__global__ void reduce_wgrad_kernel(const float* __restrict__ part, int splits, int64_t n,
                                    float* __restrict__ grad) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    float s = 0.0f;
    for (int k = 0; k < splits; ++k) s += part[(int64_t)k * n + e];
    grad[e] = s;
}

inline cudaError_t reduce_wgrad(const float* part, int splits, int64_t n, float* grad, cudaStream_t st) {
    reduce_wgrad_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, splits, n, grad);
    return cudaGetLastError();
}

// Bias gradient = column sums of dZ [B][cols], first stage: CTA (x, y) sums 32 columns
// over the y-th of gridDim.y row chunks (8 row lanes, then a shared-memory sum); the
// chunk partials [gridDim.y][cols] are added by reduce_wgrad_kernel (fixed order).
constexpr int kBiasChunks = 64;
__global__ void __launch_bounds__(256) bias_partial_kernel(const __nv_bfloat16* __restrict__ dZ, int64_t B,
                                                           int cols, float* __restrict__ part) {
    __shared__ float red[8][33];
    const int c = blockIdx.x * 32 + threadIdx.x;
    const int64_t per = (B + gridDim.y - 1) / gridDim.y;
    const int64_t b0 = (int64_t)blockIdx.y * per;
    const int64_t b1 = b0 + per < B ? b0 + per : B;
    float s = 0.0f;
    if (c < cols)
        for (int64_t b = b0 + threadIdx.y; b < b1; b += 8) s += __bfloat162float(dZ[b * cols + c]);
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && c < cols) {
        float t = 0.0f;
#pragma unroll
        for (int i = 0; i < 8; ++i) t += red[i][threadIdx.x];
        part[(int64_t)blockIdx.y * cols + c] = t;
    }
}

// Adam (Kingma & Ba) on the FP32 master parameters; refresh the BF16 weight copy.
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1,
                            float* __restrict__ m2, __nv_bfloat16* __restrict__ wb, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float a = b1 * m1[e] + (1.0f - b1) * gg;
    const float b = b2 * m2[e] + (1.0f - b2) * gg * gg;
    m1[e] = a;
    m2[e] = b;
    const float upd = lr * (a / c1) / (sqrtf(b / c2) + eps);
    const float nw = w[e] - upd;
    w[e] = nw;
    wb[e] = __float2bfloat16(nw);
}

// dO = e_j for every row (the derivative of output j), BF16.
__global__ void unit_output_kernel(int64_t B, int out_pad, int j, __nv_bfloat16* __restrict__ dO) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < B * out_pad) dO[e] = __float2bfloat16((int)(e % out_pad) == j ? 1.0f : 0.0f);
}

__global__ void to_bf16_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wb, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) wb[e] = __float2bfloat16(w[e]);
}

// Per-layer transposed BF16 copies of the weights, W_l^T [cols][rows] at the same offset
// as W_l: the K-major operand of the backward data-gradient GEMM dH = dZ W.
struct WeightMap {
    int64_t w_off[kLayers];
    int rows[kLayers], cols[kLayers];
};
__global__ void weights_t_kernel(const float* __restrict__ w, __nv_bfloat16* __restrict__ wt, WeightMap map) {
    const int l = blockIdx.y;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int rows = map.rows[l], cols = map.cols[l];
    if (e >= (int64_t)rows * cols) return;
    const int r = (int)(e / cols), c = (int)(e % cols);
    wt[map.w_off[l] + (int64_t)c * rows + r] = __float2bfloat16(w[map.w_off[l] + e]);
}

// Deterministic initialisation: W_l uniform in +-sqrt(6 / (fan_in + fan_out)) (rows beyond
// n_out and columns beyond n_in zero), biases zero; uniforms from a 64-bit mix of
// (seed, index).
__device__ __forceinline__ float hash_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)((z >> 40) * (1.0 / 16777216.0)) * 2.0f - 1.0f;
}

__global__ void init_weight_kernel(float* __restrict__ W, int rows, int cols, int rows_used,
                                   int cols_used, float scale, uint64_t seed) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * cols) return;
    const int r = (int)(e / cols), c = (int)(e % cols);
    W[e] = (r < rows_used && c < cols_used) ? scale * hash_uniform(seed, (uint64_t)e) : 0.0f;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Self-test of the bounded wait: one thread initialises an mbarrier expecting one arrival,
// arrives on it only if `arrive` is set, and waits with the given iteration limit.  With no
// arrival the wait gives up, sets *err and the kernel returns normally.
__global__ void bounded_wait_kernel(int arrive, uint32_t limit, int* err) {
    __shared__ __align__(8) uint64_t bar;
    const uint32_t b = smem_u32(&bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(b));
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (arrive) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(b) : "memory");
    mbar_wait(b, 0, err, limit);
}

// ------------------------------------------------------------------------------------
struct hjg_mlp {
    int n_in, n_out, width, in_pad, out_pad;
    int rows[kLayers], cols[kLayers];     // W_l is [rows][cols] = [out_pad_l][in_pad_l]
    int64_t w_off[kLayers], b_off[kLayers], n_params;
    float* p = nullptr;                   // FP32 master parameters
    float* g = nullptr;                   // gradients
    float* m1 = nullptr;                  // Adam moments
    float* m2 = nullptr;
    __nv_bfloat16* pb = nullptr;          // BF16 copy (weights used by the GEMMs)
    __nv_bfloat16* pbT = nullptr;         // BF16 transposed weights W_l^T (same offsets)
    float* iscal = nullptr;               // input standardisation [shift in_pad | mul in_pad]
    float* oscal = nullptr;               // output scaling [shift out_pad | mul out_pad]
    int64_t cap = 0;                      // batch capacity of the work buffers
    __nv_bfloat16* X = nullptr;           // [cap][in_pad]
    float* Z[kLayers] = {};               // pre-activations [cap][width] (layer 4: outputs)
    __nv_bfloat16* H[kLayers] = {};       // activations [cap][width] BF16
    __nv_bfloat16* dZ = nullptr;          // [cap][width] BF16
    __nv_bfloat16* dZ2 = nullptr;         // [cap][width] BF16 (the fused backward alternates)
    __nv_bfloat16* Ht[kLayers] = {};      // transposed activations H_l^T [width][pad8(B)] (training)
    __nv_bfloat16* dZt = nullptr;         // transposed dZ [D][pad8(B)]
    float* dH = nullptr;                  // [cap][width] FP32
    float* wpart = nullptr;               // split-K partial weight gradients
    __nv_bfloat16* packA = nullptr;       // K-major copies of transposed GEMM operands
    __nv_bfloat16* packB = nullptr;       //   (dZ^T, H^T, W^T) for the backward GEMMs
    double* lpart = nullptr;              // loss partial sums
    int64_t lpart_cap = 0;
    // fused training step (width 256, in_pad and out_pad <= 64): canonical copies of the BF16
    // weights, W_l and W_l^T in the tensor cores' K-major core-matrix layout, one contiguous
    // block per layer (offsets wp_off, n_w weights in all), and its work buffers
    int64_t wp_off[kLayers] = {}, n_w = 0;
    __nv_bfloat16* wc = nullptr;          // W_l [rows][cols] as B operands (N = rows, K = cols)
    __nv_bfloat16* wct = nullptr;         // W_l^T [cols][rows] as B operands (N = cols, K = rows)
    int64_t fcap = 0;                     // batch capacity of the fused buffers
    __nv_bfloat16* Xt = nullptr;          // X^T [in_pad][pad8(B)]
    __nv_bfloat16* dZt4[kLayers] = {};    // dZ_l^T [rows_l][pad8(B)] (layer 4: dO^T)
    float* fpart = nullptr;               // split-K weight-gradient partials [splits][n_w]
    double* flpart = nullptr;             // loss partial sums, one per batch tile
    int64_t step = 0;
    cudaStream_t stream = nullptr;
    std::string err;
};

namespace {

constexpr int kSplits = 32;

hjg_status mlp_ensure(hjg_mlp* m, int64_t B) {
    if (B <= m->cap) return HJG_OK;
    auto fre = [](void* p) { if (p) cudaFree(p); };
    fre(m->X); fre(m->dZ); fre(m->dZ2); fre(m->dZt); fre(m->dH); fre(m->lpart); fre(m->packA); fre(m->packB);
    m->X = m->dZ = m->dZ2 = m->dZt = m->packA = m->packB = nullptr;   // none survives a failed growth
    m->dH = nullptr;
    m->lpart = nullptr;
    for (int l = 0; l < kLayers; ++l) {
        fre(m->Z[l]); fre(m->H[l]); fre(m->Ht[l]);
        m->Z[l] = nullptr; m->H[l] = nullptr; m->Ht[l] = nullptr;
    }
    const int W = m->width;
    const int64_t D = std::max<int64_t>(W, std::max(m->in_pad, m->out_pad));
    const int64_t pa = D * pad8(B), pbk = D * std::max(pad8(B), pad8(D));
    bool ok = cudaMalloc(&m->X, (size_t)B * m->in_pad * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->dZ, (size_t)B * W * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->dH, (size_t)B * W * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->packA, (size_t)pa * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->packB, (size_t)pbk * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->dZ2, (size_t)B * W * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->dZt, (size_t)D * pad8(B) * sizeof(__nv_bfloat16)) == cudaSuccess;
    for (int l = 0; l + 1 < kLayers && ok; ++l)
        ok = cudaMalloc(&m->Ht[l], (size_t)W * pad8(B) * sizeof(__nv_bfloat16)) == cudaSuccess;
    for (int l = 0; l < kLayers && ok; ++l) {
        ok = cudaMalloc(&m->Z[l], (size_t)B * W * sizeof(float)) == cudaSuccess &&
             cudaMalloc(&m->H[l], (size_t)B * W * sizeof(__nv_bfloat16)) == cudaSuccess;
    }
    m->lpart_cap = (B * m->out_pad + 255) / 256;
    ok = ok && cudaMalloc(&m->lpart, (size_t)m->lpart_cap * sizeof(double)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();   // reported here as ENOMEM: not left for a later launch check to find
        m->cap = 0;
        m->err = "MLP work buffers: out of memory";
        return HJG_ENOMEM;
    }
    m->cap = B;
    return HJG_OK;
}

// Refresh the transposed BF16 weights from the FP32 master copy.
cudaError_t refresh_wt(hjg_mlp* m, cudaStream_t st) {
    WeightMap map{};
    int64_t mx = 0;
    for (int l = 0; l < kLayers; ++l) {
        map.w_off[l] = m->w_off[l]; map.rows[l] = m->rows[l]; map.cols[l] = m->cols[l];
        mx = std::max<int64_t>(mx, (int64_t)m->rows[l] * m->cols[l]);
    }
    weights_t_kernel<<<dim3(nblk(mx), kLayers), 256, 0, st>>>(m->p, m->pbT, map);
    return cudaGetLastError();
}

// Forward pass on X (already packed); outputs FP32 in Z[3] [B][out_pad].  With `train` the
// hidden layers also write their activations transposed (H_l^T, leading dimension
// pad8(B)), the K-major operand of the weight-gradient GEMMs.
cudaError_t mlp_forward(hjg_mlp* m, int64_t B, bool train = false) {
    cudaError_t e = cudaSuccess;
    const int64_t ldT = pad8(B);
    for (int l = 0; l < kLayers && e == cudaSuccess; ++l) {
        GemmArgs g{};
        const __nv_bfloat16* in = l == 0 ? m->X : m->H[l - 1];
        const int in_ld = l == 0 ? m->in_pad : m->width;
        g.A = in; g.sam = in_ld; g.sak = 1;
        g.B = m->pb + m->w_off[l]; g.sbk = 1; g.sbn = m->cols[l];
        g.M = (int)B; g.N = m->rows[l]; g.K = m->cols[l];
        g.C = m->Z[l]; g.ldc = m->rows[l];
        g.bias = m->p + m->b_off[l];
        if (l + 1 < kLayers) {
            g.H = m->H[l]; g.ldh = m->rows[l];
            if (train) {
                // the padding columns B..ldT-1 of H_l^T are read as K values: keep them zero
                if (ldT > B &&
                    (e = cudaMemset2DAsync(m->Ht[l] + B, ldT * sizeof(__nv_bfloat16), 0,
                                           (ldT - B) * sizeof(__nv_bfloat16), m->rows[l], m->stream)) != cudaSuccess)
                    break;
                g.Ht = m->Ht[l]; g.ldht = ldT;
            }
            e = gemm(g, kEpiBiasSilu, 1, m->stream);
        } else {
            e = gemm(g, kEpiBias, 1, m->stream);
        }
    }
    return e;
}

// Backward pass from dO (BF16 in m->dZ, [B][out_pad]) after a training forward; gradients
// into m->g.  Per layer l: dW_l = dZ_l^T H_{l-1} (split-K over the batch, both operands
// K-major with K = pad8(B): dZ_l^T from the previous layer's fused epilogue, H_{l-1}^T from
// the forward), the bias gradient, and dZ_{l-1} = (dZ_l W_l) silu'(Z_{l-1}) in one GEMM whose
// epilogue writes dZ_{l-1} and its transpose.
cudaError_t mlp_backward(hjg_mlp* m, int64_t B) {
    cudaError_t e = cudaSuccess;
    const int64_t ldT = pad8(B);
    __nv_bfloat16* dz = m->dZ;
    __nv_bfloat16* dz_next = m->dZ2;
    // the transposed operands of the output layer (dO^T) and the input layer (X^T)
    {
        const int r3 = m->rows[kLayers - 1];
        dim3 ga((unsigned)((ldT + 31) / 32), (unsigned)((r3 + 31) / 32));
        pack_kmajor_kernel<<<ga, dim3(32, 8), 0, m->stream>>>(m->dZ, 1, r3, r3, (int)B, m->dZt, ldT);
        const int c0 = m->cols[0];
        dim3 gb((unsigned)((ldT + 31) / 32), (unsigned)((c0 + 31) / 32));
        pack_kmajor_kernel<<<gb, dim3(32, 8), 0, m->stream>>>(m->X, 1, c0, c0, (int)B, m->packB, ldT);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (int l = kLayers - 1; l >= 0 && e == cudaSuccess; --l) {
        const int rows = m->rows[l], cols = m->cols[l];
        GemmArgs gw{};
        gw.A = m->dZt; gw.sam = ldT; gw.sak = 1;
        gw.B = l == 0 ? m->packB : m->Ht[l - 1]; gw.sbk = 1; gw.sbn = ldT;
        gw.M = rows; gw.N = cols; gw.K = (int)ldT;
        gw.C = m->wpart; gw.ldc = cols;
        e = gemm(gw, kEpiStore, kSplits, m->stream);
        if (e != cudaSuccess) break;
        const int64_t nw = (int64_t)rows * cols;
        if ((e = reduce_wgrad(m->wpart, kSplits, nw, m->g + m->w_off[l], m->stream)) != cudaSuccess) break;
        // the split-K partials are consumed: the bias partials reuse their buffer
        bias_partial_kernel<<<dim3((rows + 31) / 32, kBiasChunks), dim3(32, 8), 0, m->stream>>>(dz, B, rows,
                                                                                            m->wpart);
        if ((e = cudaGetLastError()) != cudaSuccess) break;
        if ((e = reduce_wgrad(m->wpart, kBiasChunks, rows, m->g + m->b_off[l], m->stream)) != cudaSuccess || l == 0)
            break;
        if (ldT > B &&
            (e = cudaMemset2DAsync(m->dZt + B, ldT * sizeof(__nv_bfloat16), 0, (ldT - B) * sizeof(__nv_bfloat16),
                                   cols, m->stream)) != cudaSuccess)
            break;
        GemmArgs gd{};
        gd.A = dz; gd.sam = rows; gd.sak = 1;
        gd.B = m->pbT + m->w_off[l]; gd.sbk = 1; gd.sbn = rows;   // W_l^T [cols][rows]
        gd.M = (int)B; gd.N = cols; gd.K = rows;
        gd.C = nullptr;
        gd.Zin = m->Z[l - 1]; gd.ldz = cols;
        gd.H = dz_next; gd.ldh = cols;
        gd.Ht = m->dZt; gd.ldht = ldT;
        e = gemm(gd, kEpiSiluBwd, 1, m->stream);
        std::swap(dz, dz_next);
    }
    return e;
}

hjg_status mlp_loss_and_grads(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy,
                              int64_t B, double* loss_out) {
    hjg_status s = mlp_ensure(m, B);
    if (s) return s;
    cudaStream_t st = m->stream;
    pack_input_kernel<<<nblk(B * m->in_pad), 256, 0, st>>>(x, ldx, B, m->n_in, m->in_pad, m->iscal, m->X);
    if (cudaGetLastError() != cudaSuccess || mlp_forward(m, B, true) != cudaSuccess) return HJG_ECUDA;
    const int64_t nb = (B * m->out_pad + 255) / 256;
    loss_grad_kernel<<<(unsigned)nb, 256, 0, st>>>(m->Z[kLayers - 1], m->out_pad, y, ldy, B, m->n_out,
                                                   m->out_pad, m->oscal, m->dZ, nullptr, m->lpart);
    if (cudaGetLastError() != cudaSuccess || mlp_backward(m, B) != cudaSuccess) return HJG_ECUDA;
    if (loss_out) {
        std::vector<double> part((size_t)nb);
        if (cudaMemcpyAsync(part.data(), m->lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return HJG_ECUDA;
        double l = 0.0;
        for (double v : part) l += v;
        *loss_out = l;
    }
    return HJG_OK;
}

// ------------------------------------------------------------------------------------
// Fused training step of the width-256 network (in_pad, out_pad <= 64), three launches:
//   A  a pair of CTAs (a thread-block cluster of two) per 128 batch rows runs the whole
//      forward pass, the loss and the backward data-gradient pass through all four layers on
//      the tensor cores.  Each CTA computes half of every 256-wide layer (128 output columns):
//      the layer's input sits in shared memory in the canonical K-major layout, the CTA's half
//      of the weights arrives by one bulk copy (issued while the previous layer's epilogue
//      runs), the 128 x 128 FP32 accumulator lives in TMEM, and the epilogue writes the CTA's
//      half of the next layer's input to shared memory, from where one bulk copy
//      (shared::cta -> the partner's shared::cluster, completion counted on the partner's
//      mbarrier) hands it to the partner: activations never leave the pair between layers.
//      The narrow output layer (N = out_pad) is computed by both CTAs.  The epilogue also
//      writes what the weight gradients need (H_l^T, dZ_l^T, X^T); the pre-activations Z_l
//      stay in TMEM (the accumulator and Z_0..Z_2 fill its 512 columns) for the backward pass;
//   B  the weight gradients dW_l = dZ_l^T H_{l-1} as 128 x N tiles (N = the layer's input
//      width, up to 256) over a split of the batch (split-K), TMA-fed four-stage pipeline;
//   C  the fixed-order sum of the splits, the bias gradients (column sums of dZ_l), Adam and
//      the BF16 weight copies (row-major, transposed, canonical) for the next step.
constexpr int kFW = 256;                         // width of the fused network
constexpr int kFHalf = 128;                      // output columns per CTA of a pair
constexpr int kFRows = 128;                      // batch rows per CTA pair (one M = 128 tile)
constexpr int kFThreads = 512;                   // 16 warps: TMEM lane quarter w % 4, column group w / 4
constexpr int kFBuf = kFRows * kFW * 2;          // 64 KB: a layer input (K <= 256), canonical K-major; two of them
constexpr int kFBufW = kFHalf * kFW * 2;         // 64 KB: this CTA's half of a layer's weights, canonical K-major
constexpr int kFPass = 16;                       // columns per epilogue pass of one column group
constexpr int kFStage = 4 * kFPass * kFRows * 2;  // 16 KB: one pass of the four column groups, transposed
constexpr int kFBias = kLayers * kFW * 4;         // 4 KB: the biases of the four layers
constexpr int kFSmemA = 2 * kFBuf + kFBufW + kFStage + kFBias;
constexpr uint32_t kFHalfBytes = kFRows * kFHalf * 2;   // 32 KB: one CTA's half of a 256-wide layer input
constexpr int kFTmemCols = 4 * kFHalf;   // TMEM: the accumulator, then Z_0, Z_1, Z_2 (128 columns each)
constexpr int kWgSplits = 16;                    // phase B split of the batch
constexpr int kWgStages = 4;                     // (32 splits at 2 stages, two CTAs per SM: 30 % slower)
constexpr int kWgStage = (kTcM + kFW) * kTcK * 2;   // A 128 rows + B up to 256 rows, one 64-wide K chunk
constexpr int kWgSmem = kWgStages * kWgStage + 1024;   // + slack to start the stages on 1,024 bytes

// Offset (elements) of element (r, k) of an [R][K] operand in the canonical K-major
// no-swizzle layout: core matrices of 8 rows x 8 K values (16 bytes a row), ordered
// [K / 8][R][8] -- core matrices 128 B apart along the rows and R x 16 B apart along K.
__host__ __device__ inline int64_t canon_idx(int64_t r, int64_t k, int64_t R) {
    return ((k >> 3) * R + r) * 8 + (k & 7);
}

// Offset of W(r, k) of an R x K weight operand in the canonical BF16 copies: a 256-row
// operand is stored as two 128-row halves [half][K / 8][128][8], so that each CTA of a
// pair loads its half with one contiguous copy; narrower operands are one block.
__host__ __device__ inline int64_t canon_w_idx(int64_t r, int64_t k, int64_t R, int64_t K) {
    if (R == kFW) return (r / kFHalf) * kFHalf * K + canon_idx(r % kFHalf, k, kFHalf);
    return canon_idx(r, k, R);
}

// Bulk copy of `bytes` from this CTA's shared memory to the same offset in the partner
// CTA's (rank `peer` of the cluster), completion counted on the partner's mbarrier at the
// same offset as `bar` here.
__device__ __forceinline__ void bulk_s2peer(uint32_t src, uint32_t bytes, uint32_t bar, uint32_t peer) {
    uint32_t dst, rbar;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(dst) : "r"(src), "r"(peer));
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(rbar) : "r"(bar), "r"(peer));
    asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "r"(src), "r"(bytes), "r"(rbar) : "memory");
}

// Four bytes from global to shared memory without a register round trip (zero-filled when
// `valid` is false, reading nothing); completed by cp_async_wait_all in the issuing thread.
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" :: "r"(dst), "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Every thread of both CTAs of the pair (release / acquire at cluster scope).
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    mbar_expect_tx(bar, bytes);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 :: "r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// D (TMEM) += A (128 x K, canonical at a) * B^T (rowsB x K, canonical at b) over the K steps
// [ks0, ks0 + nks) of 16 K values; the first step overwrites the accumulator when `first`.
__device__ __forceinline__ void mma_steps(uint32_t tmem, uint32_t a, uint32_t b, int rowsB, int ks0, int nks,
                                          bool first, uint32_t idesc) {
    for (int ks = ks0; ks < ks0 + nks; ++ks) {
        const uint64_t da = umma_desc(a + (uint32_t)(ks * kFRows * 32), kFRows * 16, 128);
        const uint64_t db = umma_desc(b + (uint32_t)(ks * rowsB * 32), (uint32_t)rowsB * 16, 128);
        const uint32_t acc = first && ks == ks0 ? 0u : 1u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
            :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" :: "r"(bar) : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t addr, float* x) {
    uint32_t v[32];
#pragma unroll
    for (int q = 0; q < 4; ++q)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[8 * q]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]),
              "=r"(v[8 * q + 4]), "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
            : "r"(addr + (uint32_t)(8 * q)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) x[j] = __uint_as_float(v[j]);
}

// Eight BF16 values of one row into the canonical layout of a 128-row operand (k0 % 8 == 0).
__device__ __forceinline__ void st_canon8(__nv_bfloat16* buf, int row, int k0, const float* v) {
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __float2bfloat16(v[j]);
    *reinterpret_cast<uint4*>(buf + canon_idx(row, k0, kFRows)) = *reinterpret_cast<const uint4*>(h);
}

struct FusedArgs {
    const float* x; int64_t ldx; const float* y; int64_t ldy; int64_t B; int64_t ldT;
    int n_in, n_out, in_pad, out_pad;
    const float* iscal; const float* oscal;          // [shift | mul] of inputs and targets
    const float* p;                                  // FP32 parameters (biases read from here)
    int64_t b_off[kLayers], wp_off[kLayers];
    const __nv_bfloat16* wc; const __nv_bfloat16* wct;
    __nv_bfloat16* Xt; __nv_bfloat16* Ht[kLayers - 1]; __nv_bfloat16* dZt[kLayers];
    double* lpart;                                   // loss / B per CTA
    int* err;
};

// 16 consecutive FP32 columns into this thread's TMEM lane.
__device__ __forceinline__ void tmem_st16(uint32_t addr, const float* x) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};"
            :: "r"(addr + (uint32_t)(8 * q)), "r"(__float_as_uint(x[8 * q])), "r"(__float_as_uint(x[8 * q + 1])),
               "r"(__float_as_uint(x[8 * q + 2])), "r"(__float_as_uint(x[8 * q + 3])),
               "r"(__float_as_uint(x[8 * q + 4])), "r"(__float_as_uint(x[8 * q + 5])),
               "r"(__float_as_uint(x[8 * q + 6])), "r"(__float_as_uint(x[8 * q + 7]))
            : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t addr, float* x) {
    uint32_t v[16];
#pragma unroll
    for (int q = 0; q < 2; ++q)
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(v[8 * q]), "=r"(v[8 * q + 1]), "=r"(v[8 * q + 2]), "=r"(v[8 * q + 3]),
              "=r"(v[8 * q + 4]), "=r"(v[8 * q + 5]), "=r"(v[8 * q + 6]), "=r"(v[8 * q + 7])
            : "r"(addr + (uint32_t)(8 * q)));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = __uint_as_float(v[j]);
}

// One pass of a tile, transposed: every thread has put its row's kFPass values into the
// staging tile [group][kFPass columns][128 rows] (BF16, one group per column quarter of
// the layer); the CTA writes them as 16-byte pieces of the destination's rows
// dst[c + column][r0 + row] with c = cbase + group * gstride (columns below cmax, rows below
// ldT), so that each store covers eight consecutive batch rows of one column.
__device__ __forceinline__ void store_transposed(const __nv_bfloat16* stg, __nv_bfloat16* dst, int64_t ldT,
                                                 int64_t r0, int gstride, int cbase, int cmax, int tid) {
    constexpr int kPieces = 4 * kFPass * (kFRows / 8);
#pragma unroll
    for (int i = 0; i < kPieces / kFThreads; ++i) {
        const int q = tid + kFThreads * i;
        const int grp = q / (kFPass * 16), col = (q / 16) % kFPass, rc = q % 16;
        const int c = cbase + grp * gstride + col;
        const int64_t b = r0 + 8 * rc;
        if (c < cmax && b < ldT)
            *reinterpret_cast<uint4*>(dst + (int64_t)c * ldT + b) =
                *reinterpret_cast<const uint4*>(stg + ((grp * kFPass + col) * kFRows + 8 * rc));
    }
}

// Product t of the fused step (0-2 hidden layers, 3 output layer, 4-6 backward data
// gradients): this CTA's weights (canonical copy; the half of rank `rank` for the 256-row
// operands, all of the output layer's), N (rows of the B operand) and K.
__device__ __forceinline__ int fused_k(const FusedArgs& a, int t) {
    return t == 0 ? a.in_pad : t == 4 ? a.out_pad : kFW;
}
__device__ __forceinline__ int fused_n(const FusedArgs& a, int t) { return t == 3 ? a.out_pad : kFHalf; }
__device__ __forceinline__ const __nv_bfloat16* fused_w(const FusedArgs& a, int t, uint32_t rank) {
    const int64_t half = t == 3 ? 0 : (int64_t)rank * kFHalf * fused_k(a, t);
    switch (t) {
    case 0: return a.wc + a.wp_off[0] + half;
    case 1: return a.wc + a.wp_off[1] + half;
    case 2: return a.wc + a.wp_off[2] + half;
    case 3: return a.wc + a.wp_off[3];
    case 4: return a.wct + a.wp_off[3] + half;
    case 5: return a.wct + a.wp_off[2] + half;
    default: return a.wct + a.wp_off[1] + half;
    }
}
__device__ __forceinline__ __nv_bfloat16* fused_t(const FusedArgs& a, bool fwd, int l) {
    if (fwd) return l == 0 ? a.Ht[0] : l == 1 ? a.Ht[1] : a.Ht[2];
    return l == 0 ? a.dZt[0] : l == 1 ? a.dZt[1] : a.dZt[2];
}

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kFThreads, 1)
    mlp_fused_fwdbwd_kernel(const __grid_constant__ FusedArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_w, bar_m, bar_x;
    __shared__ uint32_t tmem_base;
    __shared__ float s_loss[kFThreads / 32];
    __shared__ float s_isc[128], s_osc[128];   // inputs [shift | mul], targets [shift | 1 / mul]
    __shared__ int s_ok;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, cg = warp >> 2;             // TMEM lane quarter, column group (of 4)
    const int row = 32 * quarter + lane;                       // this thread's TMEM lane = tile row
    uint32_t rank;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(rank));
    const uint32_t peer = rank ^ 1u;
    const int hcol = (int)rank * kFHalf;                       // first layer column of this CTA's half
    const int64_t r0 = (int64_t)(blockIdx.x >> 1) * kFRows;
    const int64_t rg = r0 + row;                               // batch row
    const bool valid = rg < a.B;
    const uint32_t sbuf = smem_u32(smem), sW = sbuf + 2 * kFBuf;
    __nv_bfloat16* stg = reinterpret_cast<__nv_bfloat16*>(smem + 2 * kFBuf + kFBufW);
    float* s_bias = reinterpret_cast<float*>(smem + 2 * kFBuf + kFBufW + kFStage);   // [4][256]
    const uint32_t bw = smem_u32(&bar_w), bm = smem_u32(&bar_m), bx = smem_u32(&bar_x);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kFTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bw));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bm));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(bx));
        asm volatile("fence.mbarrier_init.release.cluster;");
        s_ok = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t tl = tmem + ((uint32_t)(32 * quarter) << 16);   // this warp's TMEM lanes
    // launched as a programmatic dependent of the previous kernel in the stream: the set-up
    // above overlaps its tail, and nothing global is read before it has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    uint32_t ph_w = 0, ph_m = 0, ph_x = 0;
    bool w_pending = false;   // thread 0: a weight copy in flight that no wait has consumed
    const int ip = a.in_pad, op = a.out_pad;
    if (tid == 0) {
        bulk_g2s(sW, fused_w(a, 0, rank), (uint32_t)(fused_n(a, 0) * fused_k(a, 0) * 2), bw);
        w_pending = true;
        mbar_expect_tx(bx, kFHalfBytes);   // the partner's half of the first hidden layer
    }

    // biases of the four layers, and the input tile in buffer 0: standardised features in
    // BF16 (zero beyond n_in and beyond the batch)
    for (int e = tid; e < kLayers * kFW; e += kFThreads) {
        const int l = e / kFW, i = e % kFW;
        s_bias[e] = i < (l == kLayers - 1 ? op : kFW) ? a.p[a.b_off[l] + i] : 0.0f;
    }
    if (tid < 2 * ip) s_isc[tid] = a.iscal[tid];
    else if (tid >= 128 && tid < 128 + op) s_osc[tid - 128] = a.oscal[tid - 128];
    else if (tid >= 256 && tid < 256 + op) s_osc[op + tid - 256] = 1.0f / a.oscal[op + tid - 256];
    __nv_bfloat16* buf0 = reinterpret_cast<__nv_bfloat16*>(smem);
    {   // the raw input tile [128][ip] FP32 into buffer 1 (free until the partner's first copy,
        // which comes after the cluster barrier below) by asynchronous copies, then
        // standardised into buffer 0 in the canonical layout
        float* xr = reinterpret_cast<float*>(smem + kFBuf);
        const uint32_t sxr = smem_u32(xr);
        for (int e = tid; e < kFRows * ip; e += kFThreads) {
            const int r = e / ip, j = e % ip;
            const int64_t b = r0 + r;
            const bool ok = b < a.B && j < a.n_in;
            cp_async4(sxr + 4u * (uint32_t)e, ok ? (const void*)(a.x + b * a.ldx + j) : (const void*)a.x, ok);
        }
        cp_async_wait_all();
        __syncthreads();
        for (int e = tid; e < kFRows * ip; e += kFThreads) {
            const int r = e / ip, j = e % ip;
            buf0[canon_idx(r, j, kFRows)] =
                __float2bfloat16(j < a.n_in ? (xr[e] - s_isc[j]) * s_isc[ip + j] : 0.0f);
        }
    }
    __syncthreads();
    {   // X^T, the K-major operand of dW_1: each CTA of the pair writes half of its columns
        const int half = kFRows * ip / 2;
        for (int e = (int)rank * half + tid; e < ((int)rank + 1) * half; e += kFThreads) {
            const int j = e / kFRows, r = e % kFRows;
            if (r0 + r < a.ldT) a.Xt[(int64_t)j * a.ldT + r0 + r] = buf0[canon_idx(r, j, kFRows)];
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    cluster_sync();   // both CTAs' barriers are initialised before any copy reaches them

    // Step t reads buffer t % 2 and writes the next input into buffer (t + 1) % 2.  The
    // partner's half arrives (on bar_x) for the inputs of steps 1, 2, 3, 5 and 6; this CTA
    // sends its half after steps 0, 1, 2, 4 and 5.  A copy into the partner's buffer
    // (t + 1) % 2 cannot overtake the partner's product t - 1 that reads it: this CTA's
    // product t needed the partner's output of step t - 1, written after that product --
    // except after step 3, whose inputs are local, hence the cluster barrier there.  The
    // sequence of cluster barriers is the same on every path (a failed wait skips work, not
    // barriers), so neither CTA can wait on one the other never reaches.
    float loss = 0.0f;
    for (int t = 0; t < 7; ++t) {
        const bool recv = t == 1 || t == 2 || t == 3 || t == 5 || t == 6;
        const bool send = t == 0 || t == 1 || t == 2 || t == 4 || t == 5;
        const uint32_t s_in = sbuf + (uint32_t)((t & 1) * kFBuf);
        __nv_bfloat16* out = reinterpret_cast<__nv_bfloat16*>(smem + ((t + 1) & 1) * kFBuf);
        // the output layer's targets of the tile, copied row by row (coalesced) by warps 1-15
        // while thread 0 waits for the product, into the upper half of buffer 0:
        // nothing reads or writes it during step 3 (its inputs were consumed by product 2, dO
        // goes to the lower half, and the partner's next copy into it comes after step 3)
        float* ys = reinterpret_cast<float*>(smem + kFBuf / 2);
        if (t == 3 && warp > 0) {   // raw, by asynchronous copies; standardised at use
            const uint32_t sys = smem_u32(ys);
            for (int e = tid - 32; e < kFRows * op; e += kFThreads - 32) {
                const int r = e / op, col = e % op;
                const int64_t b = r0 + r;
                const bool ok = b < a.B && col < a.n_out;
                cp_async4(sys + 4u * (uint32_t)e, ok ? (const void*)(a.y + b * a.ldy + col) : (const void*)a.y, ok);
            }
            cp_async_wait_all();
        }
        // thread 0: the product of step t once its weights (and the partner's half of its
        // input) have landed, and its completion; the other threads wait at the barrier
        if (tid == 0 && s_ok) {
            bool ok = mbar_wait(bw, ph_w, a.err);
            if (ok) { w_pending = false; ph_w ^= 1u; }
            if (ok) {
                const int n = fused_n(a, t), kst = fused_k(a, t) / 16;
                const uint32_t idesc = umma_idesc_bf16(kFRows, n);
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (recv) {
                    // this CTA's half of the input (its own epilogue wrote it) while the
                    // partner's half is still on its way, then the partner's half
                    const int kh = kFHalf / 16;
                    mma_steps(tmem, s_in, sW, n, (int)rank * kh, kh, true, idesc);
                    ok = mbar_wait(bx, ph_x, a.err);
                    if (ok) {
                        ph_x ^= 1u;
                        if (t != 6) mbar_expect_tx(bx, kFHalfBytes);   // the next reception
                        mma_steps(tmem, s_in, sW, n, (int)peer * kh, kh, false, idesc);
                    }
                } else {
                    mma_steps(tmem, s_in, sW, n, 0, kst, true, idesc);
                }
                mma_commit(bm);   // also after a failed wait: the issued products must finish
                const bool done = mbar_wait(bm, ph_m, a.err);
                ph_m ^= 1u;
                ok = ok && done;
            }
            if (!ok) s_ok = 0;
        }
        __syncthreads();   // operands free, accumulator complete (or a wait gave up)
        asm volatile("tcgen05.fence::after_thread_sync;");
        const bool ok = s_ok != 0;   // uniform over the CTA
        if (t == 3) cluster_sync();  // both products of step 3 are done with buffer 1
        if (ok && tid == 0 && t + 1 < 7) {
            bulk_g2s(sW, fused_w(a, t + 1, rank), (uint32_t)(fused_n(a, t + 1) * fused_k(a, t + 1) * 2), bw);
            w_pending = true;
        }
        // staging tile of this thread: column j of its group, its row
        __nv_bfloat16* my_stg = stg + cg * kFPass * kFRows + row;
        if (ok && t != 3) {
            // hidden layer t (t < 3): z = acc + b -> Z_t (TMEM), h = silu(z) -> next input, H_t^T;
            // backward (t = 4, 5, 6): dZ_l = (dZ_{l+1} W_{l+1}) silu'(Z_l) for the hidden layer
            // l = 6 - t (2, 1, 0) -> next input (l > 0), dZ_l^T; 32 columns per thread
            const bool fwd = t < 3;
            const int l = fwd ? t : 6 - t;
            __nv_bfloat16* tdst = fused_t(a, fwd, l);
            const uint32_t tz = tl + (uint32_t)(kFHalf * (l + 1) + cg * 32);   // Z_l, this thread's 32 columns
            float acc[32];
            float zin[32];
            tmem_ld32(tl + (uint32_t)(cg * 32), acc);
            if (!fwd) tmem_ld32(tz, zin);
#pragma unroll
            for (int pass = 0; pass < 32 / kFPass; ++pass) {
                const int c0 = hcol + cg * 32 + kFPass * pass;   // layer column
                float* v = acc + kFPass * pass;
                if (fwd) {
                    const float* bias = s_bias + t * kFW + c0;
#pragma unroll
                    for (int j = 0; j < kFPass; ++j) v[j] += bias[j];
                    tmem_st16(tz + (uint32_t)(kFPass * pass), v);   // Z_t stays on the SM for the backward pass
#pragma unroll
                    for (int j = 0; j < kFPass; ++j) v[j] = valid ? silu_t(v[j]) : 0.0f;
                } else {
#pragma unroll
                    for (int j = 0; j < kFPass; ++j) {
                        const float z = zin[kFPass * pass + j];
                        const float sg = sigmoid_t(z);
                        v[j] = valid ? v[j] * sg * (1.0f + z * (1.0f - sg)) : 0.0f;
                    }
                }
                if (fwd || l > 0) {
#pragma unroll
                    for (int g = 0; g < kFPass / 8; ++g) st_canon8(out, row, c0 + 8 * g, v + 8 * g);
                }
#pragma unroll
                for (int j = 0; j < kFPass; ++j) my_stg[j * kFRows] = __float2bfloat16(v[j]);
                __syncthreads();
                store_transposed(stg, tdst, a.ldT, r0, 32, hcol + kFPass * pass, kFW, tid);
                __syncthreads();
            }
            if (fwd) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        } else if (ok) {
            // output layer (both CTAs): o = acc + b, dO against the standardised targets ->
            // next input; the loss and dO^T from rank 0; each column group covers kFPass of
            // the (at most 64) outputs
            const int c0 = cg * kFPass;
            float v[kFPass];
            if (c0 < op) {
                tmem_ld16(tl + (uint32_t)c0, v);
                const float winv = a.n_out > 1 ? 1.0f / (float)(a.n_out - 1) : 0.0f;
#pragma unroll
                for (int j = 0; j < kFPass; ++j) {
                    const int col = c0 + j;
                    float g = 0.0f;
                    if (valid && col < a.n_out) {
                        const float o = v[j] + s_bias[3 * kFW + col];
                        const float d = o - (ys[row * op + col] - s_osc[col]) * s_osc[op + col];
                        const float w = col == 0 ? 1.0f : winv;
                        if (rank == 0) loss += w * d * d;
                        g = 2.0f * w * d / (float)a.B;
                    }
                    v[j] = g;
                }
#pragma unroll
                for (int g = 0; g < kFPass / 8; ++g) st_canon8(out, row, c0 + 8 * g, v + 8 * g);
            } else {
#pragma unroll
                for (int j = 0; j < kFPass; ++j) v[j] = 0.0f;
            }
#pragma unroll
            for (int j = 0; j < kFPass; ++j) my_stg[j * kFRows] = __float2bfloat16(v[j]);
            __syncthreads();
            if (rank == 0) store_transposed(stg, a.dZt[3], a.ldT, r0, kFPass, 0, op, tid);
            __syncthreads();
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (ok && send && tid == 0)   // this CTA's half of the next input to the partner
            bulk_s2peer(smem_u32(out) + (uint32_t)rank * kFHalfBytes, kFHalfBytes, bx, peer);
    }
    // the loss of this tile (FP32 per thread, then the warps in a fixed order)
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) loss += __shfl_xor_sync(0xffffffffu, loss, off);
    if (lane == 0) s_loss[warp] = loss;
    if (tid == 0 && w_pending) mbar_wait(bw, ph_w, a.err);   // no copy may land after the exit
    __syncthreads();
    if (tid == 0 && rank == 0) {
        float t = 0.0f;
        for (int w = 0; w < kFThreads / 32; ++w) t += s_loss[w];
        a.lpart[blockIdx.x >> 1] = (double)t / (double)a.B;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");   // every global write is done
    // neither CTA leaves while the partner may still copy into its shared memory: every copy
    // was consumed by the receiver's wait before the receiver reached this barrier
    cluster_sync();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kFTmemCols));
}

// Phase B: split-K weight gradients.  Item i = (layer, 128-row tile of dW_l), split s of the
// batch: part[s][wp_off[l] + r cols_l + c] = sum over its batch rows of dZ_l^T[r][b] X_l^T[c][b]
// (X_l = the layer's input: X, H_1, H_2, H_3).  Both operands are K-major in global memory
// (K = the batch) and arrive by TMA, 8-element K slices of 128 (A) and cols_l (B) rows.
struct WgradArgs {
    CUtensorMap ta[kLayers], tb[kLayers];
    int rows[kLayers], cols[kLayers];
    int64_t wp_off[kLayers], n_w, K;
    int item_l[8], item_m[8];
    int splits, kper;
    float* part;
    int* err;
};

__global__ void __launch_bounds__(128, 1) mlp_wgrad_kernel(const __grid_constant__ WgradArgs g) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages];
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int item = blockIdx.x / g.splits, split = blockIdx.x % g.splits;
    const int l = g.item_l[item], m0 = g.item_m[item] * kTcM;
    const int N = g.cols[l];
    const int64_t kbeg = (int64_t)split * g.kper, kend = min(g.K, kbeg + g.kper);
    const int nch = kend > kbeg ? (int)((kend - kbeg + kTcK - 1) / kTcK) : 0;
    const uint32_t s0 = (smem_u32(smem) + 1023u) & ~1023u;   // the swizzle pattern repeats every 1,024 B
    const uint32_t stage_bytes = (uint32_t)((kTcM + N) * kTcK * 2);
    const CUtensorMap* tmA = &g.ta[l];
    const CUtensorMap* tmB = &g.tb[l];
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"(smem_u32(&tmem_base)), "r"(kFW));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
#pragma unroll
        for (int i = 0; i < kWgStages; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&full[i])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(&empty[i])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    const uint32_t idesc = umma_idesc_bf16(kTcM, N);
    asm volatile("griddepcontrol.wait;" ::: "memory");   // phase A's operands are complete
    auto chunk = [&](uint32_t st, int64_t k0, uint32_t bar) {   // A rows then B rows, 128 B each
        mbar_expect_tx(bar, stage_bytes);
        tma_load_2d(st, tmA, (int)k0, m0, bar);
        tma_load_2d(st + (uint32_t)(kTcM * kTcK * 2), tmB, (int)k0, 0, bar);
    };
    bool ok = true;
    if (tid == 0 && nch > 0) {
        // chunk c uses stage c % S; its copies complete phase c / S of full[c % S] and its
        // products' commit phase c / S of empty[c % S], so every wait takes its parity from
        // the chunk index.  The stage of chunk c - 1 is refilled right after chunk c's
        // products are issued: the tensor core works on chunk c while chunk c - 1 retires.
        int issued = 0, landed = 0, last = -1;
        for (; issued < nch && issued < kWgStages; ++issued)
            chunk(s0 + (uint32_t)(issued * kWgStage), kbeg + (int64_t)issued * kTcK, smem_u32(&full[issued]));
        for (int c = 0; c < nch; ++c) {
            const int s = c % kWgStages;
            if (!mbar_wait(smem_u32(&full[s]), (uint32_t)(c / kWgStages) & 1u, g.err)) { ok = false; break; }
            landed = c + 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = s0 + (uint32_t)(s * kWgStage), sb = sa + kTcM * kTcK * 2;
#pragma unroll
            for (int ks = 0; ks < kTcK / 16; ++ks) {
                const uint64_t da = umma_desc_sw128(sa + (uint32_t)(ks * 32));
                const uint64_t db = umma_desc_sw128(sb + (uint32_t)(ks * 32));
                const uint32_t acc = (c > 0 || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
                    :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            mma_commit(smem_u32(&empty[s]));
            last = c;
            if (c >= 1 && issued < nch) {   // issued == c - 1 + S: the stage of chunk c - 1
                const int sp = (c - 1) % kWgStages;
                if (!mbar_wait(smem_u32(&empty[sp]), (uint32_t)((c - 1) / kWgStages) & 1u, g.err)) {
                    ok = false;
                    break;
                }
                chunk(s0 + (uint32_t)(sp * kWgStage), kbeg + (int64_t)issued * kTcK, smem_u32(&full[sp]));
                ++issued;
            }
        }
        // the last chunk's commit arrives once every product issued so far has completed
        if (last >= 0 &&
            !mbar_wait(smem_u32(&empty[last % kWgStages]), (uint32_t)(last / kWgStages) & 1u, g.err))
            ok = false;
        if (!ok)   // no copy may land after the exit
            for (int c = landed; c < issued; ++c)
                mbar_wait(smem_u32(&full[c % kWgStages]), (uint32_t)(c / kWgStages) & 1u, g.err);
    }
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    // the 128 x N tile through shared memory (the stages are free: every product has
    // completed), then out as consecutive 16-byte pieces of its contiguous rows
    const int row = warp * 32 + lane;
    const bool have = ok && nch > 0;   // uniform over the CTA: the TMEM loads are warp-collective
    const int ldt = N + 4;             // padded row of the staging tile (floats)
    float* stile = reinterpret_cast<float*>(smem + (s0 - smem_u32(smem)));
    for (int c0 = 0; c0 < N; c0 += 32) {
        float v[32];
        if (have) {
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = 0.0f;
        }
        const int nv = min(32, N - c0);   // N is a multiple of 16
        for (int q = 0; q < nv / 4; ++q)
            *reinterpret_cast<float4*>(stile + row * ldt + c0 + 4 * q) =
                make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    const int nrow = min(kTcM, g.rows[l] - m0);
    float* dst = g.part + (int64_t)split * g.n_w + g.wp_off[l] + (int64_t)m0 * N;
    for (int i = tid; i < nrow * N / 4; i += 128) {
        const int r = (4 * i) / N, c = (4 * i) % N;
        reinterpret_cast<float4*>(dst)[i] = *reinterpret_cast<const float4*>(stile + r * ldt + c);
    }
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(kFW));
}

// Phase C: gradients and (with lr > 0) the Adam step and the BF16 weight copies.  Blocks
// [0, nwb): one 8 x 32 weight tile each, the splits added in order; blocks [nwb, ...): one
// block per bias, the column sum of dZ_l over the batch (eight warps over the rows, lanes
// within a warp, then fixed-order combines).
struct ApplyArgs {
    int64_t w_off[kLayers], b_off[kLayers], wp_off[kLayers], n_w;
    int rows[kLayers], cols[kLayers];
    const float* part; int splits;
    const __nv_bfloat16* dZt[kLayers]; int64_t ldT, B;
    float* p; float* g; float* m1; float* m2;
    __nv_bfloat16* pb; __nv_bfloat16* pbT; __nv_bfloat16* wc; __nv_bfloat16* wct;
    float lr, b1, b2, eps, c1, c2;
    int nwb, n_bias;
    int tile_off[kLayers + 1];   // first block of each layer's 8 x 32 weight tiles
};

__device__ __forceinline__ float adam_update(const ApplyArgs& a, int64_t pi, float gg) {
    const float m = a.b1 * a.m1[pi] + (1.0f - a.b1) * gg;
    const float v = a.b2 * a.m2[pi] + (1.0f - a.b2) * gg * gg;
    a.m1[pi] = m;
    a.m2[pi] = v;
    const float nw = a.p[pi] - a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
    a.p[pi] = nw;
    a.pb[pi] = __float2bfloat16(nw);
    return nw;
}

__global__ void __launch_bounds__(256) mlp_apply_kernel(const ApplyArgs a) {
    asm volatile("griddepcontrol.wait;" ::: "memory");   // the weight-gradient partials are complete
    if ((int)blockIdx.x < a.nwb) {
        // one block per 8 x 32 tile of one layer's weights, one weight per thread: the split
        // sums, the gradient and Adam (row-major, coalesced), then the BF16 copies through a
        // shared tile so that the transposed and canonical copies go out as 16-byte or longer
        // runs
        __shared__ __nv_bfloat16 sh[8][34];
        int l = 0;
        while (l + 1 < kLayers && (int)blockIdx.x >= a.tile_off[l + 1]) ++l;
        const int R = a.rows[l], Cc = a.cols[l];
        const int tcn = (Cc + 31) / 32, t = (int)blockIdx.x - a.tile_off[l];
        const int r0 = (t / tcn) * 8, c0 = (t % tcn) * 32;
        const int tid = threadIdx.x;
        {
            const int r = tid >> 5, c = tid & 31;
            if (r0 + r < R && c0 + c < Cc) {
                const int64_t k = (int64_t)(r0 + r) * Cc + c0 + c;
                const int64_t e = a.wp_off[l] + k;
                float part[kWgSplits];
#pragma unroll
                for (int q = 0; q < kWgSplits; ++q) part[q] = a.part[(int64_t)q * a.n_w + e];
                float sum = 0.0f;
#pragma unroll
                for (int q = 0; q < kWgSplits; ++q) sum += part[q];
                const int64_t pi = a.w_off[l] + k;
                a.g[pi] = sum;
                if (a.lr > 0.0f) sh[r][c] = __float2bfloat16(adam_update(a, pi, sum));
            }
        }
        if (!(a.lr > 0.0f)) return;   // uniform over the block
        __syncthreads();
        {   // W^T row-major: 8 consecutive rows of W per column
            const int c = tid >> 3, r = tid & 7;
            if (r0 + r < R && c0 + c < Cc) a.pbT[a.w_off[l] + (int64_t)(c0 + c) * R + r0 + r] = sh[r][c];
        }
        {   // canonical W: 8 columns of the 8 rows
            const int c = 8 * (tid >> 6) + (tid & 7), r = (tid >> 3) & 7;
            if (r0 + r < R && c0 + c < Cc) a.wc[a.wp_off[l] + canon_w_idx(r0 + r, c0 + c, R, Cc)] = sh[r][c];
        }
        {   // canonical W^T: the 8 rows of W for consecutive columns
            const int c = tid >> 3, r = tid & 7;
            if (r0 + r < R && c0 + c < Cc) a.wct[a.wp_off[l] + canon_w_idx(c0 + c, r0 + r, Cc, R)] = sh[r][c];
        }
        return;
    }
    // one block per bias: warp w sums the batch rows [w B / 8, (w + 1) B / 8) of its dZ_l^T row,
    // then thread 0 adds the eight warp sums in order
    __shared__ float s_part[8];
    const int gb = (int)blockIdx.x - a.nwb, warp = (int)(threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (gb >= a.n_bias) return;
    int l = 0, i = gb;
    while (l + 1 < kLayers && i >= a.rows[l]) { i -= a.rows[l]; ++l; }
    const __nv_bfloat16* row = a.dZt[l] + (int64_t)i * a.ldT;   // 16-byte aligned (ldT % 8 == 0)
    const int64_t nfull = a.B / 8;                                // 8-row pieces
    const int64_t q0 = nfull * warp / 8, q1 = nfull * (warp + 1) / 8;
    float s = 0.0f;
#pragma unroll 4
    for (int64_t q = q0 + lane; q < q1; q += 32) {
        const uint4 u = *reinterpret_cast<const uint4*>(row + 8 * q);
        const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
        for (int j = 0; j < 8; ++j) s += __bfloat162float(h[j]);
    }
    if (warp == 7)
        for (int64_t b = 8 * nfull + lane; b < a.B; b += 32) s += __bfloat162float(row[b]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) s_part[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.0f;
        for (int w = 0; w < 8; ++w) t += s_part[w];
        const int64_t pi = a.b_off[l] + i;
        a.g[pi] = t;
        if (a.lr > 0.0f) adam_update(a, pi, t);
    }
}

// Canonical BF16 copies of the weights from the FP32 parameters (creation, set_params).
__global__ void canon_weights_kernel(const float* __restrict__ p, ApplyArgs a) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= a.n_w) return;
    int l = 0;
    while (l + 1 < kLayers && e >= a.wp_off[l + 1]) ++l;
    const int64_t k = e - a.wp_off[l];
    const int R = a.rows[l], Cc = a.cols[l];
    const int r = (int)(k / Cc), c = (int)(k % Cc);
    const __nv_bfloat16 hb = __float2bfloat16(p[a.w_off[l] + k]);
    a.wc[a.wp_off[l] + canon_w_idx(r, c, R, Cc)] = hb;
    a.wct[a.wp_off[l] + canon_w_idx(c, r, Cc, R)] = hb;
}

// Launch as a programmatic dependent of the previous kernel in the stream: its blocks may be
// scheduled while that kernel's last blocks finish; the kernel itself waits
// (griddepcontrol.wait) before its first global read.
template <typename Kern, typename Arg>
cudaError_t launch_dependent(Kern kern, unsigned grid, unsigned block, size_t smem, cudaStream_t st, const Arg& arg) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    memset(at, 0, sizeof at);
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, arg);
}

bool fused_ok(const hjg_mlp* m) {
    return m->width == kFW && m->in_pad <= 64 && m->out_pad <= 64 && m->wc && m->wct;
}

ApplyArgs apply_args(const hjg_mlp* m) {
    ApplyArgs a;
    memset(&a, 0, sizeof a);
    for (int l = 0; l < kLayers; ++l) {
        a.w_off[l] = m->w_off[l]; a.b_off[l] = m->b_off[l]; a.wp_off[l] = m->wp_off[l];
        a.rows[l] = m->rows[l]; a.cols[l] = m->cols[l];
        a.dZt[l] = m->dZt4[l];
    }
    a.n_w = m->n_w;
    a.part = m->fpart; a.splits = kWgSplits;
    a.p = m->p; a.g = m->g; a.m1 = m->m1; a.m2 = m->m2;
    a.pb = m->pb; a.pbT = m->pbT; a.wc = m->wc; a.wct = m->wct;
    a.tile_off[0] = 0;
    for (int l = 0; l < kLayers; ++l)
        a.tile_off[l + 1] = a.tile_off[l] + ((m->rows[l] + 7) / 8) * ((m->cols[l] + 31) / 32);
    a.nwb = a.tile_off[kLayers];
    int nb = 0;
    for (int l = 0; l < kLayers; ++l) nb += m->rows[l];
    a.n_bias = nb;
    return a;
}

cudaError_t refresh_canon(hjg_mlp* m, cudaStream_t st) {
    if (!m->wc) return cudaSuccess;
    const ApplyArgs a = apply_args(m);
    canon_weights_kernel<<<nblk(m->n_w), 256, 0, st>>>(m->p, a);
    return cudaGetLastError();
}

hjg_status fused_ensure(hjg_mlp* m, int64_t B) {
    if (B <= m->fcap) return HJG_OK;
    auto fre = [](void* p) { if (p) cudaFree(p); };
    fre(m->Xt); fre(m->fpart); fre(m->flpart);
    m->Xt = nullptr; m->fpart = nullptr; m->flpart = nullptr;
    for (int l = 0; l < kLayers; ++l) { fre(m->dZt4[l]); m->dZt4[l] = nullptr; }
    m->fcap = 0;
    const int64_t ldT = pad8(B);
    bool ok = cudaMalloc(&m->Xt, (size_t)m->in_pad * ldT * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->fpart, (size_t)kWgSplits * m->n_w * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->flpart, (size_t)((B + kFRows - 1) / kFRows) * sizeof(double)) == cudaSuccess;
    for (int l = 0; l < kLayers && ok; ++l)
        ok = cudaMalloc(&m->dZt4[l], (size_t)m->rows[l] * ldT * sizeof(__nv_bfloat16)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        m->err = "fused training buffers: out of memory";
        return HJG_ENOMEM;
    }
    m->fcap = B;
    return HJG_OK;
}

// One fused training step (lr > 0: gradients and Adam) or the gradients alone (lr = 0).
hjg_status mlp_fused_step(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t B,
                          float lr, double* loss_out) {
    hjg_status s = mlp_ensure(m, B);
    if (s || (s = fused_ensure(m, B))) return s;
    if (!g_tc_err) {
        if (cudaMalloc(&g_tc_err, sizeof(int)) != cudaSuccess || cudaMemset(g_tc_err, 0, sizeof(int)) != cudaSuccess)
            return HJG_ENOMEM;
    }
    cudaStream_t st = m->stream;
    const int64_t ldT = pad8(B);
    static bool attrA = false, attrB = false;
    if (!attrA) {
        if (cudaFuncSetAttribute(mlp_fused_fwdbwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFSmemA) !=
            cudaSuccess)
            return HJG_ECUDA;
        attrA = true;
    }
    if (!attrB) {
        if (cudaFuncSetAttribute(mlp_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem) !=
            cudaSuccess)
            return HJG_ECUDA;
        attrB = true;
    }
    FusedArgs fa;
    memset(&fa, 0, sizeof fa);
    fa.x = x; fa.ldx = ldx; fa.y = y; fa.ldy = ldy; fa.B = B; fa.ldT = ldT;
    fa.n_in = m->n_in; fa.n_out = m->n_out; fa.in_pad = m->in_pad; fa.out_pad = m->out_pad;
    fa.iscal = m->iscal; fa.oscal = m->oscal; fa.p = m->p;
    for (int l = 0; l < kLayers; ++l) { fa.b_off[l] = m->b_off[l]; fa.wp_off[l] = m->wp_off[l]; fa.dZt[l] = m->dZt4[l]; }
    fa.wc = m->wc; fa.wct = m->wct;
    for (int l = 0; l + 1 < kLayers; ++l) fa.Ht[l] = m->Ht[l];
    fa.Xt = m->Xt; fa.lpart = m->flpart; fa.err = g_tc_err;
    const int ntile = (int)((B + kFRows - 1) / kFRows);
    if (launch_dependent(mlp_fused_fwdbwd_kernel, 2u * (unsigned)ntile, kFThreads, kFSmemA, st, fa) !=
        cudaSuccess)   // clusters of two
        return HJG_ECUDA;

    WgradArgs wa;
    memset(&wa, 0, sizeof wa);
    int items = 0;
    for (int l = 0; l < kLayers; ++l) {
        wa.rows[l] = m->rows[l]; wa.cols[l] = m->cols[l]; wa.wp_off[l] = m->wp_off[l];
        const __nv_bfloat16* opB = l == 0 ? m->Xt : m->Ht[l - 1];
        if (!operand_map_sw128(&wa.ta[l], m->dZt4[l], m->rows[l], B, ldT, kTcM) ||
            !operand_map_sw128(&wa.tb[l], opB, m->cols[l], B, ldT, m->cols[l]))
            return HJG_ECUDA;
        for (int t = 0; t < (m->rows[l] + kTcM - 1) / kTcM; ++t) { wa.item_l[items] = l; wa.item_m[items] = t; ++items; }
    }
    wa.n_w = m->n_w; wa.K = B; wa.splits = kWgSplits;
    wa.kper = (int)(((B + kWgSplits - 1) / kWgSplits + kTcK - 1) / kTcK * kTcK);
    wa.part = m->fpart; wa.err = g_tc_err;
    if (launch_dependent(mlp_wgrad_kernel, (unsigned)(items * kWgSplits), 128, kWgSmem, st, wa) != cudaSuccess)
        return HJG_ECUDA;

    ApplyArgs aa = apply_args(m);
    aa.ldT = ldT; aa.B = B;
    aa.lr = lr;
    if (lr > 0.0f) {
        m->step += 1;
        aa.b1 = 0.9f; aa.b2 = 0.999f; aa.eps = 1e-8f;
        aa.c1 = 1.0f - powf(aa.b1, (float)m->step);
        aa.c2 = 1.0f - powf(aa.b2, (float)m->step);
    }
    if (launch_dependent(mlp_apply_kernel, (unsigned)(aa.nwb + aa.n_bias), 256, 0, st, aa) != cudaSuccess)
        return HJG_ECUDA;
    if (loss_out) {
        std::vector<double> part((size_t)ntile);
        if (cudaMemcpyAsync(part.data(), m->flpart, ntile * sizeof(double), cudaMemcpyDeviceToHost, st) !=
                cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return HJG_ECUDA;
        double l = 0.0;
        for (double v : part) l += v;
        *loss_out = l;
    }
    return HJG_OK;
}

}  // namespace

extern "C" {

hjg_status hjg_mlp_create(int n_in, int n_out, int width, uint64_t seed, hjg_mlp** out) {
    if (!out || n_in < 1 || n_in > 256 || n_out < 1 || n_out > 256 || width < 16 || width > 1024 ||
        width % 16 || pad16(n_out) > width || pad16(n_in) > width)
        return HJG_EINVAL;
    hjg_mlp* m = new (std::nothrow) hjg_mlp();
    if (!m) return HJG_ENOMEM;
    m->n_in = n_in; m->n_out = n_out; m->width = width;
    m->in_pad = pad16(n_in); m->out_pad = pad16(n_out);
    const int ins[kLayers] = {m->in_pad, width, width, width};
    const int outs[kLayers] = {width, width, width, m->out_pad};
    int64_t off = 0;
    for (int l = 0; l < kLayers; ++l) {
        m->rows[l] = outs[l]; m->cols[l] = ins[l];
        m->w_off[l] = off; off += (int64_t)outs[l] * ins[l];
        m->b_off[l] = off; off += outs[l];
    }
    m->n_params = off;
    int64_t woff = 0;
    for (int l = 0; l < kLayers; ++l) { m->wp_off[l] = woff; woff += (int64_t)m->rows[l] * m->cols[l]; }
    m->n_w = woff;
    const size_t nb = (size_t)off * sizeof(float);
    int64_t wpart = 0;
    for (int l = 0; l < kLayers; ++l) wpart = std::max<int64_t>(wpart, (int64_t)m->rows[l] * m->cols[l]);
    wpart *= kSplits;
    for (int l = 0; l < kLayers; ++l) wpart = std::max<int64_t>(wpart, (int64_t)kBiasChunks * m->rows[l]);
    if (cudaMalloc(&m->p, nb) != cudaSuccess || cudaMalloc(&m->g, nb) != cudaSuccess ||
        cudaMalloc(&m->m1, nb) != cudaSuccess || cudaMalloc(&m->m2, nb) != cudaSuccess ||
        cudaMalloc(&m->pb, (size_t)off * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&m->pbT, (size_t)off * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&m->iscal, 2 * (size_t)m->in_pad * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->oscal, 2 * (size_t)m->out_pad * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&m->wpart, (size_t)wpart * sizeof(float)) != cudaSuccess) {
        hjg_mlp_destroy(m);
        return HJG_ENOMEM;
    }
    if (width == kFW && m->in_pad <= 64 && m->out_pad <= 64 &&
        (cudaMalloc(&m->wc, (size_t)m->n_w * sizeof(__nv_bfloat16)) != cudaSuccess ||
         cudaMalloc(&m->wct, (size_t)m->n_w * sizeof(__nv_bfloat16)) != cudaSuccess)) {
        hjg_mlp_destroy(m);
        return HJG_ENOMEM;
    }
    cudaMemset(m->p, 0, nb);
    cudaMemset(m->m1, 0, nb);
    cudaMemset(m->m2, 0, nb);
    cudaMemset(m->g, 0, nb);
    const int used_in[kLayers] = {n_in, width, width, width};
    const int used_out[kLayers] = {width, width, width, n_out};
    for (int l = 0; l < kLayers; ++l) {
        const float scale = sqrtf(6.0f / (float)(used_in[l] + used_out[l]));
        const int64_t n = (int64_t)m->rows[l] * m->cols[l];
        init_weight_kernel<<<nblk(n), 256>>>(m->p + m->w_off[l], m->rows[l], m->cols[l], used_out[l],
                                             used_in[l], scale, seed * 31 + l);
    }
    to_bf16_kernel<<<nblk(off), 256>>>(m->p, m->pb, off);
    {   // identity scaling until hjg_mlp_fit_scaling / hjg_mlp_set_scaling
        std::vector<float> si(2 * (size_t)m->in_pad, 0.0f), so(2 * (size_t)m->out_pad, 0.0f);
        std::fill(si.begin() + m->in_pad, si.end(), 1.0f);
        std::fill(so.begin() + m->out_pad, so.end(), 1.0f);
        cudaMemcpy(m->iscal, si.data(), si.size() * sizeof(float), cudaMemcpyHostToDevice);
        cudaMemcpy(m->oscal, so.data(), so.size() * sizeof(float), cudaMemcpyHostToDevice);
    }
    if (refresh_wt(m, nullptr) != cudaSuccess || refresh_canon(m, nullptr) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        hjg_mlp_destroy(m);
        return HJG_ECUDA;
    }
    *out = m;
    return HJG_OK;
}

void hjg_mlp_destroy(hjg_mlp* m) {
    if (!m) return;
    auto fre = [](void* p) { if (p) cudaFree(p); };
    fre(m->p); fre(m->g); fre(m->m1); fre(m->m2); fre(m->pb); fre(m->pbT); fre(m->iscal); fre(m->oscal);
    fre(m->wpart); fre(m->packA);
    fre(m->packB); fre(m->X); fre(m->dZ); fre(m->dZ2); fre(m->dZt); fre(m->dH); fre(m->lpart);
    for (int l = 0; l < kLayers; ++l) { fre(m->Z[l]); fre(m->H[l]); fre(m->Ht[l]); fre(m->dZt4[l]); }
    fre(m->wc); fre(m->wct); fre(m->Xt); fre(m->fpart); fre(m->flpart);
    delete m;
}

hjg_status hjg_mlp_set_stream(hjg_mlp* m, void* stream) {
    if (!m) return HJG_EINVAL;
    m->stream = (cudaStream_t)stream;
    return HJG_OK;
}

int64_t hjg_mlp_num_params(const hjg_mlp* m) { return m ? m->n_params : -1; }

hjg_status hjg_mlp_get_params(hjg_mlp* m, float* out, int on_device) {
    if (!m || !out) return HJG_EINVAL;
    if (cudaMemcpyAsync(out, m->p, m->n_params * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_mlp_set_params(hjg_mlp* m, const float* in, int on_device) {
    if (!m || !in) return HJG_EINVAL;
    if (cudaMemcpyAsync(m->p, in, m->n_params * sizeof(float),
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, m->stream) != cudaSuccess)
        return HJG_ECUDA;
    to_bf16_kernel<<<nblk(m->n_params), 256, 0, m->stream>>>(m->p, m->pb, m->n_params);
    if (cudaGetLastError() != cudaSuccess || refresh_wt(m, m->stream) != cudaSuccess ||
        refresh_canon(m, m->stream) != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess)
        return HJG_ECUDA;
    m->step = 0;
    cudaMemsetAsync(m->m1, 0, m->n_params * sizeof(float), m->stream);
    cudaMemsetAsync(m->m2, 0, m->n_params * sizeof(float), m->stream);
    return HJG_OK;
}

hjg_status hjg_mlp_forward(hjg_mlp* m, const float* x, int64_t ldx, int64_t B, float* out, int64_t ldout) {
    if (!m || B < 0 || ldx < m->n_in || ldout < m->n_out || (B > 0 && (!x || !out))) return HJG_EINVAL;
    if (B == 0) return HJG_OK;
    hjg_status s = mlp_ensure(m, B);
    if (s) return s;
    pack_input_kernel<<<nblk(B * m->in_pad), 256, 0, m->stream>>>(x, ldx, B, m->n_in, m->in_pad, m->iscal,
                                                                  m->X);
    if (cudaGetLastError() != cudaSuccess || mlp_forward(m, B) != cudaSuccess) return HJG_ECUDA;
    unscale_output_kernel<<<nblk(B * m->n_out), 256, 0, m->stream>>>(m->Z[kLayers - 1], m->out_pad, B, m->n_out,
                                                                     m->oscal, out, ldout);
    return cudaGetLastError() == cudaSuccess ? HJG_OK : HJG_ECUDA;
}

hjg_status hjg_mlp_gradients(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy,
                             int64_t B, double* loss_out, float* grad_out) {
    if (!m || B < 1 || !x || !y || ldx < m->n_in || ldy < m->n_out) return HJG_EINVAL;
    hjg_status s = fused_ok(m) ? mlp_fused_step(m, x, ldx, y, ldy, B, 0.0f, loss_out)
                               : mlp_loss_and_grads(m, x, ldx, y, ldy, B, loss_out);
    if (s) return s;
    if (grad_out &&
        (cudaMemcpyAsync(grad_out, m->g, m->n_params * sizeof(float), cudaMemcpyDeviceToHost, m->stream) !=
             cudaSuccess ||
         cudaStreamSynchronize(m->stream) != cudaSuccess))
        return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_mlp_input_grad(hjg_mlp* m, const float* x, int64_t ldx, int64_t B, int j, float* gx,
                              int64_t ldg) {
    if (!m || B < 0 || j < 0 || j >= m->n_out || ldx < m->n_in || ldg < m->n_in || (B > 0 && (!x || !gx)))
        return HJG_EINVAL;
    if (B == 0) return HJG_OK;
    hjg_status s = mlp_ensure(m, B);
    if (s) return s;
    cudaStream_t st = m->stream;
    pack_input_kernel<<<nblk(B * m->in_pad), 256, 0, st>>>(x, ldx, B, m->n_in, m->in_pad, m->iscal, m->X);
    if (cudaGetLastError() != cudaSuccess || mlp_forward(m, B) != cudaSuccess) return HJG_ECUDA;
    unit_output_kernel<<<nblk(B * m->out_pad), 256, 0, st>>>(B, m->out_pad, j, m->dZ);
    for (int l = kLayers - 1; l >= 0; --l) {   // chain rule down to the inputs (no weight gradients)
        const int rows = m->rows[l], cols = m->cols[l];
        GemmArgs gd{};
        gd.A = m->dZ; gd.sam = rows; gd.sak = 1;
        gd.B = m->pbT + m->w_off[l]; gd.sbk = 1; gd.sbn = rows;   // W_l^T [cols][rows]
        gd.M = (int)B; gd.N = cols; gd.K = rows;
        gd.C = m->dH; gd.ldc = cols;
        if (gemm(gd, kEpiStore, 1, st, m->packA, m->packB) != cudaSuccess) return HJG_ECUDA;
        if (l == 0) break;
        const int64_t nh = B * (int64_t)cols;
        silu_backward_kernel<<<nblk(nh), 256, 0, st>>>(m->dH, m->Z[l - 1], nh, m->dZ);
        if (cudaGetLastError() != cudaSuccess) return HJG_ECUDA;
    }
    scale_input_grad_kernel<<<nblk(B * m->n_in), 256, 0, st>>>(m->dH, m->in_pad, B, m->n_in, m->iscal, m->oscal,
                                                               m->out_pad, j, gx, ldg);
    return cudaGetLastError() == cudaSuccess ? HJG_OK : HJG_ECUDA;
}

hjg_status hjg_mlp_fit_scaling(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t B) {
    if (!m || B < 1 || !x || !y || ldx < m->n_in || ldy < m->n_out) return HJG_EINVAL;
    feature_stats_kernel<<<m->n_in, 256, 0, m->stream>>>(x, ldx, B, m->in_pad, 1, m->iscal);
    feature_stats_kernel<<<m->n_out, 256, 0, m->stream>>>(y, ldy, B, m->out_pad, 0, m->oscal);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(m->stream) != cudaSuccess) return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_mlp_get_scaling(hjg_mlp* m, float* out) {
    if (!m || !out) return HJG_EINVAL;
    const size_t ni = (size_t)m->n_in, no = (size_t)m->n_out;
    if (cudaMemcpyAsync(out, m->iscal, ni * sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(out + ni, m->iscal + m->in_pad, ni * sizeof(float), cudaMemcpyDeviceToHost, m->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(out + 2 * ni, m->oscal, no * sizeof(float), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(out + 2 * ni + no, m->oscal + m->out_pad, no * sizeof(float), cudaMemcpyDeviceToHost,
                        m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_mlp_set_scaling(hjg_mlp* m, const float* in) {
    if (!m || !in) return HJG_EINVAL;
    const size_t ni = (size_t)m->n_in, no = (size_t)m->n_out;
    for (size_t i = 0; i < ni; ++i)
        if (!(in[ni + i] > 0.0f) || !std::isfinite(in[i])) return HJG_EINVAL;
    for (size_t i = 0; i < no; ++i)
        if (!(in[2 * ni + no + i] > 0.0f) || !std::isfinite(in[2 * ni + i])) return HJG_EINVAL;
    if (cudaMemcpyAsync(m->iscal, in, ni * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->iscal + m->in_pad, in + ni, ni * sizeof(float), cudaMemcpyHostToDevice, m->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(m->oscal, in + 2 * ni, no * sizeof(float), cudaMemcpyHostToDevice, m->stream) != cudaSuccess ||
        cudaMemcpyAsync(m->oscal + m->out_pad, in + 2 * ni + no, no * sizeof(float), cudaMemcpyHostToDevice,
                        m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_gemm_bf16(const void* A, int64_t sam, int64_t sak, const void* B, int64_t sbk, int64_t sbn,
                         int M, int N, int K, float* C, int64_t ldc, int* timed_out, void* stream) {
    if (M < 0 || N < 0 || K < 0 || (M > 0 && N > 0 && (!C || (K > 0 && (!A || !B)))) || ldc < N)
        return HJG_EINVAL;
    if (M == 0 || N == 0) return HJG_OK;
    GemmArgs g{};
    g.A = (const __nv_bfloat16*)A; g.sam = sam; g.sak = sak;
    g.B = (const __nv_bfloat16*)B; g.sbk = sbk; g.sbn = sbn;
    g.M = M; g.N = N; g.K = K; g.C = C; g.ldc = ldc;
    cudaStream_t st = (cudaStream_t)stream;
    // operands in other layouts are packed into stream-ordered temporaries
    const int64_t na = gemm_scratch_a(g), nb = gemm_scratch_b(g);
    __nv_bfloat16 *sa = nullptr, *sb = nullptr;
    if ((na && cudaMallocAsync((void**)&sa, (size_t)na * sizeof(__nv_bfloat16), st) != cudaSuccess) ||
        (nb && cudaMallocAsync((void**)&sb, (size_t)nb * sizeof(__nv_bfloat16), st) != cudaSuccess)) {
        if (sa) cudaFreeAsync(sa, st);
        return HJG_ENOMEM;
    }
    const cudaError_t ge = gemm(g, kEpiStore, 1, st, sa, sb);
    if (sa) cudaFreeAsync(sa, st);
    if (sb) cudaFreeAsync(sb, st);
    if (ge != cudaSuccess) return HJG_ECUDA;
    if (timed_out) {
        int e = 0;
        if (cudaMemcpyAsync(&e, g_tc_err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return HJG_ECUDA;
        *timed_out = e;
        if (e) return HJG_ETIMEOUT;
    }
    return HJG_OK;
}

hjg_status hjg_selftest_bounded_wait(int arrive, int64_t limit, void* stream) {
    if (limit < 1 || limit > 0xFFFFFFFFll) return HJG_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int* err = nullptr;
    if (cudaMallocAsync((void**)&err, sizeof(int), st) != cudaSuccess) return HJG_ENOMEM;
    int h = 0;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        bounded_wait_kernel<<<1, 1, 0, st>>>(arrive, (uint32_t)limit, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(err, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return HJG_ECUDA;
    return h ? HJG_ETIMEOUT : HJG_OK;
}

hjg_status hjg_mlp_train_step(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy,
                              int64_t B, float lr, double* loss_out) {
    if (!m || B < 1 || !x || !y || ldx < m->n_in || ldy < m->n_out || !(lr > 0)) return HJG_EINVAL;
    if (fused_ok(m)) return mlp_fused_step(m, x, ldx, y, ldy, B, lr, loss_out);
    hjg_status s = mlp_loss_and_grads(m, x, ldx, y, ldy, B, loss_out);
    if (s) return s;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)m->step), c2 = 1.0f - powf(b2, (float)m->step);
    adam_kernel<<<nblk(m->n_params), 256, 0, m->stream>>>(m->p, m->g, m->m1, m->m2, m->pb, m->n_params, lr,
                                                           b1, b2, 1e-8f, c1, c2);
    if (cudaGetLastError() != cudaSuccess || refresh_wt(m, m->stream) != cudaSuccess) return HJG_ECUDA;
    return HJG_OK;
}

hjg_status hjg_mlp_fit(hjg_mlp* m, const float* x, int64_t ldx, const float* y, int64_t ldy, int64_t n,
                       int epochs, int64_t batch, float lr, float lr_final, int standardize, double* hist) {
    if (!m || !x || !y || n < 1 || epochs < 1 || batch < 1 || !(lr > 0) || !(lr_final > 0)) return HJG_EINVAL;
    hjg_status s;
    if (standardize && (s = hjg_mlp_fit_scaling(m, x, ldx, y, ldy, n))) return s;
    const int64_t per = n >= batch ? n / batch : 1;   // minibatches per epoch
    const int64_t steps = (int64_t)epochs * per;
    const double ratio = (double)lr_final / (double)lr;
    int64_t t = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t q = 0; q < per; ++q, ++t) {
            const int64_t b0 = q * batch, b1 = std::min(n, b0 + batch);
            const float rate = (float)((double)lr * std::pow(ratio, (double)t / (double)std::max<int64_t>(1, steps - 1)));
            double loss = 0.0;
            const bool last = q + 1 == per;
            if ((s = hjg_mlp_train_step(m, x + b0 * ldx, ldx, y + b0 * ldy, ldy, b1 - b0, rate,
                                        last && hist ? &loss : nullptr)))
                return s;
            if (last && hist) hist[ep] = loss;
        }
    }
    return HJG_OK;
}

}  // extern "C"
