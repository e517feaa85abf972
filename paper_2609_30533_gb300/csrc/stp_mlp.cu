// Learned proposal network on the 5th-generation tensor cores (sm_103a).
//
// A 4-layer MLP of width 256 (input 32 features padded to 64, output 160
// padded to 256) maps a problem summary to a mixture over the normalised
// arrival time and to 16 space-time waypoints (the learned sampling branch of
// the method's GPU form). Weights are BF16 copies of FP32 master weights; every
// product accumulates in FP32.
//
// GEMM: D[M x N] = A[M x K] . B[N x K]^T, BF16 operands in the canonical
// no-swizzle tile order of the tensor cores (core matrices of 8 rows x 16
// bytes), FP32 accumulation in TMEM. Every BF16 matrix [R][K] (activations,
// their gradients, weights) is stored once, tiled: element (r, k) sits at
//   (((k / BW) * (R / 8) + r / 8) * (BW / 8) + (k % BW) / 8) * 64 + (r % 8) * 8 + k % 8
// with column blocks of BW = 128 (BW = 64 for the 64-wide input): the BW / 8
// core matrices of one 8-row group and one column block are consecutive, then
// the row groups, then the column blocks. So a 128-row x BW stage is one
// contiguous block for a K-major operand (the forward products and the input
// gradients, K = features), and the 64 rows of one column block are one
// contiguous block for an MN-major operand (the weight gradients, K = batch,
// which read the same activations without a transposed copy). Stages move
// into shared memory by bulk asynchronous copies (cp.async.bulk, completion
// on an mbarrier); one elected thread issues tcgen05.mma (kind::f16, M = 128,
// K = 16 per instruction) and tcgen05.commit releases a stage when its MMAs
// have read it; warps read the accumulator back with tcgen05.ld (warp w owns
// TMEM lanes 32 (w % 4) .. + 31 = tile rows) into a fused epilogue.
// Two kernels: the products over K <= 256 (forward layers: bias + ReLU with
// BF16 stores, or bias with FP32 stores for the output layer; input
// gradients: ReLU mask, BF16 stores and bias-gradient partials) run
// persistent with the weight operand resident in shared memory
// (k_gemm_res); the weight gradients (K = batch) run split-K with FP32
// partials (k_gemm_wgrad).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "stp.h"
#include "stp_internal.cuh"

namespace stp {
namespace mlp {

constexpr int kIn = 32, kInP = 64, kHid = 256, kOut = 160, kOutP = 256;
constexpr int kMix = 8, kWp = 16, kWpDim = 8, kTgt = 130;
// Weight-gradient products: eight warps (warp w reads TMEM lane quadrant
// w % 4 and columns [(w / 4) N/2, (w / 4 + 1) N/2) in the epilogue), 64-wide
// K stages through a four-stage pipeline, one CTA per SM.
constexpr int kTileM = 128, kStageK = 64, kThreads = 256, kWStages = 4;
constexpr float kSMin = -7.f, kSMax = 2.f;
// Bias gradients: every 32 batch rows (a warp of an input-gradient epilogue,
// or a CTA of the loss kernel) write the column sums of their rows as one
// partial [256]; Adam adds the partials in a fixed order.

enum Mode { kHidden = 0, kOutput = 1, kBackward = 2, kWGrad = 3 };

// Tiled index (layout above) with column blocks of 1 << lbw (lbw 6 or 7).
__host__ __device__ inline size_t tixb(int r, int k, int R, int lbw) {
    const int cpb = 1 << (lbw - 3);  // core matrices per 8-row group and block
    return ((((size_t)(k >> lbw) * (size_t)(R >> 3) + (size_t)(r >> 3)) * (size_t)cpb +
             (size_t)((k >> 3) & (cpb - 1)))
            << 6) +
           (size_t)((r & 7) << 3) + (size_t)(k & 7);
}
__host__ __device__ constexpr int lbw_of(int K) { return K >= 128 ? 7 : 6; }
constexpr int kActLbw = 7;  // the 256-wide activations and gradients

// ---------------------------------------------------------------------------
// tcgen05 / TMEM helpers (inline PTX).
// ---------------------------------------------------------------------------
// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between core matrices adjacent along K), stride-dimension byte
// offset (between core matrices adjacent along M or N), descriptor version 1,
// no swizzle. A K-major core matrix holds 8 rows (M or N) of 16 bytes of K;
// an MN-major one holds 8 rows of K of 16 bytes of M or N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
// The same with A and B MN-major (bit 15: A, bit 16: B).
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int M, int N) {
    return idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct GemmArgs {
    const __nv_bfloat16* A;  // output gradient, tiled [RA][256] (M = its columns)
    int RA;                  // batch rows (multiple of 128)
    const __nv_bfloat16* B;  // layer input, tiled [RA][N] (N = its columns)
    int KT;                  // 64-row K stages (batch) in total
    int kt_per_split;        // split-K (blockIdx.z): stages [z*kps, min(KT, (z+1)*kps))
    float* out_f;            // FP32 partials [splits][m_valid][ld_f]
    int ld_f;
    int m_valid;             // rows written
    int* err;
};

// BF16 stores of 16 consecutive columns c0..c0+15 (c0 % 16 == 0) of row r
// into a tiled [R][256] activation (two 16-byte stores).
__device__ __forceinline__ void store_row16(__nv_bfloat16* t, int r, int c0, int R, const float (&v)[16]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) b[i] = __float2bfloat16_rn(v[8 * h + i]);
        *reinterpret_cast<uint4*>(t + tixb(r, c0 + 8 * h, R, kActLbw)) = *reinterpret_cast<const uint4*>(b);
    }
}

// Column sums over the 32 lanes of 16 per-lane values by recursive halving:
// at offset o each lane keeps the half of its columns selected by its lane
// bit and adds its partner's copy of them, so lane l ends with the sum of
// column l & 15 over all 32 lanes (16 shuffles instead of 80).
__device__ __forceinline__ float warp_colsum16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 8, n = 8; o >= 1; o >>= 1, n >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            if (i < n) {
                const float send = up ? v[i] : v[i + n];
                const float keep = up ? v[i + n] : v[i];
                v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
            }
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// Weight gradient dW = dT^T . X: M = 128 output features per tile (column
// block of dT), N = the layer's input features, K = the batch rows of split
// blockIdx.z. MT = 1: the CTA computes tile blockIdx.x; MT = 2: both 128-row
// tiles (two accumulators in TMEM), reading each activation stage once. Both
// operands are MN-major: a stage is 64 batch rows, so an A tile is one
// contiguous 16 KB piece of dT's column block and B one piece of 8 row groups
// per column block of X (one MMA of N = BW per tile, block and K step). The
// dynamic shared memory ends with a guard region so that every
// descriptor-addressed read stays inside the allocation.
template <int N, int MT>
__host__ __device__ constexpr int wgrad_stages() {
    return (MT == 2 && N > 64) ? 3 : kWStages;
}
template <int N, int LBWB, int MT>
__host__ __device__ constexpr int wgrad_smem_bytes() {
    return 1024 + wgrad_stages<N, MT>() * (MT * kTileM * kStageK * 2 + N * kStageK * 2) + 21 * 2048 + 256 -
           (1 << LBWB) * kStageK * 2;
}
template <int N, int LBWB, int MT>
__global__ void __launch_bounds__(kThreads, 1) k_gemm_wgrad(GemmArgs g) {
    constexpr int kStages = wgrad_stages<N, MT>();
    constexpr int kBW = 1 << LBWB;                      // B column block
    constexpr int kNB = N / kBW;                        // B blocks (MMAs per K step and tile)
    constexpr uint32_t kATile = kTileM * kStageK * 2;   // 16 KB
    constexpr uint32_t kABytes = MT * kATile;
    constexpr uint32_t kBBlk = kBW * kStageK * 2;
    constexpr uint32_t kBBytes = kNB * kBBlk;
    constexpr uint32_t kTmemCols = MT * N < 32 ? 32 : MT * N;
    constexpr uint32_t kIdesc = idesc_bf16_mn(kTileM, kBW);
    constexpr uint32_t kALbo = 16 * 128, kBLbo = (kBW / 8) * 128;  // one 8-row group of a column block
    static_assert(N % kBW == 0 && (MT == 1 || MT == 2), "whole column blocks");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int fail_sh;

    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sA = smem;
    unsigned char* sB = smem + kStages * kABytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int z = blockIdx.z;
    const int kt0 = z * g.kt_per_split;
    const int kt1 = min(g.KT, kt0 + g.kt_per_split);
    const int nk = kt1 > kt0 ? kt1 - kt0 : 0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fail_sh = 0;
    }
    if (warp == 0) tmem_alloc(&tmem_base_sh, kTmemCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base_sh;

    // Producer + MMA issuer: one thread, prefetch distance kStages - 1.
    if (tid == 0 && nk > 0) {
        const size_t rg = (size_t)(g.RA >> 3);
        int issued = 0, consumed = 0;
        bool ok = true;
        for (int it = 0; it < nk + kStages - 1 && ok; ++it) {
            if (it < nk) {
                const int s = it % kStages;
                if (it >= kStages) ok = mbar_wait(&empty[s], ((it / kStages) - 1) & 1);
                if (!ok) break;
                const size_t kg = (size_t)(kt0 + it) * (kStageK / 8);  // first 8-row group of the stage
                mbar_expect_tx(&full[s], kABytes + kBBytes);
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                    const size_t cb = MT == 2 ? (size_t)mt : (size_t)blockIdx.x;  // column block of dT
                    bulk_g2s(sA + s * kABytes + mt * kATile, g.A + ((cb * rg + kg) * 16) * 64, kATile, &full[s]);
                }
#pragma unroll
                for (int nb = 0; nb < kNB; ++nb)
                    bulk_g2s(sB + s * kBBytes + nb * kBBlk, g.B + (((size_t)nb * rg + kg) * (kBW / 8)) * 64, kBBlk,
                             &full[s]);
                ++issued;
            }
            const int j = it - (kStages - 1);
            if (j >= 0) {
                const int s = j % kStages;
                ok = mbar_wait(&full[s], (j / kStages) & 1);
                if (!ok) break;
                fence_after_sync();
                const uint32_t a0 = smem_u32(sA + s * kABytes), b0 = smem_u32(sB + s * kBBytes);
#pragma unroll
                for (int ks = 0; ks < kStageK / 16; ++ks) {
                    // K step of 16 batch rows = two 8-row groups.
#pragma unroll
                    for (int mt = 0; mt < MT; ++mt) {
                        const uint64_t da = smem_desc(a0 + mt * kATile + ks * 2 * kALbo, kALbo, 128);
#pragma unroll
                        for (int nb = 0; nb < kNB; ++nb) {
                            const uint64_t db = smem_desc(b0 + nb * kBBlk + ks * 2 * kBLbo, kBLbo, 128);
                            mma_bf16(tmem + (uint32_t)(mt * N + nb * kBW), da, db, kIdesc,
                                     (j > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                }
                mma_commit(&empty[s]);
                ++consumed;
            }
        }
        // Always close with a commit so that `done` tracks every issued MMA.
        mma_commit(&done);
        if (!ok) {
            fail_sh = 1;
            if (g.err) atomicOr(g.err, kErrTimeout);
            // Wait (bounded) for copies still in flight before the CTA exits.
            for (int j = consumed; j < issued; ++j) mbar_wait(&full[j % kStages], (j / kStages) & 1);
        }
    }
    __syncthreads();
    bool have = nk > 0;
    if (have) {
        if (!mbar_wait(&done, 0)) {
            if (lane == 0 && g.err) atomicOr(g.err, kErrTimeout);
            fail_sh = 1;
        }
    }
    fence_after_sync();
    __syncthreads();
    if (fail_sh) have = false;

    // Epilogue: thread (warp, lane) owns row 32 (warp % 4) + lane of each
    // tile and half of the columns; FP32 partial rows of split z.
    const int quad = warp & 3;
    const int cb = (warp >> 2) * (N / 2), ce = cb + N / 2;
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
        const int r = (MT == 2 ? mt : (int)blockIdx.x) * kTileM + 32 * quad + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(mt * N);
#pragma unroll 1
        for (int c0 = cb; c0 < ce; c0 += 16) {
            float v[16];
            if (have) tmem_ld16(trow + (uint32_t)c0, v);
            else {
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
            }
            if (r < g.m_valid) {
                float4* o = reinterpret_cast<float4*>(g.out_f + ((size_t)z * g.m_valid + r) * g.ld_f + c0);
#pragma unroll
                for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Products with K <= 256 (every forward layer and every input gradient) as a
// persistent kernel with the weight operand resident in shared memory.
//
// Work unit = (128-row tile t, column half h): columns [h NU, (h + 1) NU) of
// the output. The grid is even and CTA c takes units c, c + grid, ..., so it
// always computes the same half h = c & 1 and loads that half of the weight
// operand (NU x K BF16, at most 64 KB) into shared memory once; only the A
// stages (128 rows x 64 K, 16 KB) stream through a ring of kRing stages.
// The TMEM accumulator is double-buffered (two 128-column slots), so the
// epilogue of one unit overlaps the copies and MMAs of the next.
// Warps 0-7 run the epilogue (warp w reads TMEM lane quadrant w % 4 = tile
// rows 32 (w % 4) .. + 31, and every other 16-column chunk starting at w / 4),
// warp 8 lane 0 issues the bulk copies, warp 9 lane 0 the MMAs. Every wait
// is bounded; a role whose wait runs out sets the error flag and stops, and
// the copy issuer waits (bounded) for its copies in flight before the CTA
// frees its TMEM and exits.
// ---------------------------------------------------------------------------
constexpr int kRingBytes = 128 * 1024, kResThreads = 320, kEpiWarps = 8;
constexpr int kOutPad = 20;  // FP32 staging row (16 + 4: no bank conflicts)

// K stage = one column block of A (BW = 1 << lbw wide): 16 or 32 KB.
__host__ __device__ constexpr int res_smem_bytes(int nu, int kb, int lbw, int mode) {
    return 1024 + kb * nu * (1 << lbw) * 2 + kRingBytes + (mode == kOutput ? kEpiWarps * 32 * kOutPad * 4 : 0);
}

// Programmatic dependent launch: let the next kernel in the stream start its
// CTAs (and their prologue) as this kernel's CTAs finish, and wait for the
// previous kernel's completion and memory before touching its outputs. Both
// are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

struct ResArgs {
    const __nv_bfloat16* A;    // tiled [RA][KB * BW]
    int RA;                    // rows of A (multiple of 128)
    const __nv_bfloat16* B;    // tiled [NB][KB * BW], output column n = row n of B
    int NB;                    // rows of B's tiled layout
    int units;                 // 2 * RA / 128
    const float* bias;         // [2 NU] (forward modes)
    const __nv_bfloat16* act;  // kBackward: forward activation, tiled [RA][256]
    __nv_bfloat16* out_t;      // tiled [RA][256]
    float* out_f;              // kOutput: FP32 [RA][ld_f]; kBackward: bias-gradient partials [RA / 32][256]
    int ld_f;
    int* err;
};

template <int NU, int KB, int LBW, int MODE>
__global__ void __launch_bounds__(kResThreads, 1) k_gemm_res(ResArgs g) {
    static_assert(NU % 16 == 0 && NU <= 128 && KB >= 1 && KB <= 2 && (LBW == 6 || LBW == 7), "unit shape");
    constexpr int kBW = 1 << LBW;
    constexpr uint32_t kAStage = kTileM * kBW * 2;  // one column block of a 128-row tile
    constexpr int kRing = kRingBytes / (int)kAStage;
    constexpr uint32_t kBBytes = NU * kBW * 2;      // one column block of the resident half
    constexpr uint32_t kSbo = (kBW / 8) * 128;      // between 8-row groups
    constexpr uint32_t kIdesc = idesc_bf16(kTileM, NU);
    constexpr int kChunks = NU / 16;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kRing], empty[kRing], bfull, tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ float sbias[NU];

    unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* sB = smem;
    unsigned char* sA = smem + KB * kBBytes;
    float* sOut = reinterpret_cast<float*>(sA + kRing * kAStage);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int h = blockIdx.x & 1;

    if (tid == 0) {
        for (int s = 0; s < kRing; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&bfull, 1);
        mbar_init(&done, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiWarps);
        }
        abort_sh = 0;
    }
    if (MODE == kHidden || MODE == kOutput)
        for (int i = tid; i < NU; i += kResThreads) sbias[i] = g.bias[h * NU + i];
    if (warp == 0) tmem_alloc(&tmem_base_sh, 256);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base_sh;
    auto fail = [&]() {
        abort_sh = 1;
        if (g.err) atomicOr(g.err, kErrTimeout);
    };
    if (tid == 0) pdl_launch_dependents();

    if (warp == kEpiWarps) {
        // Copy issuer.
        if (lane == 0) {
            mbar_expect_tx(&bfull, KB * kBBytes);
            for (int kb = 0; kb < KB; ++kb)
                bulk_g2s(sB + kb * kBBytes,
                         g.B + (((size_t)kb * (g.NB >> 3) + (size_t)h * (NU >> 3)) * (kBW / 8)) * 64, kBBytes, &bfull);
            // The weights are no kernel's output within a pass; the A
            // operand is the previous kernel's.
            pdl_wait();
            const size_t rgA = (size_t)(g.RA >> 3);
            int it = 0;
            for (int u = blockIdx.x; u < g.units && !abort_sh; u += gridDim.x) {
                const int t = u >> 1;
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % kRing;
                    if (it >= kRing && !mbar_wait(&empty[s], ((it / kRing) - 1) & 1)) {
                        fail();
                        break;
                    }
                    mbar_expect_tx(&full[s], kAStage);
                    bulk_g2s(sA + s * kAStage,
                             g.A + (((size_t)kb * rgA + (size_t)t * (kTileM >> 3)) * (kBW / 8)) * 64, kAStage,
                             &full[s]);
                }
            }
            // Drain: the last copy issued into each stage (and the weight
            // copies) have landed before the CTA may exit.
            for (int s = 0; s < kRing && s < it; ++s) {
                const int j = s + ((it - 1 - s) / kRing) * kRing;  // last issue index on stage s
                mbar_wait(&full[s], (j / kRing) & 1);
            }
            mbar_wait(&bfull, 0);
        }
    } else if (warp == kEpiWarps + 1) {
        // MMA issuer.
        if (lane == 0) {
            pdl_wait();
            bool ok = mbar_wait(&bfull, 0);
            if (!ok) fail();
            int it = 0, i = 0;
            for (int u = blockIdx.x; ok && u < g.units && !abort_sh; u += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[b], ((i >> 1) - 1) & 1)) {
                    fail();
                    break;
                }
                fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * 128);
                for (int kb = 0; kb < KB; ++kb, ++it) {
                    const int s = it % kRing;
                    if (!mbar_wait(&full[s], (it / kRing) & 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t a0 = smem_u32(sA + s * kAStage), b0 = smem_u32(sB + kb * kBBytes);
#pragma unroll
                    for (int ks = 0; ks < kBW / 16; ++ks)
                        mma_bf16(d, smem_desc(a0 + ks * 256, 128, kSbo), smem_desc(b0 + ks * 256, 128, kSbo), kIdesc,
                                 (kb > 0 || ks > 0) ? 1u : 0u);
                    mma_commit(&empty[s]);
                }
                mma_commit(&tfull[b]);
            }
            // Every MMA has completed before the TMEM is freed.
            mma_commit(&done);
            if (!mbar_wait(&done, 0)) fail();
        }
    } else {
        // Epilogue warps. Warp (quad, hw) takes chunks hw, hw + 2, ... of 16
        // columns. The input-gradient mode's ReLU mask (the forward activation
        // at the same rows and columns) of the next unit is loaded into
        // registers while the current unit's stores drain.
        const int quad = warp & 3, hw = warp >> 2;
        constexpr int kWChunks = (kChunks + 1) / 2;
        uint4 pa[MODE == kBackward ? kWChunks : 1][2];
        auto load_mask = [&](int uu) {
            if constexpr (MODE == kBackward) {
                const int rr = (uu >> 1) * kTileM + 32 * quad + lane;
#pragma unroll
                for (int ci = 0; ci < kWChunks; ++ci) {
                    const int c = hw + 2 * ci;
                    if (c < kChunks) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh)
                            pa[ci][hh] = *reinterpret_cast<const uint4*>(
                                g.act + tixb(rr, h * NU + 16 * c + 8 * hh, g.RA, kActLbw));
                    }
                }
            }
        };
        pdl_wait();
        if (blockIdx.x < g.units) load_mask(blockIdx.x);
        int i = 0;
        for (int u = blockIdx.x; u < g.units; u += gridDim.x, ++i) {
            const int b = i & 1, t = u >> 1;
            if (abort_sh || !mbar_wait(&tfull[b], (i >> 1) & 1)) {
                if (lane == 0) fail();
                break;
            }
            __syncwarp();
            fence_after_sync();
            const int r0 = t * kTileM + 32 * quad;
            const int r = r0 + lane;
            const uint32_t trow = tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(b * 128);
#pragma unroll
            for (int ci = 0; ci < kWChunks; ++ci) {
                const int c = hw + 2 * ci;
                if (c >= kChunks) break;
                const int cl = 16 * c, cg = h * NU + cl;  // local / global column
                float v[16];
                tmem_ld16(trow + (uint32_t)cl, v);
                if constexpr (MODE == kHidden) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) v[k] = fmaxf(v[k] + sbias[cl + k], 0.f);
                    store_row16(g.out_t, r, cg, g.RA, v);
                } else if constexpr (MODE == kOutput) {
                    float* so = sOut + warp * 32 * kOutPad;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4*>(so + lane * kOutPad + 4 * q) =
                            make_float4(v[4 * q] + sbias[cl + 4 * q], v[4 * q + 1] + sbias[cl + 4 * q + 1],
                                        v[4 * q + 2] + sbias[cl + 4 * q + 2], v[4 * q + 3] + sbias[cl + 4 * q + 3]);
                    __syncwarp();
                    // Four rounds of eight rows x 64 contiguous bytes.
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int rr = 8 * q + (lane >> 2), cc = 4 * (lane & 3);
                        *reinterpret_cast<float4*>(g.out_f + (size_t)(r0 + rr) * g.ld_f + cg + cc) =
                            *reinterpret_cast<const float4*>(so + rr * kOutPad + cc);
                    }
                    __syncwarp();
                } else {  // kBackward
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        __align__(16) __nv_bfloat16 a[8];
                        *reinterpret_cast<uint4*>(a) = pa[ci][hh];
#pragma unroll
                        for (int k = 0; k < 8; ++k)
                            if (!(__bfloat162float(a[k]) > 0.f)) v[8 * hh + k] = 0.f;
                    }
                    store_row16(g.out_t, r, cg, g.RA, v);
                    // Bias-gradient partial of these 32 rows: row r0 / 32 of
                    // the partials, each element written by one warp.
                    const float cs = warp_colsum16(v);
                    if (lane < 16) g.out_f[(size_t)(r0 >> 5) * 256 + cg + lane] = cs;
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[b]);
            if (u + (int)gridDim.x < g.units) load_mask(u + gridDim.x);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// Elementwise kernels.
// ---------------------------------------------------------------------------
// FP32 features [B][32] -> BF16 tiled [Bp][64] (zero padded). Thread i
// writes the 16-byte piece i of the tiled buffer: row 8 (i / 64) + i % 8,
// columns 8 ((i / 8) % 8) .. + 7, so consecutive threads store consecutive
// pieces.
__global__ void k_pack_input(const float* __restrict__ X, int B, int Bp, __nv_bfloat16* xt) {
    static_assert(lbw_of(kInP) == 6 && kInP == 64 && kIn % 8 == 0, "one 64-wide column block");
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Bp * (kInP / 8)) return;
    const int r = 8 * (i >> 6) + (i & 7), c = (i >> 3) & 7;
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < B && 8 * c < kIn) {
        const float4* src = reinterpret_cast<const float4*>(X + (size_t)r * kIn + 8 * c);
        const float4 u0 = __ldg(src), u1 = __ldg(src + 1);
        v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
        v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
    }
    __align__(16) __nv_bfloat16 h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) h[q] = __float2bfloat16_rn(v[q]);
    *reinterpret_cast<uint4*>(xt + (size_t)i * 8) = *reinterpret_cast<const uint4*>(h);
}

// Per-sample loss (mixture NLL of tau + masked waypoint MSE) and dL/dy / B.
// A CTA takes 32 consecutive rows (one bias-gradient partial): their network
// outputs and targets are staged in shared memory by coalesced 16-byte loads
// (the 32 target rows are one contiguous block), four threads share a row
// (mixture components p and p + 4, waypoint elements p, p + 4, ...; the row's
// reductions are shuffles within the four lanes), the gradient overwrites
// the staged outputs, and the CTA then writes its BF16 tiles with consecutive
// threads on consecutive 16-byte pieces, the 256 column sums of its rows, and
// the row losses.
constexpr int kLossRows = 32, kLossThreads = 128;
constexpr int kLossYS = kOut + 4;                 // staged row stride (floats)
constexpr int kOutUsed = 3 * kMix + kWp * kWpDim;  // 152 network outputs in use
static_assert(kLossThreads == 4 * kLossRows, "four threads per row");
static_assert(kMix == 8 && kWpDim == 8 && (kWp * kWpDim) % 4 == 0, "components and elements split over four lanes");
static_assert((kLossRows * kTgt) % 4 == 0 && (kLossYS * 4) % 16 == 0, "16-byte staging");

__global__ void __launch_bounds__(kLossThreads) k_loss(const float* __restrict__ Y, const float* __restrict__ T,
                                                       int B, float* bpart, __nv_bfloat16* dyt, int Bp,
                                                       float* loss) {
    __shared__ __align__(16) float sy[kLossRows * kLossYS];
    __shared__ __align__(16) float st[kLossRows * kTgt];
    const int tid = threadIdx.x;
    const int n0 = blockIdx.x * kLossRows;
    const int nrow = max(0, min(kLossRows, B - n0));  // rows of this CTA inside the batch
    constexpr int kYv = kOut / 4;                     // float4 per output row
    constexpr int kTv = kLossRows * kTgt / 4;         // float4 of a full target block
    if (nrow == kLossRows) {
        // Row n0 of the targets starts at byte 520 n0, a multiple of 16 (n0 % 32 == 0).
        float4 yv[kLossRows * kYv / kLossThreads];
        float4 tv[(kTv + kLossThreads - 1) / kLossThreads];
        const float4* t4 = reinterpret_cast<const float4*>(T + (size_t)n0 * kTgt);
#pragma unroll
        for (int q = 0; q < kLossRows * kYv / kLossThreads; ++q) {
            const int i = tid + q * kLossThreads, r = i / kYv, c = i % kYv;
            yv[q] = __ldg(reinterpret_cast<const float4*>(Y + (size_t)(n0 + r) * kOutP) + c);
        }
#pragma unroll
        for (int q = 0; q < (kTv + kLossThreads - 1) / kLossThreads; ++q) {
            const int i = tid + q * kLossThreads;
            if (i < kTv) tv[q] = __ldg(t4 + i);
        }
#pragma unroll
        for (int q = 0; q < kLossRows * kYv / kLossThreads; ++q) {
            const int i = tid + q * kLossThreads, r = i / kYv, c = i % kYv;
            *reinterpret_cast<float4*>(sy + r * kLossYS + 4 * c) = yv[q];
        }
#pragma unroll
        for (int q = 0; q < (kTv + kLossThreads - 1) / kLossThreads; ++q) {
            const int i = tid + q * kLossThreads;
            if (i < kTv) reinterpret_cast<float4*>(st)[i] = tv[q];
        }
    } else if (nrow > 0) {  // the batch's last, partial CTA
        for (int i = tid; i < nrow * kYv; i += kLossThreads) {
            const int r = i / kYv, c = i % kYv;
            *reinterpret_cast<float4*>(sy + r * kLossYS + 4 * c) =
                __ldg(reinterpret_cast<const float4*>(Y + (size_t)(n0 + r) * kOutP) + c);
        }
        for (int i = tid; i < nrow * kTgt; i += kLossThreads) st[i] = __ldg(T + (size_t)n0 * kTgt + i);
    }
    __syncthreads();

    // Every lane runs the row arithmetic (the shuffles need the whole warp);
    // rows past the batch read zeros and write nothing.
    const int r = tid >> 2, p = tid & 3;
    const bool valid = r < nrow;
    float* y = sy + r * kLossYS;
    const float* t = st + r * kTgt;
    const float invB = 1.f / (float)B;
    const float tau = valid ? t[0] : 0.f;
    const int dof = valid ? (int)t[kTgt - 1] : 0;
    // Mixture over tau: this thread's components p and p + 4.
    float a[2], l[2], z[2], sig[2], sr[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int k = p + 4 * h;
        a[h] = valid ? y[k] : 0.f;
        sr[h] = valid ? y[2 * kMix + k] : 0.f;
        const float mu = valid ? y[kMix + k] : 0.f;
        const float s = fminf(fmaxf(sr[h], kSMin), kSMax);
        sig[h] = expf(s);
        z[h] = (tau - mu) / sig[h];
        l[h] = -0.5f * z[h] * z[h] - s - 0.91893853320467274f;  // log N(tau; mu, sig)
    }
    float amax = fmaxf(a[0], a[1]);
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 1));
    amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, 2));
    float asum = expf(a[0] - amax) + expf(a[1] - amax);
    asum += __shfl_xor_sync(0xffffffffu, asum, 1);
    asum += __shfl_xor_sync(0xffffffffu, asum, 2);
    const float lse_a = amax + logf(asum);
#pragma unroll
    for (int h = 0; h < 2; ++h) l[h] += a[h] - lse_a;
    float lmax = fmaxf(l[0], l[1]);
    lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, 1));
    lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, 2));
    float lsum = expf(l[0] - lmax) + expf(l[1] - lmax);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 1);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, 2);
    const float lse_l = lmax + logf(lsum);
    // Waypoints: element e = 4 m + p (waypoint e / 8, coordinate e % 8);
    // the coordinates in use are the arm's dof joints and the time.
    const float cnt = (float)(kWp * (dof + 1));
    const float gscale = 2.f * invB / cnt;  // d(mse / cnt) / B per unit error
    float mse = 0.f;
    if (valid) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = p + 4 * h;
            const float gam = expf(l[h] - lse_l);
            const float pi = expf(a[h] - lse_a);
            y[k] = (pi - gam) * invB;
            y[kMix + k] = -gam * z[h] / sig[h] * invB;
            y[2 * kMix + k] = (sr[h] >= kSMin && sr[h] <= kSMax) ? gam * (1.f - z[h] * z[h]) * invB : 0.f;
        }
#pragma unroll 8
        for (int m = 0; m < kWp * kWpDim / 4; ++m) {
            const int e = 4 * m + p, j = e & (kWpDim - 1);
            const int o = 3 * kMix + e;
            float g = 0.f;
            if (j < dof || j == kWpDim - 1) {
                const float d = y[o] - t[1 + e];
                mse += d * d;
                g = d * gscale;
            }
            y[o] = g;
        }
    }
    mse += __shfl_xor_sync(0xffffffffu, mse, 1);
    mse += __shfl_xor_sync(0xffffffffu, mse, 2);
    if (valid && p == 0) loss[n0 + r] = -lse_l + mse / cnt;
    __syncthreads();

    // dL/dy as BF16 tiles: piece c = (s, core matrix cm, row i) holds columns
    // 128 (s & 1) + 8 cm .. + 7 of row 8 (s >> 1) + i; the 128 pieces of one
    // (s, cm) range are 2 KB of contiguous memory.
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        const int c = tid + s * kLossThreads;
        const int i = c & 7, cm = (c >> 3) & 15;
        const int rr = 8 * (s >> 1) + i, k0 = 128 * (s & 1) + 8 * cm;
        float v[8];
        if (rr < nrow && k0 < kOutUsed) {
            const float4 u0 = *reinterpret_cast<const float4*>(sy + rr * kLossYS + k0);
            const float4 u1 = *reinterpret_cast<const float4*>(sy + rr * kLossYS + k0 + 4);
            v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
            v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.f;
        }
        __align__(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = __float2bfloat16_rn(v[q]);
        *reinterpret_cast<uint4*>(dyt + tixb(n0 + rr, k0, Bp, kActLbw)) = *reinterpret_cast<const uint4*>(b);
    }
    // Bias-gradient partial of these 32 rows (row n0 / 32 of the partials,
    // as the input-gradient products write theirs; rows added in order, no
    // atomics, so the sums are the same on every run).
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int col = tid + h * kLossThreads;
        float sum = 0.f;
        if (col < kOutUsed)
            for (int rr = 0; rr < nrow; ++rr) sum += sy[rr * kLossYS + col];
        bpart[(size_t)blockIdx.x * kOutP + col] = sum;
    }
}

struct AdamArgs {
    float* w;                 // FP32 master [rows][cols] row-major (or bias [rows])
    float* m;
    float* v;
    const float* gpart;       // gradient partials [nparts][rows][cols]
    int nparts;
    int rows, cols;
    int rows_used;            // rows beyond stay zero
    __nv_bfloat16* wt;        // tiled [rows][cols] (weights only)
    __nv_bfloat16* wtT;       // tiled [cols][rows] (weights only)
    float* gout;              // optional: summed gradient [rows][cols]
    float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
    int update;               // 0: only sum gradients (and refresh BF16 copies)
};

// Element i of a parameter tensor: store the summed gradient (optional),
// take the Adam step, refresh the BF16 operand copies.
__device__ __forceinline__ void adam_apply(const AdamArgs& a, int i, float gsum) {
    const int r = i / a.cols, c = i % a.cols;
    if (r >= a.rows_used) gsum = 0.f;
    if (a.gout) a.gout[i] = gsum;
    float w = a.w[i];
    if (a.update && r < a.rows_used) {
        const float m = a.b1 * a.m[i] + (1.f - a.b1) * gsum;
        const float v = a.b2 * a.v[i] + (1.f - a.b2) * gsum * gsum;
        a.m[i] = m;
        a.v[i] = v;
        w -= a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
        a.w[i] = w;
    }
    if (a.wt) {
        const __nv_bfloat16 b = __float2bfloat16_rn(w);
        a.wt[tixb(r, c, a.rows, lbw_of(a.cols))] = b;
        a.wtT[tixb(c, r, a.cols, lbw_of(a.rows))] = b;
    }
}

// Every parameter tensor of one Adam step in one launch. Blocks
// [0, wblk[4]) take 1,024 weight elements each: a thread sums the split-K
// partials of four consecutive elements in split order, eight 16-byte loads in
// flight. The remaining blocks take 16 bias elements each: 64 row lanes sum
// the per-32-row partials (lane k: rows k, k + 64, ...) and the lanes' sums
// are added in lane order. Fixed orders throughout, so every run gives the
// same sums.
struct AdamAll {
    AdamArgs t[8];  // weights of layer l at 2 l, its bias at 2 l + 1
    int wblk[5];    // weight blocks before layer l
    int bblk[5];    // bias blocks before layer l
};
constexpr int kAdamThreads = 256, kAdamWElems = 4 * kAdamThreads, kAdamBElems = 16, kAdamLanes = 64;
static_assert(kAdamLanes * (kAdamBElems / 4) == kAdamThreads, "bias block shape");

__global__ void __launch_bounds__(kAdamThreads) k_adam_all(const __grid_constant__ AdamAll A) {
    __shared__ float part[kAdamLanes][kAdamBElems + 1];
    int b = blockIdx.x;
    if (b < A.wblk[4]) {
        int l = 0;
        while (l < 3 && b >= A.wblk[l + 1]) ++l;
        const AdamArgs& a = A.t[2 * l];
        const int n = a.rows * a.cols;
        const int i0 = (b - A.wblk[l]) * kAdamWElems + 4 * (int)threadIdx.x;
        if (i0 >= n) return;
        float g[4] = {0.f, 0.f, 0.f, 0.f};
        if (a.gpart) {
            const float4* src = reinterpret_cast<const float4*>(a.gpart + i0);
            const size_t stride = (size_t)n / 4;
            int p = 0;
            for (; p + 8 <= a.nparts; p += 8) {
                float4 v[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) v[q] = src[(size_t)(p + q) * stride];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    g[0] += v[q].x;
                    g[1] += v[q].y;
                    g[2] += v[q].z;
                    g[3] += v[q].w;
                }
            }
            for (; p < a.nparts; ++p) {
                const float4 v = src[(size_t)p * stride];
                g[0] += v.x;
                g[1] += v.y;
                g[2] += v.z;
                g[3] += v.w;
            }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) adam_apply(a, i0 + q, g[q]);
        return;
    }
    b -= A.wblk[4];
    int l = 0;
    while (l < 3 && b >= A.bblk[l + 1]) ++l;
    const AdamArgs& a = A.t[2 * l + 1];
    const int n = a.rows;  // a bias: rows x 1
    const int c0 = (b - A.bblk[l]) * kAdamBElems;
    const int quad = threadIdx.x & 3, lane = threadIdx.x >> 2;
    float s[4] = {0.f, 0.f, 0.f, 0.f};
    if (a.gpart && c0 + 4 * quad < n) {
        const float* src = a.gpart + c0 + 4 * quad;
#pragma unroll 8
        for (int p = lane; p < a.nparts; p += kAdamLanes) {
            const float4 v = *reinterpret_cast<const float4*>(src + (size_t)p * n);
            s[0] += v.x;
            s[1] += v.y;
            s[2] += v.z;
            s[3] += v.w;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) part[lane][4 * quad + q] = s[q];
    __syncthreads();
    const int e = threadIdx.x;
    if (e < kAdamBElems && c0 + e < n) {
        float g = 0.f;
        for (int k = 0; k < kAdamLanes; ++k) g += part[k][e];
        adam_apply(a, c0 + e, g);
    }
}

// FP32 [Bp][256] -> user [B][160].
__global__ void k_unpack_out(const float* __restrict__ Y, int B, float* out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * kOut) return;
    out[i] = Y[(size_t)(i / kOut) * kOutP + i % kOut];
}

}  // namespace mlp
}  // namespace stp

// ---------------------------------------------------------------------------
// Host side and C ABI.
// ---------------------------------------------------------------------------
using namespace stp;
using namespace stp::mlp;

namespace {
// Logical parameter layout (W1 [256][32], b1, W2 [256][256], b2, W3, b3,
// W4 [160][256], b4 [160]) against the padded device tensors.
struct Layer {
    int out, in, out_used, in_used;  // padded / logical
};
constexpr Layer kLayers[4] = {{kHid, kInP, kHid, kIn}, {kHid, kHid, kHid, kHid}, {kHid, kHid, kHid, kHid},
                              {kOutP, kHid, kOut, kHid}};
}  // namespace

struct stp_mlp {
    int max_batch = 0, Bp_max = 0;
    cudaStream_t stream = nullptr;
    char* arena = nullptr;
    size_t arena_bytes = 0;
    // parameters
    float* w[4]{};
    float* b[4]{};
    float *mw[4]{}, *vw[4]{}, *mb[4]{}, *vb[4]{};
    __nv_bfloat16 *wt[4]{}, *wtT[4]{};
    // activations (tiled BF16 in both layouts), FP32 buffers
    __nv_bfloat16* xt = nullptr;
    __nv_bfloat16* ht[3]{};
    __nv_bfloat16* dt[4]{};  // gradient wrt layer outputs (dt[3] = dY)
    float* y = nullptr;       // [Bp][256]
    float* wpart = nullptr;   // weight-gradient partials
    float* bpart = nullptr;   // bias-gradient partials [4][Bp/32][256]
    float* gsum = nullptr;    // summed gradients (gradients API)
    float* loss = nullptr;    // [Bp]
    float* X = nullptr;       // staged inputs [max_batch][32]
    float* T = nullptr;       // staged targets [max_batch][130]
    float* Yout = nullptr;    // [max_batch][160]
    int* err = nullptr;
    int nsm = 0;              // SMs of the device (persistent product grid)
    cudaStream_t side = nullptr;          // weight gradients beside the input gradients
    cudaEvent_t fork = nullptr, join = nullptr;
    int step = 0;
    bool profiling = false;
    // Profiling intervals: 0 forward chain, 1 backward pass, 2 whole training
    // step (event pairs 2i, 2i + 1), read once the stream has been synchronised.
    cudaEvent_t ev[6]{};
    bool ev_pending[3]{};
    double ev_flops[3]{}, ev_bytes[3]{};
    double gemm_ms = 0, gemm_flops = 0, gemm_bytes = 0;
    double step_ms = 0;
    int steps = 0;
    std::string last_error;
};

namespace {
thread_local std::string g_mlp_err;

stp_status fail(stp_mlp* m, stp_status st, const std::string& msg) {
    if (m) m->last_error = msg;
    g_mlp_err = msg;
    return st;
}
#define MLP_CUDA(m, call)                                                               \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess) return fail((m), STP_ERR_CUDA, cudaGetErrorString(e_)); \
    } while (0)

// Split-K of the weight-gradient products: at most kSplitMax splits (the
// partial buffers), at least four K stages each.
constexpr int kSplitMax = 80;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

template <int N, int LBWB, int MT>
cudaError_t launch_wgrad(const GemmArgs& g, int splits, cudaStream_t st) {
    constexpr int smem = wgrad_smem_bytes<N, LBWB, MT>();
    static SmemAttr attr;
    cudaError_t e = ensure_smem((const void*)k_gemm_wgrad<N, LBWB, MT>, attr, smem);
    if (e != cudaSuccess) return e;
    k_gemm_wgrad<N, LBWB, MT><<<dim3(MT == 2 ? 1 : kOutP / kTileM, 1, splits), kThreads, smem, st>>>(g);
    return cudaGetLastError();
}

// max_ctas: the SMs this launch may take (the rest run a concurrent product);
// pdl: launch as a programmatic dependent of the previous kernel in st.
template <int NU, int KB, int LBW, int MODE>
cudaError_t launch_res(const ResArgs& g, int max_ctas, cudaStream_t st, bool pdl = false) {
    constexpr int smem = res_smem_bytes(NU, KB, LBW, MODE);
    static SmemAttr attr;
    cudaError_t e = ensure_smem((const void*)k_gemm_res<NU, KB, LBW, MODE>, attr, smem);
    if (e != cudaSuccess) return e;
    // Even grid (a CTA keeps one column half), at most one CTA per SM.
    const int grid = std::max(2, std::min(g.units, max_ctas & ~1));
    if (!pdl) {
        k_gemm_res<NU, KB, LBW, MODE><<<grid, kResThreads, smem, st>>>(g);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kResThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute la[1];
    la[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    la[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gemm_res<NU, KB, LBW, MODE>, g);
}

// Bias-gradient partials per layer: one row per 32 batch rows (written by the
// input-gradient products, and for the last layer by the loss kernel).
size_t bpart_stride(int Bp_max) { return (size_t)(Bp_max / 32) * kOutP; }

// Algorithmic HBM bytes of one product of a training step at batch B over the
// layer's logical shape (in x out, no padding): every operand read once,
// every output written once in one layout (BF16 activations and input
// gradients, FP32 network outputs and weight gradients); the input-gradient
// product also reads the forward activation for the ReLU mask. The second
// (transposed) BF16 copy of each activation, the padding and the split-K
// partials are this design's choices and are not counted.
double alg_bytes(int B, int in, int out, int mode) {
    const double b = B, i = in, o = out;
    if (mode == kHidden) return 2 * b * i + 2 * i * o + 2 * b * o;
    if (mode == kOutput) return 2 * b * i + 2 * i * o + 4 * b * o;
    if (mode == kWGrad) return 2 * b * o + 2 * b * i + 4 * i * o;
    return 2 * b * o + 2 * i * o + 2 * b * i + 2 * b * i;  // kBackward
}

// Event interval `slot` on the main stream (no host synchronisation inside
// a call: the intervals are read by collect_profile after the stream sync).
void interval_start(stp_mlp* m, int slot) {
    if (m->profiling) cudaEventRecord(m->ev[2 * slot], m->stream);
}
void interval_stop(stp_mlp* m, int slot, double flops, double bytes) {
    if (!m->profiling) return;
    cudaEventRecord(m->ev[2 * slot + 1], m->stream);
    m->ev_pending[slot] = true;
    m->ev_flops[slot] = flops;
    m->ev_bytes[slot] = bytes;
}
void collect_profile(stp_mlp* m) {
    for (int slot = 0; slot < 3; ++slot) {
        if (!m->ev_pending[slot]) continue;
        m->ev_pending[slot] = false;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m->ev[2 * slot], m->ev[2 * slot + 1]) != cudaSuccess) continue;
        if (slot == 2) {
            m->step_ms += ms;
            ++m->steps;
        } else {
            m->gemm_ms += ms;
            m->gemm_flops += m->ev_flops[slot];
            m->gemm_bytes += m->ev_bytes[slot];
        }
    }
}

stp_status forward_impl(stp_mlp* m, int B) {
    const int Bp = (B + kTileM - 1) / kTileM * kTileM;
    const int mt = Bp / kTileM;
    cudaStream_t st = m->stream;
    {
        const int n = Bp * (kInP / 8);
        k_pack_input<<<(n + 255) / 256, 256, 0, st>>>(m->X, B, Bp, m->xt);
        MLP_CUDA(m, cudaGetLastError());
    }
    // The four products are timed as one interval: each is launched as a
    // programmatic dependent of the previous kernel, so its prologue (barriers,
    // TMEM, the resident weights) overlaps the previous product's tail.
    double chain_flops = 0.0, chain_bytes = 0.0;
    for (int l = 0; l < 4; ++l) {
        const Layer& L = kLayers[l];
        chain_flops += 2.0 * B * L.in_used * L.out_used;
        chain_bytes += alg_bytes(B, L.in_used, L.out_used, l < 3 ? kHidden : kOutput);
    }
    interval_start(m, 0);
    const __nv_bfloat16* in = m->xt;
    for (int l = 0; l < 4; ++l) {
        const Layer& L = kLayers[l];
        ResArgs g{};
        g.A = in;
        g.RA = Bp;
        g.B = m->wt[l];
        g.NB = L.out;
        g.units = 2 * mt;
        g.bias = m->b[l];
        g.err = m->err;
        if (l < 3) {
            g.out_t = m->ht[l];
            if (l == 0) MLP_CUDA(m, (launch_res<kHid / 2, 1, lbw_of(kInP), kHidden>(g, m->nsm, st, true)));
            else MLP_CUDA(m, (launch_res<kHid / 2, 2, kActLbw, kHidden>(g, m->nsm, st, true)));
            in = m->ht[l];
        } else {
            g.out_f = m->y;
            g.ld_f = kOutP;
            MLP_CUDA(m, (launch_res<kOut / 2, 2, kActLbw, kOutput>(g, m->nsm, st, true)));
        }
    }
    interval_stop(m, 0, chain_flops, chain_bytes);
    return STP_OK;
}

// Backward from dY (already in dt[3], its bias partials written by
// the loss kernel) to every parameter's gradient partials.
stp_status backward_impl(stp_mlp* m, int B, int* nwpart, int* nbpart) {
    const int Bp = (B + kTileM - 1) / kTileM * kTileM;
    const int mt = Bp / kTileM;
    cudaStream_t st = m->stream;
    const int KTb = Bp / kStageK;
    // Splits: the weight gradients of layers 2-4 take about 7/16 of the SMs
    // (one CTA a split), the input gradients beside them the rest (measured
    // balance of the two streams).
    const int target = std::max(1, std::min({kSplitMax, m->nsm * 7 / 16, KTb / 4}));
    const int kps = (KTb + target - 1) / target;
    const int splits = (KTb + kps - 1) / kps;  // every split non-empty
    *nwpart = splits;
    *nbpart = Bp / 32;
    // The weight gradients (one CTA per split computing both output tiles, so
    // each activation stage is read once) run on the side stream, each as
    // soon as its output gradient exists; the input gradients run back to
    // back on the main stream over the remaining SMs. The whole backward
    // pass is timed as one interval.
    double chain_flops = 0.0, chain_bytes = 0.0;
    for (int l = 3; l >= 0; --l) {
        chain_flops += 2.0 * B * kLayers[l].in_used * kLayers[l].out_used;
        chain_bytes += alg_bytes(B, kLayers[l].in_used, kLayers[l].out_used, kWGrad);
        if (l > 0) {
            chain_flops += 2.0 * B * kLayers[l].in_used * kLayers[l].out_used;
            chain_bytes += alg_bytes(B, kLayers[l].in_used, kLayers[l].out_used, kBackward);
        }
    }
    interval_start(m, 1);
    MLP_CUDA(m, cudaEventRecord(m->fork, st));  // dT_3 (the loss gradient) is ready
    for (int l = 3; l >= 0; --l) {
        // weight gradient: dW_l = dT_l^T . act_{l-1}   (M = out, N = in, K = batch)
        GemmArgs g{};
        g.A = m->dt[l];
        g.RA = Bp;
        g.B = (l == 0) ? m->xt : m->ht[l - 1];
        g.KT = KTb;
        g.kt_per_split = kps;
        g.out_f = m->wpart + (size_t)l * kSplitMax * kOutP * kHid;
        g.ld_f = kLayers[l].in;
        g.m_valid = kLayers[l].out;
        g.err = m->err;
        MLP_CUDA(m, cudaStreamWaitEvent(m->side, m->fork, 0));
        // The first layer's weight gradient follows the last input gradient,
        // when the main stream has no more work: its two output tiles take
        // separate CTAs, so it spreads over every SM as they free up.
        if (l == 0) MLP_CUDA(m, (launch_wgrad<kInP, lbw_of(kInP), 1>(g, splits, m->side)));
        else MLP_CUDA(m, (launch_wgrad<kHid, kActLbw, 2>(g, splits, m->side)));
        if (l == 0) break;
        // input gradient: dH_{l-1} = (dT_l . W_l) * relu'(h_{l-1})   (M = batch, N = in, K = out)
        ResArgs h{};
        h.A = m->dt[l];
        h.RA = Bp;
        h.B = m->wtT[l];
        h.NB = kLayers[l].in;
        h.units = 2 * mt;
        h.act = m->ht[l - 1];
        h.out_t = m->dt[l - 1];
        h.out_f = m->bpart + (size_t)(l - 1) * bpart_stride(m->Bp_max);
        h.err = m->err;
        MLP_CUDA(m, (launch_res<kHid / 2, 2, kActLbw, kBackward>(h, std::max(2, m->nsm - splits), st)));
        MLP_CUDA(m, cudaEventRecord(m->fork, st));  // dT_{l-1} is ready
    }
    MLP_CUDA(m, cudaEventRecord(m->join, m->side));
    MLP_CUDA(m, cudaStreamWaitEvent(st, m->join, 0));
    interval_stop(m, 1, chain_flops, chain_bytes);
    return STP_OK;
}

stp_status adam_impl(stp_mlp* m, int nwpart, int nbpart, float lr, bool update, bool keep_grads) {
    if (update) ++m->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = update ? 1.f - powf(b1, (float)m->step) : 1.f;
    const float c2 = update ? 1.f - powf(b2, (float)m->step) : 1.f;
    float* gout = m->gsum;
    AdamAll A{};
    for (int l = 0; l < 4; ++l) {
        const Layer& L = kLayers[l];
        AdamArgs a{};
        a.w = m->w[l];
        a.m = m->mw[l];
        a.v = m->vw[l];
        a.gpart = m->wpart + (size_t)l * kSplitMax * kOutP * kHid;
        a.nparts = nwpart;
        a.rows = L.out;
        a.cols = L.in;
        a.rows_used = L.out_used;
        a.wt = m->wt[l];
        a.wtT = m->wtT[l];
        a.gout = keep_grads ? gout : nullptr;
        a.lr = lr;
        a.b1 = b1;
        a.b2 = b2;
        a.eps = 1e-8f;
        a.c1 = c1;
        a.c2 = c2;
        a.update = update ? 1 : 0;
        const int n = L.out * L.in;
        gout += n;
        AdamArgs bb = a;
        bb.w = m->b[l];
        bb.m = m->mb[l];
        bb.v = m->vb[l];
        // bias partials are [chunk][256]: element e of chunk p at p * 256 + e
        bb.gpart = m->bpart + (size_t)l * bpart_stride(m->Bp_max);
        bb.nparts = nbpart;
        bb.rows = L.out;
        bb.cols = 1;
        bb.wt = nullptr;
        bb.wtT = nullptr;
        bb.gout = keep_grads ? gout : nullptr;
        gout += L.out;
        A.t[2 * l] = a;
        A.t[2 * l + 1] = bb;
        A.wblk[l + 1] = A.wblk[l] + (n + kAdamWElems - 1) / kAdamWElems;
        A.bblk[l + 1] = A.bblk[l] + (L.out + kAdamBElems - 1) / kAdamBElems;
    }
    k_adam_all<<<A.wblk[4] + A.bblk[4], kAdamThreads, 0, m->stream>>>(A);
    MLP_CUDA(m, cudaGetLastError());
    return STP_OK;
}

stp_status stage_in(stp_mlp* m, float* dst, const float* src, size_t n, int flags) {
    MLP_CUDA(m, cudaMemcpyAsync(dst, src, n * sizeof(float),
                                (flags & STP_MLP_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                m->stream));
    return STP_OK;
}

stp_status check_err(stp_mlp* m) {
    int e = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    collect_profile(m);
    if (e) {
        cudaMemsetAsync(m->err, 0, sizeof(int), m->stream);
        return fail(m, STP_ERR_TIMEOUT, "tensor-core pipeline wait exceeded its limit");
    }
    return STP_OK;
}

// Logical parameter count and offsets.
size_t nparam() {
    size_t n = 0;
    for (const Layer& L : kLayers) n += (size_t)L.out_used * L.in_used + L.out_used;
    return n;
}
}  // namespace

extern "C" {

stp_status stp_mlp_create(int max_batch, stp_mlp** out) {
    if (nparam() != (size_t)STP_MLP_NPARAM) return fail(nullptr, STP_ERR_INVALID, "parameter layout mismatch");
    if (!out) return fail(nullptr, STP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (max_batch <= 0 || max_batch > STP_MLP_MAX_BATCH) return fail(nullptr, STP_ERR_INVALID, "max_batch out of range");
    stp_mlp* m = new (std::nothrow) stp_mlp();
    if (!m) return fail(nullptr, STP_ERR_CAPACITY, "host allocation failed");
    m->max_batch = max_batch;
    const int Bp = (max_batch + kTileM - 1) / kTileM * kTileM;
    m->Bp_max = Bp;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || m->nsm < 2) {
            delete m;
            return fail(nullptr, STP_ERR_CUDA, "device query failed");
        }
    }
    // arena layout
    std::vector<std::pair<void**, size_t>> parts;
    for (int l = 0; l < 4; ++l) {
        const size_t n = (size_t)kLayers[l].out * kLayers[l].in;
        parts.push_back({(void**)&m->w[l], n * 4});
        parts.push_back({(void**)&m->mw[l], n * 4});
        parts.push_back({(void**)&m->vw[l], n * 4});
        parts.push_back({(void**)&m->wt[l], n * 2});
        parts.push_back({(void**)&m->wtT[l], n * 2});
        parts.push_back({(void**)&m->b[l], (size_t)kLayers[l].out * 4});
        parts.push_back({(void**)&m->mb[l], (size_t)kLayers[l].out * 4});
        parts.push_back({(void**)&m->vb[l], (size_t)kLayers[l].out * 4});
    }
    parts.push_back({(void**)&m->xt, (size_t)Bp * kInP * 2});
    for (int l = 0; l < 3; ++l) {
        parts.push_back({(void**)&m->ht[l], (size_t)Bp * kHid * 2});
    }
    for (int l = 0; l < 4; ++l) {
        parts.push_back({(void**)&m->dt[l], (size_t)Bp * kOutP * 2});
    }
    parts.push_back({(void**)&m->y, (size_t)Bp * kOutP * 4});
    parts.push_back({(void**)&m->wpart, (size_t)4 * kSplitMax * kOutP * kHid * 4});
    parts.push_back({(void**)&m->bpart, (size_t)4 * bpart_stride(Bp) * 4});
    parts.push_back({(void**)&m->gsum, (size_t)4 * (kOutP * kHid + kOutP) * 4});
    parts.push_back({(void**)&m->loss, (size_t)Bp * 4});
    parts.push_back({(void**)&m->X, (size_t)max_batch * kIn * 4});
    parts.push_back({(void**)&m->T, (size_t)max_batch * kTgt * 4});
    parts.push_back({(void**)&m->Yout, (size_t)max_batch * kOut * 4});
    parts.push_back({(void**)&m->err, 256});
    size_t total = 0;
    for (auto& p : parts) total += up256(p.second);
    if (cudaMalloc(&m->arena, total) != cudaSuccess) {
        delete m;
        return fail(nullptr, STP_ERR_CUDA, "device allocation failed");
    }
    m->arena_bytes = total;
    size_t off = 0;
    for (auto& p : parts) {
        *p.first = m->arena + off;
        off += up256(p.second);
    }
    bool events_ok = true;
    for (cudaEvent_t& e : m->ev) events_ok = events_ok && cudaEventCreate(&e) == cudaSuccess;
    if (cudaMemset(m->arena, 0, total) != cudaSuccess || !events_ok ||
        cudaStreamCreateWithFlags(&m->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&m->join, cudaEventDisableTiming) != cudaSuccess) {
        stp_mlp_free(m);
        return fail(nullptr, STP_ERR_CUDA, "device initialisation failed");
    }
    *out = m;
    return STP_OK;
}

void stp_mlp_free(stp_mlp* m) {
    if (!m) return;
    if (m->stream) cudaStreamSynchronize(m->stream);
    else cudaDeviceSynchronize();
    if (m->side) cudaStreamSynchronize(m->side);
    cudaFree(m->arena);
    for (cudaEvent_t e : m->ev)
        if (e) cudaEventDestroy(e);
    if (m->fork) cudaEventDestroy(m->fork);
    if (m->join) cudaEventDestroy(m->join);
    if (m->side) cudaStreamDestroy(m->side);
    delete m;
}

stp_status stp_mlp_set_stream(stp_mlp* m, void* stream) {
    if (!m) return fail(nullptr, STP_ERR_INVALID, "mlp is NULL");
    m->stream = (cudaStream_t)stream;
    return STP_OK;
}

stp_status stp_mlp_set_params(stp_mlp* m, const float* params) {
    if (!m || !params) return fail(m, STP_ERR_INVALID, "NULL argument");
    const float* p = params;
    for (int l = 0; l < 4; ++l) {
        const Layer& L = kLayers[l];
        std::vector<float> W((size_t)L.out * L.in, 0.f), b(L.out, 0.f);
        for (int r = 0; r < L.out_used; ++r)
            for (int c = 0; c < L.in_used; ++c) W[(size_t)r * L.in + c] = *p++;
        for (int r = 0; r < L.out_used; ++r) b[r] = *p++;
        MLP_CUDA(m, cudaMemcpyAsync(m->w[l], W.data(), W.size() * 4, cudaMemcpyHostToDevice, m->stream));
        MLP_CUDA(m, cudaMemcpyAsync(m->b[l], b.data(), b.size() * 4, cudaMemcpyHostToDevice, m->stream));
        MLP_CUDA(m, cudaMemsetAsync(m->mw[l], 0, W.size() * 4, m->stream));
        MLP_CUDA(m, cudaMemsetAsync(m->vw[l], 0, W.size() * 4, m->stream));
        MLP_CUDA(m, cudaMemsetAsync(m->mb[l], 0, b.size() * 4, m->stream));
        MLP_CUDA(m, cudaMemsetAsync(m->vb[l], 0, b.size() * 4, m->stream));
        MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    }
    m->step = 0;
    // refresh the BF16 operand copies (no update)
    stp_status s = adam_impl(m, 0, 0, 0.f, false, false);
    if (s != STP_OK) return s;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return STP_OK;
}

stp_status stp_mlp_get_params(stp_mlp* m, float* params) {
    if (!m || !params) return fail(m, STP_ERR_INVALID, "NULL argument");
    float* p = params;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    for (int l = 0; l < 4; ++l) {
        const Layer& L = kLayers[l];
        std::vector<float> W((size_t)L.out * L.in), b(L.out);
        MLP_CUDA(m, cudaMemcpy(W.data(), m->w[l], W.size() * 4, cudaMemcpyDeviceToHost));
        MLP_CUDA(m, cudaMemcpy(b.data(), m->b[l], b.size() * 4, cudaMemcpyDeviceToHost));
        for (int r = 0; r < L.out_used; ++r)
            for (int c = 0; c < L.in_used; ++c) *p++ = W[(size_t)r * L.in + c];
        for (int r = 0; r < L.out_used; ++r) *p++ = b[r];
    }
    return STP_OK;
}

stp_status stp_mlp_forward(stp_mlp* m, int B, const float* X, float* Y, int flags) {
    if (!m || !X || !Y) return fail(m, STP_ERR_INVALID, "NULL argument");
    if (B <= 0 || B > m->max_batch) return fail(m, STP_ERR_INVALID, "batch out of range");
    stp_status s = stage_in(m, m->X, X, (size_t)B * kIn, flags);
    if (s != STP_OK) return s;
    if ((s = forward_impl(m, B)) != STP_OK) return s;
    const int n = B * kOut;
    k_unpack_out<<<(n + 255) / 256, 256, 0, m->stream>>>(m->y, B, m->Yout);
    MLP_CUDA(m, cudaGetLastError());
    MLP_CUDA(m, cudaMemcpyAsync(Y, m->Yout, (size_t)n * 4,
                                (flags & STP_MLP_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                m->stream));
    return check_err(m);
}

static stp_status loss_grad(stp_mlp* m, int B, const float* X, const float* T, int flags, int* nw, int* nb) {
    if (!m || !X || !T) return fail(m, STP_ERR_INVALID, "NULL argument");
    if (B <= 0 || B > m->max_batch) return fail(m, STP_ERR_INVALID, "batch out of range");
    stp_status s = stage_in(m, m->X, X, (size_t)B * kIn, flags);
    if (s != STP_OK) return s;
    if ((s = stage_in(m, m->T, T, (size_t)B * kTgt, flags)) != STP_OK) return s;
    interval_start(m, 2);  // the training step's device work, inputs staged
    if ((s = forward_impl(m, B)) != STP_OK) return s;
    const int Bp = (B + kTileM - 1) / kTileM * kTileM;
    k_loss<<<Bp / kLossRows, kLossThreads, 0, m->stream>>>(
        m->y, m->T, B, m->bpart + (size_t)3 * bpart_stride(m->Bp_max), m->dt[3], Bp, m->loss);
    MLP_CUDA(m, cudaGetLastError());
    return backward_impl(m, B, nw, nb);
}

static stp_status read_loss(stp_mlp* m, int B, float* loss) {
    if (!loss) return STP_OK;
    std::vector<float> l(B);
    MLP_CUDA(m, cudaMemcpyAsync(l.data(), m->loss, (size_t)B * 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    double s = 0;
    for (float v : l) s += v;
    *loss = (float)(s / B);
    return STP_OK;
}

stp_status stp_mlp_gradients(stp_mlp* m, int B, const float* X, const float* T, float* loss, float* grads,
                             int flags) {
    int nw = 0, nb = 0;
    stp_status s = loss_grad(m, B, X, T, flags, &nw, &nb);
    if (s != STP_OK) return s;
    if ((s = adam_impl(m, nw, nb, 0.f, false, true)) != STP_OK) return s;
    interval_stop(m, 2, 0.0, 0.0);
    if ((s = check_err(m)) != STP_OK) return s;
    if ((s = read_loss(m, B, loss)) != STP_OK) return s;
    if (grads) {
        // padded gradient tensors -> logical order
        float* p = grads;
        const float* g = m->gsum;
        for (int l = 0; l < 4; ++l) {
            const Layer& L = kLayers[l];
            std::vector<float> W((size_t)L.out * L.in), b(L.out);
            MLP_CUDA(m, cudaMemcpy(W.data(), g, W.size() * 4, cudaMemcpyDeviceToHost));
            g += W.size();
            MLP_CUDA(m, cudaMemcpy(b.data(), g, b.size() * 4, cudaMemcpyDeviceToHost));
            g += b.size();
            for (int r = 0; r < L.out_used; ++r)
                for (int c = 0; c < L.in_used; ++c) *p++ = W[(size_t)r * L.in + c];
            for (int r = 0; r < L.out_used; ++r) *p++ = b[r];
        }
    }
    return STP_OK;
}

stp_status stp_mlp_train_step(stp_mlp* m, int B, const float* X, const float* T, float lr, float* loss, int flags) {
    if (!(lr >= 0.f)) return fail(m, STP_ERR_INVALID, "learning rate must be >= 0");
    int nw = 0, nb = 0;
    stp_status s = loss_grad(m, B, X, T, flags, &nw, &nb);
    if (s != STP_OK) return s;
    if ((s = adam_impl(m, nw, nb, lr, true, false)) != STP_OK) return s;
    interval_stop(m, 2, 0.0, 0.0);
    if ((s = check_err(m)) != STP_OK) return s;
    return read_loss(m, B, loss);
}

stp_status stp_mlp_set_profiling(stp_mlp* m, int on) {
    if (!m) return fail(nullptr, STP_ERR_INVALID, "mlp is NULL");
    m->profiling = on != 0;
    m->gemm_ms = 0;
    m->gemm_flops = 0;
    m->gemm_bytes = 0;
    m->step_ms = 0;
    m->steps = 0;
    for (bool& p : m->ev_pending) p = false;
    return STP_OK;
}

stp_status stp_mlp_profile(stp_mlp* m, double* gemm_ms, double* gemm_flops, double* gemm_bytes) {
    if (!m) return fail(nullptr, STP_ERR_INVALID, "mlp is NULL");
    if (gemm_ms) *gemm_ms = m->gemm_ms;
    if (gemm_flops) *gemm_flops = m->gemm_flops;
    if (gemm_bytes) *gemm_bytes = m->gemm_bytes;
    m->gemm_bytes = 0;
    m->gemm_ms = 0;
    m->gemm_flops = 0;
    return STP_OK;
}
stp_status stp_mlp_profile_step(stp_mlp* m, double* step_ms, int* steps) {
    if (!m) return fail(nullptr, STP_ERR_INVALID, "mlp is NULL");
    if (step_ms) *step_ms = m->step_ms;
    if (steps) *steps = m->steps;
    m->step_ms = 0;
    m->steps = 0;
    return STP_OK;
}

const char* stp_mlp_last_error(const stp_mlp* m) { return m ? m->last_error.c_str() : g_mlp_err.c_str(); }

}  // extern "C"
