// Fused inference of the learned slope predictor (the network of mlp.cu) for one
// block's share of the subapertures, run by the consumer warps of the frame and
// loop kernels between their two grid barriers:
//   pixel stage -> grid barrier -> predict (this file) -> grid barrier -> MVM.
//
// The network is small (200 -> 64 -> 64 -> 2), so the phase is latency-bound:
// the BF16 weight fragments of both hidden layers, their biases and the
// neighbour indices are loaded into registers in the same round of L2 loads as
// the first tile's features, and each hidden layer is one pass of
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate) by 8 warps, one 8-column slice
// each over both 16-row halves of a 32-sample tile.
//
// Arithmetic per element is that of the stand-alone predictor kernel: the same
// BF16 operands, the same k order of the tensor-core steps, bias added after the
// sum, exact-erf GELU, the output layer as one FMA chain in j order, and
//     s_pred = fma(sigma, y, s_k),
// so the fused and stand-alone forms give identical predictions.
#pragma once

#include <cuda_bf16.h>

#include "stream_mvm.cuh"

#ifndef RTC_PRED_STAMP
#define RTC_PRED_STAMP(i) \
    do {                  \
    } while (0)
#endif

namespace rtc_pred {

using rtc_mvm::consumer_sync;
using rtc_mvm::kConsumers;

constexpr int NF = 200;                 // features: 5x5 neighbours x (x, y) x 4 frames
constexpr int KP = 208;                 // W1 row pitch (features padded to a multiple of 16)
constexpr int NH = 64;                  // hidden width
constexpr int NO = 2;                   // outputs (x and y slope)
constexpr int TS = 32;                  // samples per tile (two 16-row MMA halves)
constexpr int XP = 216;                 // X row pitch in BF16 (bank-conflict-free fragments)
constexpr int HP = 72;                  // H1 row pitch in BF16
constexpr int H2P = 68;                 // H2 row pitch in FP32
constexpr int kMmaWarps = NH / 8;       // one 8-column slice per warp
constexpr int kPairs = TS * 25;         // (sample, neighbour) pairs of a tile
constexpr int kPairRounds = (kPairs + kConsumers - 1) / kConsumers;

// Offsets of the parameters in the flat vector (W1, b1, W2, b2, W3, b3).
constexpr int OFF_B1 = NH * NF;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NO * NH;

// Shared-memory layout of the phase (byte offsets).
constexpr int SM_X = 0;                              // bf16 [TS][XP]
constexpr int SM_H1 = SM_X + TS * XP * 2;            // bf16 [TS][HP]
constexpr int SM_H2 = SM_H1 + TS * HP * 2;           // f32 [TS][H2P]
constexpr int SM_W3 = SM_H2 + TS * H2P * 4;          // f32 W3 [NO][NH], then b3 [NO]
constexpr int kSmemBytes = SM_W3 + (NO * NH + NO + 2) * 4;

static_assert(kPairRounds == 2, "gather registers assume two rounds of pairs");
static_assert(SM_H1 % 16 == 0 && SM_H2 % 16 == 0 && SM_W3 % 16 == 0, "alignment");
static_assert(OFF_B3 == OFF_W3 + NO * NH, "W3 and b3 are one run of the parameters");
static_assert(NF % 8 == 0 && NF + 8 == KP, "the last k step holds 8 features and 8 zero columns");

struct PredArgs {
    const __nv_bfloat16* w1;  // [NH][KP] BF16 copy of W1, zero padded
    const __nv_bfloat16* w2;  // [NH][NH] BF16 copy of W2
    const float* params;      // flat FP32 parameters (b1, b2, W3, b3 are read from here)
    const int* nbr;           // [nv][25] neighbour index or -1, (dr, dc) row-major
    float* ring;              // [4][kpad] measured slope vectors (x block, then y block)
    float* s_pred;            // [kpad] predicted next slopes
    int kpad, nv;
    float sigma, inv_sigma;
};

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
}

__device__ __forceinline__ uint32_t ld32g(const __nv_bfloat16* p) {
    return __ldg(reinterpret_cast<const unsigned int*>(p));
}
__device__ __forceinline__ uint32_t ld32s(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// What a consumer thread keeps in registers for the phase.
struct Regs {
    uint32_t w1f[KP / 16][2];   // B fragments of W1 for this warp's 8 columns
    uint32_t w2f[NH / 16][2];   // B fragments of W2
    float b1v[2], b2v[2];       // biases of the thread's two accumulator columns
    int jn[kPairRounds];        // neighbour indices of the first tile's pairs
    float vo[kPairRounds][6];   // their slopes of the three older frames (lags 1-3)
};

// Neighbour index of pair p (sample p / 25, neighbour p % 25) of the tile at t0.
__device__ __forceinline__ int pair_nbr(const PredArgs& pa, int t0, int i1, int p) {
    if (p >= kPairs) return -1;
    const int i = t0 + p / 25;
    return i < i1 ? __ldg(pa.nbr + static_cast<size_t>(i) * 25 + (p - (p / 25) * 25)) : -1;
}

// What the first tile needs that does not depend on this frame's slopes: the
// weight fragments, biases and neighbour indices in registers, the first tile's
// features of the three older frames (ring rows head-1 .. head-3, written by earlier
// frames) in registers, and the output layer's weights in the scratch sm
// (asynchronous copies, complete once predict's first barrier has passed).
// [i0, i1): the block's subapertures.  Call it after the block's grid-barrier
// arrival (a release would wait for these loads) and before its wait.
__device__ __forceinline__ void prefetch(const PredArgs& pa, unsigned char* sm, int tid, int i0, int i1,
                                         int head, Regs& r) {
    float* w3s = reinterpret_cast<float*>(sm + SM_W3);
    for (int k = tid; k < NO * NH + NO; k += kConsumers) rtc_mvm::cp_async4(w3s + k, pa.params + OFF_W3 + k);
    asm volatile("cp.async.commit_group;" ::: "memory");
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    if (warp < kMmaWarps) {
        const __nv_bfloat16* w1 = pa.w1 + static_cast<size_t>(warp * 8 + g) * KP + 2 * t;
#pragma unroll
        for (int ks = 0; ks < KP / 16; ++ks) {
            r.w1f[ks][0] = ld32g(w1 + ks * 16);
            r.w1f[ks][1] = ld32g(w1 + ks * 16 + 8);
        }
        const __nv_bfloat16* w2 = pa.w2 + static_cast<size_t>(warp * 8 + g) * NH + 2 * t;
#pragma unroll
        for (int ks = 0; ks < NH / 16; ++ks) {
            r.w2f[ks][0] = ld32g(w2 + ks * 16);
            r.w2f[ks][1] = ld32g(w2 + ks * 16 + 8);
        }
        const int c = warp * 8 + 2 * t;
        r.b1v[0] = __ldg(pa.params + OFF_B1 + c);
        r.b1v[1] = __ldg(pa.params + OFF_B1 + c + 1);
        r.b2v[0] = __ldg(pa.params + OFF_B2 + c);
        r.b2v[1] = __ldg(pa.params + OFF_B2 + c + 1);
    }
#pragma unroll
    for (int q = 0; q < kPairRounds; ++q) r.jn[q] = pair_nbr(pa, i0, i1, tid + q * kConsumers);
#pragma unroll
    for (int q = 0; q < kPairRounds; ++q)
#pragma unroll
        for (int la = 2; la < 8; ++la) {
            const float* row = pa.ring + static_cast<size_t>((head - (la >> 1)) & 3) * pa.kpad;
            r.vo[q][la - 2] = r.jn[q] >= 0 ? __ldcg(row + (la & 1) * pa.nv + r.jn[q]) : 0.f;
        }
}

// After the grid barrier that completes the measured slopes: predictions of
// subapertures [i0, i1) from the ring rows head, head-1, head-2, head-3 (newest
// first), with the registers and scratch `prefetch` filled (before the barrier, so
// that the weight and neighbour loads overlap the wait).  Every consumer thread
// calls it; sm is TS-sample scratch of kSmemBytes.  src(i, axis) gives the block's
// own copy of the measured slope s_k of subaperture i (the value in ring row head);
// each prediction goes to pa.s_pred and to sink(i, axis, value), after the same
// thread's src read of that slope.  Ends with a consumer barrier.
template <typename Src, typename Sink>
__device__ __forceinline__ void predict(const PredArgs& pa, unsigned char* sm, int tid, int i0, int i1,
                                        int head, const Regs& r, const Src& src, const Sink& sink) {
    const int warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t = lane & 3;
    __nv_bfloat16* X = reinterpret_cast<__nv_bfloat16*>(sm + SM_X);
    __nv_bfloat16* H1 = reinterpret_cast<__nv_bfloat16*>(sm + SM_H1);
    float* H2 = reinterpret_cast<float*>(sm + SM_H2);
    const float* W3 = reinterpret_cast<const float*>(sm + SM_W3);
    const float* b3 = W3 + NO * NH;
    const float* rows[4];
#pragma unroll
    for (int lag = 0; lag < 4; ++lag)
        rows[lag] = pa.ring + static_cast<size_t>((head - lag) & 3) * pa.kpad;

    RTC_PRED_STAMP(0);
    for (int t0 = i0; t0 < i1; t0 += TS) {
        int jn[kPairRounds];
#pragma unroll
        for (int q = 0; q < kPairRounds; ++q)
            jn[q] = t0 == i0 ? r.jn[q] : pair_nbr(pa, t0, i1, tid + q * kConsumers);
        // gather: every load of the thread's pairs in flight before any store; the
        // newest row was written by other blocks of this kernel, so it is read from
        // L2 (the first tile's older rows came with prefetch)
        float v[kPairRounds][8];
#pragma unroll
        for (int q = 0; q < kPairRounds; ++q)
#pragma unroll
            for (int la = 0; la < 8; ++la) {
                const int j = jn[q];
                if (la >= 2 && t0 == i0) v[q][la] = r.vo[q][la - 2];
                else v[q][la] = j >= 0 ? __ldcg(rows[la >> 1] + (la & 1) * pa.nv + j) : 0.f;
            }
#pragma unroll
        for (int q = 0; q < kPairRounds; ++q) {
            const int p = tid + q * kConsumers;
            if (p < kPairs) {
                const int s = p / 25, nb = p - s * 25;
#pragma unroll
                for (int la = 0; la < 8; ++la)
                    X[s * XP + la * 25 + nb] = __float2bfloat16_rn(v[q][la] * pa.inv_sigma);
            }
        }
        if (t0 == i0) rtc_mvm::rows_landed();     // the output layer's weights (prefetch)
        consumer_sync();
        RTC_PRED_STAMP(1);

        // hidden layer 1: z1 = X W1^T + b1, h1 = GELU(z1) as BF16; the upper half of
        // the last k step is the zero padding of W1 and X (not stored: zero fragments)
        if (warp < kMmaWarps) {
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int ks = 0; ks < KP / 16; ++ks) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const __nv_bfloat16* A = X + (mt * 16 + g) * XP + ks * 16 + 2 * t;
                    const bool hi = ks * 16 + 8 < NF;
                    const uint32_t a[4] = {ld32s(A), ld32s(A + 8 * XP), hi ? ld32s(A + 8) : 0u,
                                           hi ? ld32s(A + 8 * XP + 8) : 0u};
                    mma16816(acc[mt], a, r.w1f[ks][0], r.w1f[ks][1]);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int row = mt * 16 + g + (h >> 1) * 8, col = warp * 8 + 2 * t + (h & 1);
                    H1[row * HP + col] = __float2bfloat16_rn(gelu(acc[mt][h] + r.b1v[h & 1]));
                }
        }
        consumer_sync();
        RTC_PRED_STAMP(2);

        // hidden layer 2: z2 = h1 W2^T + b2, h2 = GELU(z2) in FP32
        if (warp < kMmaWarps) {
            float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
#pragma unroll
            for (int ks = 0; ks < NH / 16; ++ks) {
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    const __nv_bfloat16* A = H1 + (mt * 16 + g) * HP + ks * 16 + 2 * t;
                    const uint32_t a[4] = {ld32s(A), ld32s(A + 8 * HP), ld32s(A + 8), ld32s(A + 8 * HP + 8)};
                    mma16816(acc[mt], a, r.w2f[ks][0], r.w2f[ks][1]);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int row = mt * 16 + g + (h >> 1) * 8, col = warp * 8 + 2 * t + (h & 1);
                    H2[row * H2P + col] = gelu(acc[mt][h] + r.b2v[h & 1]);
                }
        }
        consumer_sync();
        RTC_PRED_STAMP(3);

        // output layer on CUDA cores and the predicted next slopes
        if (tid < TS * NO) {
            const int s = tid >> 1, o = tid & 1;
            const int i = t0 + s;
            if (i < i1) {
                float y = b3[o];
#pragma unroll 16
                for (int j = 0; j < NH; ++j) y = fmaf(H2[s * H2P + j], W3[o * NH + j], y);
                const float sp = __fmaf_rn(pa.sigma, y, src(i, o));
                pa.s_pred[o * pa.nv + i] = sp;
                sink(i, o, sp);
            }
        }
        consumer_sync();
        RTC_PRED_STAMP(4);
    }
    if (i0 >= i1) rtc_mvm::rows_landed();         // no tile: still no copy left in flight
}

}  // namespace rtc_pred

// Predictor arguments of a handle with a loaded predictor (defined in frame_kernel.cu).
rtc_pred::PredArgs pred_args(const rtc_handle* h);
