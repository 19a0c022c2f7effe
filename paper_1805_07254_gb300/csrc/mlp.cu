// Learned slope predictor: a shared MLP 200 -> 64 -> 64 -> 2 with exact GELU,
// BF16 weights and activations in BF16 tensor-core GEMMs with FP32 accumulation.
//
// The paper has no learned component; this predictor offsets the one-frame servo
// lag of the integrator by predicting each subaperture's next slopes from the
// 5x5 neighbourhood of subapertures over the last 4 frames (200 features):
//   feature f = ((lag*2 + axis)*5 + (dr+2))*5 + (dc+2),   value / sigma
//   z1 = X W1^T + b1, h1 = GELU(z1), z2 = h1 W2^T + b2, h2 = GELU(z2),
//   y = h2 W3^T + b3,  next slopes = s_k + sigma * y.
// Training minimises sum((y - t)^2) / (2B) with t = (s_{k+1} - s_k) / sigma, by
// Adam with bias correction, on FP32 master weights.
//
// One CTA of 4 warps takes 64 samples.  Every GEMM is a warp-level loop of
// mma.sync.m16n8k16 (BF16 in, FP32 accumulate) over operands kept in shared
// memory K-contiguous (A as [M][K], B as [N][K]), so the backward weight-gradient
// GEMMs read transposed copies of X, h1 and dz written during the forward pass.
// The 64 -> 2 output layer and its gradient run on CUDA cores in FP32.  Weight
// gradients are written per CTA and summed over CTAs in a fixed pairwise order by
// the update kernel, which also applies Adam and refreshes the BF16 copies.

#include <cuda_bf16.h>
#include <math.h>

#include "rtc_internal.h"
#include "mlp.h"
#include "pred_tile.cuh"

namespace {

constexpr int NF = 200;          // features
constexpr int KP = 208;          // features padded to a multiple of 16
constexpr int NH = 64;           // hidden width
constexpr int NO = 2;            // outputs
constexpr int TM = 64;           // samples per CTA
constexpr int kWarps = 4;
constexpr int kThreads = kWarps * 32;

// Offsets of each parameter in the flat vector (W1, b1, W2, b2, W3, b3, row-major).
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NF;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NO * NH;
constexpr int NPARAM = OFF_B3 + NO;
static_assert(NPARAM == RTC_MLP_NPARAMS, "parameter count");

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t ld32(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// acc[16 rows from m0][N] += A[m0.., 0:K] * B[0:N, 0:K]^T; A is [*][lda], B is [N][ldb].
// Fragment layout of m16n8k16: g = lane/4, t = lane%4; a0 = (g, 2t..2t+1),
// a1 = (g+8, 2t..), a2 = (g, 2t+8..), a3 = (g+8, 2t+8..); b0 = (k 2t..2t+1, n g),
// b1 = (k 2t+8.., n g); c0,c1 = (g, 2t..2t+1), c2,c3 = (g+8, 2t..2t+1).
template <int N, int K>
__device__ __forceinline__ void warp_gemm(const bf16* A, int lda, int m0, const bf16* B, int ldb,
                                          float acc[N / 8][4]) {
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll 1
    for (int k0 = 0; k0 < K; k0 += 16) {
        uint32_t a[4];
        a[0] = ld32(A + (m0 + g) * lda + k0 + 2 * t);
        a[1] = ld32(A + (m0 + g + 8) * lda + k0 + 2 * t);
        a[2] = ld32(A + (m0 + g) * lda + k0 + 2 * t + 8);
        a[3] = ld32(A + (m0 + g + 8) * lda + k0 + 2 * t + 8);
#pragma unroll
        for (int nt = 0; nt < N / 8; ++nt) {
            uint32_t b[2];
            b[0] = ld32(B + (nt * 8 + g) * ldb + k0 + 2 * t);
            b[1] = ld32(B + (nt * 8 + g) * ldb + k0 + 2 * t + 8);
            mma16816(acc[nt], a, b);
        }
    }
}

using rtc_pred::gelu;     // the same function as the fused inference
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Shared-memory layout of one CTA (byte offsets).
struct Smem {
    static constexpr int W1 = 0;                                   // bf16 [NH][KP]
    static constexpr int W2 = W1 + NH * KP * 2;                     // bf16 [NH][NH] (W2[n][k])
    static constexpr int W2T = W2 + NH * NH * 2;                    // bf16 [NH][NH] (W2[k][n] at [n][k])
    static constexpr int B1 = W2T + NH * NH * 2;                    // f32 [NH]
    static constexpr int B2 = B1 + NH * 4;                          // f32 [NH]
    static constexpr int W3 = B2 + NH * 4;                          // f32 [NO][NH]
    static constexpr int B3 = W3 + NO * NH * 4;                     // f32 [NO] (+pad)
    static constexpr int X = B3 + 16;                               // bf16 [TM][KP]
    static constexpr int XT = X + TM * KP * 2;                      // bf16 [KP][TM]
    static constexpr int Z1 = XT + KP * TM * 2;                     // f32 [TM][NH]
    static constexpr int H1 = Z1 + TM * NH * 4;                     // bf16 [TM][NH]
    static constexpr int H1T = H1 + TM * NH * 2;                    // bf16 [NH][TM]
    static constexpr int Z2 = H1T + NH * TM * 2;                    // f32 [TM][NH]
    static constexpr int H2 = Z2 + TM * NH * 4;                     // f32 [TM][NH]
    static constexpr int DZ2 = H2 + TM * NH * 4;                    // bf16 [TM][NH]
    static constexpr int DZ2T = DZ2 + TM * NH * 2;                  // bf16 [NH][TM]
    static constexpr int DZ1T = DZ2T + NH * TM * 2;                 // bf16 [NH][TM]
    static constexpr int Y = DZ1T + NH * TM * 2;                    // f32 [TM][NO]
    static constexpr int DY = Y + TM * NO * 4;                      // f32 [TM][NO]
    static constexpr int TGT = DY + TM * NO * 4;                    // f32 [TM][NO]
    static constexpr int RED = TGT + TM * NO * 4;                   // f32 [NH] scratch sums
    static constexpr int LOSS = RED + NH * 4 * 2;                   // f32 [kWarps]
    static constexpr int SAMP = (LOSS + 64 + 15) / 16 * 16;         // int2 [TM] (subap, frame)
    static constexpr int TOTAL = SAMP + TM * 8;
};

// Weights into shared memory: BF16 copies of W1 (padded), W2 and W2^T; FP32 rest.
__device__ void load_weights(unsigned char* sm, const MlpDev& w) {
    bf16* W1 = reinterpret_cast<bf16*>(sm + Smem::W1);
    bf16* W2 = reinterpret_cast<bf16*>(sm + Smem::W2);
    bf16* W2T = reinterpret_cast<bf16*>(sm + Smem::W2T);
    float* b1 = reinterpret_cast<float*>(sm + Smem::B1);
    float* b2 = reinterpret_cast<float*>(sm + Smem::B2);
    float* W3 = reinterpret_cast<float*>(sm + Smem::W3);
    float* b3 = reinterpret_cast<float*>(sm + Smem::B3);
    // 16-byte copies of the BF16 weights, then W2^T from the shared copy
    for (int i = threadIdx.x; i < NH * KP / 8; i += kThreads)
        reinterpret_cast<uint4*>(W1)[i] = __ldg(reinterpret_cast<const uint4*>(w.w1_bf16) + i);
    for (int i = threadIdx.x; i < NH * NH / 8; i += kThreads)
        reinterpret_cast<uint4*>(W2)[i] = __ldg(reinterpret_cast<const uint4*>(w.w2_bf16) + i);
    for (int i = threadIdx.x; i < NH; i += kThreads) {
        b1[i] = w.master[OFF_B1 + i];
        b2[i] = w.master[OFF_B2 + i];
    }
    for (int i = threadIdx.x; i < NO * NH; i += kThreads) W3[i] = w.master[OFF_W3 + i];
    if (threadIdx.x < NO) b3[threadIdx.x] = w.master[OFF_B3 + threadIdx.x];
    __syncthreads();
    for (int i = threadIdx.x; i < NH * NH; i += kThreads) {
        const int n = i / NH, k = i - n * NH;
        W2T[i] = W2[k * NH + n];
    }
}

// Features of the CTA's samples from slope rows, by (sample, neighbour) pairs: for a
// batch of pairs every neighbour index is loaded at once, then every slope value of
// the batch, before the stores (the gather is latency-bound).  X[s][f] and, if
// want_t, XT[f][s] get bf16(value / sigma) with f = (lag*2 + axis)*25 + nb; off-pupil
// neighbours and invalid samples give 0.  subap_of(s): the sample's subaperture or
// -1; row_of(s, lag): its slope row at that lag (x block then y block).
template <typename SubFn, typename RowFn>
__device__ void gather_pairs(unsigned char* sm, bool want_t, const int* __restrict__ nbr, int nv,
                             float inv_sigma, const SubFn& subap_of, const RowFn& row_of) {
    bf16* X = reinterpret_cast<bf16*>(sm + Smem::X);
    bf16* XT = reinterpret_cast<bf16*>(sm + Smem::XT);
    constexpr int kPairs = TM * 25;
    constexpr int kBatch = 5;
    for (int p0 = threadIdx.x; p0 < kPairs; p0 += kBatch * kThreads) {
        int j[kBatch];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int p = p0 + b * kThreads;
            j[b] = -1;
            if (p < kPairs) {
                const int si = p / 25;
                const int i = subap_of(si);
                if (i >= 0) j[b] = __ldg(nbr + i * 25 + (p - si * 25));
            }
        }
        float v[kBatch][8];
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int si = (p0 + b * kThreads) / 25;
#pragma unroll
            for (int la = 0; la < 8; ++la)
                v[b][la] = j[b] >= 0 ? row_of(si, la >> 1)[(la & 1) * nv + j[b]] : 0.f;
        }
#pragma unroll
        for (int b = 0; b < kBatch; ++b) {
            const int p = p0 + b * kThreads;
            if (p < kPairs) {
                const int si = p / 25, nb = p - si * 25;
#pragma unroll
                for (int la = 0; la < 8; ++la) {
                    const int f = la * 25 + nb;
                    const bf16 x = __float2bfloat16_rn(v[b][la] * inv_sigma);
                    X[si * KP + f] = x;
                    if (want_t) XT[f * TM + si] = x;
                }
            }
        }
    }
    // the K padding columns
    for (int q = threadIdx.x; q < TM * (KP - NF); q += kThreads) {
        const int si = q / (KP - NF), c = NF + (q - si * (KP - NF));
        X[si * KP + c] = __float2bfloat16_rn(0.f);
        if (want_t) XT[c * TM + si] = __float2bfloat16_rn(0.f);
    }
}

// Feature rows of the CTA's samples: x[s][f] for s < ns (zero rows beyond), as BF16
// in X (and, if want_t, transposed in XT).  feat(s, f) gives the FP32 value.
template <typename Feat>
__device__ void gather_tile(unsigned char* sm, int ns, bool want_t, const Feat& feat) {
    bf16* X = reinterpret_cast<bf16*>(sm + Smem::X);
    bf16* XT = reinterpret_cast<bf16*>(sm + Smem::XT);
    for (int i = threadIdx.x; i < TM * KP; i += kThreads) {
        const int s = i / KP, f = i - s * KP;
        const float v = (s < ns && f < NF) ? feat(s, f) : 0.f;
        const bf16 b = __float2bfloat16_rn(v);
        X[i] = b;
        if (want_t) XT[f * TM + s] = b;
    }
}

// Forward pass of the CTA tile; y (FP32) left in Smem::Y.  want_t keeps the
// transposed h1 for the backward pass.
__device__ void forward_tile(unsigned char* sm, bool want_t) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int m0 = warp * 16;
    const bf16* X = reinterpret_cast<const bf16*>(sm + Smem::X);
    const bf16* W1 = reinterpret_cast<const bf16*>(sm + Smem::W1);
    const bf16* W2 = reinterpret_cast<const bf16*>(sm + Smem::W2);
    const float* b1 = reinterpret_cast<const float*>(sm + Smem::B1);
    const float* b2 = reinterpret_cast<const float*>(sm + Smem::B2);
    float* Z1 = reinterpret_cast<float*>(sm + Smem::Z1);
    bf16* H1 = reinterpret_cast<bf16*>(sm + Smem::H1);
    bf16* H1T = reinterpret_cast<bf16*>(sm + Smem::H1T);
    float* Z2 = reinterpret_cast<float*>(sm + Smem::Z2);
    float* H2 = reinterpret_cast<float*>(sm + Smem::H2);

    float acc[NH / 8][4];
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<NH, KP>(X, KP, m0, W1, KP, acc);
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int r = m0 + g + (h >> 1) * 8, c = nt * 8 + 2 * t + (h & 1);
            const float z = acc[nt][h] + b1[c];
            Z1[r * NH + c] = z;
            const bf16 a = __float2bfloat16_rn(gelu(z));
            H1[r * NH + c] = a;
            if (want_t) H1T[c * TM + r] = a;
        }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_gemm<NH, NH>(H1, NH, m0, W2, NH, acc);
#pragma unroll
    for (int nt = 0; nt < NH / 8; ++nt)
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int r = m0 + g + (h >> 1) * 8, c = nt * 8 + 2 * t + (h & 1);
            const float z = acc[nt][h] + b2[c];
            Z2[r * NH + c] = z;
            H2[r * NH + c] = gelu(z);
        }
    __syncthreads();
    // output layer on CUDA cores: y[s][o] = b3[o] + sum_j h2[s][j] W3[o][j]
    const float* W3 = reinterpret_cast<const float*>(sm + Smem::W3);
    const float* b3 = reinterpret_cast<const float*>(sm + Smem::B3);
    float* Y = reinterpret_cast<float*>(sm + Smem::Y);
    for (int i = threadIdx.x; i < TM * NO; i += kThreads) {
        const int s = i / NO, o = i - s * NO;
        float v = b3[o];
        for (int j = 0; j < NH; ++j) v = fmaf(H2[s * NH + j], W3[o * NH + j], v);
        Y[i] = v;
    }
    __syncthreads();
}

// Backward pass of the CTA tile given targets in Smem::TGT; writes this CTA's
// gradient contribution (and loss sum) to part[NPARAM + 1].
__device__ void backward_tile(unsigned char* sm, int ns, float inv_batch, float* __restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const float* Y = reinterpret_cast<const float*>(sm + Smem::Y);
    const float* TG = reinterpret_cast<const float*>(sm + Smem::TGT);
    float* DY = reinterpret_cast<float*>(sm + Smem::DY);
    const float* H2 = reinterpret_cast<const float*>(sm + Smem::H2);
    const float* Z2 = reinterpret_cast<const float*>(sm + Smem::Z2);
    const float* Z1 = reinterpret_cast<const float*>(sm + Smem::Z1);
    const float* W3 = reinterpret_cast<const float*>(sm + Smem::W3);
    bf16* DZ2 = reinterpret_cast<bf16*>(sm + Smem::DZ2);
    bf16* DZ2T = reinterpret_cast<bf16*>(sm + Smem::DZ2T);
    bf16* DZ1T = reinterpret_cast<bf16*>(sm + Smem::DZ1T);
    float* LOSS = reinterpret_cast<float*>(sm + Smem::LOSS);

    // dy = (y - t) / B for real samples, 0 for padding rows; loss partial sum
    float l = 0.f;
    for (int i = threadIdx.x; i < TM * NO; i += kThreads) {
        const int s = i / NO;
        const float e = (s < ns) ? Y[i] - TG[i] : 0.f;
        DY[i] = e * inv_batch;
        l = fmaf(e, e, l);
    }
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if (lane == 0) LOSS[warp] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int w = 0; w < kWarps; ++w) s += LOSS[w];
        part[NPARAM] = s;
    }
    // dW3[o][j] = sum_s dy[s][o] h2[s][j]; db3[o] = sum_s dy[s][o]
    for (int i = threadIdx.x; i < NO * NH + NO; i += kThreads) {
        float v = 0.f;
        if (i < NO * NH) {
            const int o = i / NH, j = i - o * NH;
            for (int s = 0; s < TM; ++s) v = fmaf(DY[s * NO + o], H2[s * NH + j], v);
            part[OFF_W3 + i] = v;
        } else {
            const int o = i - NO * NH;
            for (int s = 0; s < TM; ++s) v += DY[s * NO + o];
            part[OFF_B3 + o] = v;
        }
    }
    __syncthreads();     // h2 is overwritten by dz2 below
    // dz2 = (dy W3) * gelu'(z2), as BF16 in both layouts; db2 = sum_s dz2 (FP32)
    for (int i = threadIdx.x; i < TM * NH; i += kThreads) {
        const int s = i / NH, j = i - s * NH;
        float dh = 0.f;
#pragma unroll
        for (int o = 0; o < NO; ++o) dh = fmaf(DY[s * NO + o], W3[o * NH + j], dh);
        const float dz = dh * gelu_grad(Z2[i]);
        reinterpret_cast<float*>(sm + Smem::H2)[i] = dz;       // h2 no longer needed: keep dz2 in FP32
        const bf16 b = __float2bfloat16_rn(dz);
        DZ2[i] = b;
        DZ2T[j * TM + s] = b;
    }
    __syncthreads();
    const float* DZ2F = reinterpret_cast<const float*>(sm + Smem::H2);
    if (threadIdx.x < NH) {
        float v = 0.f;
        for (int s = 0; s < TM; ++s) v += DZ2F[s * NH + threadIdx.x];
        part[OFF_B2 + threadIdx.x] = v;
    }
    // dh1 = dz2 W2 (B = W2^T as [N][K]); dz1 = dh1 * gelu'(z1) -> DZ1T; db1 partials
    {
        const bf16* W2T = reinterpret_cast<const bf16*>(sm + Smem::W2T);
        float acc[NH / 8][4];
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        warp_gemm<NH, NH>(DZ2, NH, warp * 16, W2T, NH, acc);
        float* DZ1F = reinterpret_cast<float*>(sm + Smem::Z2);   // z2 no longer needed
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = warp * 16 + g + (h >> 1) * 8, c = nt * 8 + 2 * t + (h & 1);
                const float dz = acc[nt][h] * gelu_grad(Z1[r * NH + c]);
                DZ1F[r * NH + c] = dz;
                DZ1T[c * TM + r] = __float2bfloat16_rn(dz);
            }
    }
    __syncthreads();
    if (threadIdx.x < NH) {
        const float* DZ1F = reinterpret_cast<const float*>(sm + Smem::Z2);
        float v = 0.f;
        for (int s = 0; s < TM; ++s) v += DZ1F[s * NH + threadIdx.x];
        part[OFF_B1 + threadIdx.x] = v;
    }
    // dW2 = dz2^T h1: A = dz2^T [64][TM], B = h1^T as [N=64][K=TM]
    {
        const bf16* H1T = reinterpret_cast<const bf16*>(sm + Smem::H1T);
        float acc[NH / 8][4];
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        warp_gemm<NH, TM>(DZ2T, TM, warp * 16, H1T, TM, acc);
#pragma unroll
        for (int nt = 0; nt < NH / 8; ++nt)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = warp * 16 + g + (h >> 1) * 8, c = nt * 8 + 2 * t + (h & 1);
                part[OFF_W2 + r * NH + c] = acc[nt][h];
            }
    }
    // dW1 = dz1^T X: A = dz1^T [64][TM], B = X^T as [N=KP][K=TM]; keep the first NF columns
    {
        const bf16* XT = reinterpret_cast<const bf16*>(sm + Smem::XT);
        float acc[KP / 8][4];
#pragma unroll
        for (int nt = 0; nt < KP / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
        warp_gemm<KP, TM>(DZ1T, TM, warp * 16, XT, TM, acc);
#pragma unroll
        for (int nt = 0; nt < KP / 8; ++nt)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = warp * 16 + g + (h >> 1) * 8, c = nt * 8 + 2 * t + (h & 1);
                if (c < NF) part[OFF_W1 + r * NF + c] = acc[nt][h];
            }
    }
}

// ---- kernels --------------------------------------------------------------------

// Explicit batch: X [B][NF] FP32 (row-major), targets T [B][NO].
__global__ void __launch_bounds__(kThreads) mlp_train_kernel(MlpDev w, const float* __restrict__ X,
                                                             const float* __restrict__ T, int B,
                                                             float* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int s0 = blockIdx.x * TM;
    const int ns = min(TM, B - s0);
    load_weights(sm, w);
    gather_tile(sm, ns, true, [&](int s, int f) { return X[static_cast<size_t>(s0 + s) * NF + f]; });
    float* TG = reinterpret_cast<float*>(sm + Smem::TGT);
    for (int i = threadIdx.x; i < TM * NO; i += kThreads)
        TG[i] = (i / NO < ns) ? T[static_cast<size_t>(s0) * NO + i] : 0.f;
    __syncthreads();
    forward_tile(sm, true);
    backward_tile(sm, ns, 1.f / static_cast<float>(B), parts + static_cast<size_t>(blockIdx.x) * (NPARAM + 1));
}

__global__ void __launch_bounds__(kThreads) mlp_forward_kernel(MlpDev w, const float* __restrict__ X,
                                                               int B, float* __restrict__ Yout) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int s0 = blockIdx.x * TM;
    const int ns = min(TM, B - s0);
    load_weights(sm, w);
    gather_tile(sm, ns, false, [&](int s, int f) { return X[static_cast<size_t>(s0 + s) * NF + f]; });
    __syncthreads();
    forward_tile(sm, false);
    const float* Y = reinterpret_cast<const float*>(sm + Smem::Y);
    for (int i = threadIdx.x; i < ns * NO; i += kThreads) Yout[static_cast<size_t>(s0) * NO + i] = Y[i];
}

// Training samples from a slope sequence S [nframes][2 nv]: sample (i, k) uses frames
// k..k-3 as features and (S[k+1] - S[k]) / sigma of subaperture i as the target.
__global__ void __launch_bounds__(kThreads) mlp_train_seq_kernel(MlpDev w, const float* __restrict__ S,
                                                                 int n_frames, int nv,
                                                                 const int* __restrict__ nbr,
                                                                 const int2* __restrict__ samples, int B,
                                                                 float inv_sigma, float* __restrict__ parts) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int s0 = blockIdx.x * TM;
    const int ns = min(TM, B - s0);
    load_weights(sm, w);
    const size_t row = 2 * static_cast<size_t>(nv);
    // a sample outside the sequence or the pupil contributes zero features and target
    auto valid = [&](int2 sk) { return sk.x >= 0 && sk.x < nv && sk.y >= 3 && sk.y <= n_frames - 2; };
    int2* samp = reinterpret_cast<int2*>(sm + Smem::SAMP);
    for (int si = threadIdx.x; si < TM; si += kThreads) {
        const int2 sk = si < ns ? samples[s0 + si] : make_int2(-1, 0);
        samp[si] = valid(sk) ? sk : make_int2(-1, 0);
    }
    __syncthreads();
    gather_pairs(sm, true, nbr, nv, inv_sigma, [&](int si) { return samp[si].x; },
                 [&](int si, int lag) { return S + static_cast<size_t>(samp[si].y - lag) * row; });
    float* TG = reinterpret_cast<float*>(sm + Smem::TGT);
    for (int q = threadIdx.x; q < TM * NO; q += kThreads) {
        const int s = q / NO, o = q - s * NO;
        float v = 0.f;
        if (s < ns) {
            const int2 sk = samples[s0 + s];
            if (valid(sk))
                v = (S[(sk.y + 1) * row + o * nv + sk.x] - S[sk.y * row + o * nv + sk.x]) * inv_sigma;
        }
        TG[q] = v;
    }
    __syncthreads();
    forward_tile(sm, true);
    backward_tile(sm, ns, 1.f / static_cast<float>(B), parts + static_cast<size_t>(blockIdx.x) * (NPARAM + 1));
}

// Predicted next slopes of every subaperture from the 4 newest rows of a history
// ring: s_pred = s_k + sigma * y (x block then y block).
__global__ void __launch_bounds__(kThreads) mlp_predict_kernel(MlpDev w, const float* __restrict__ ring,
                                                               int kpad, int head, int nv,
                                                               const int* __restrict__ nbr, float sigma,
                                                               float* __restrict__ s_pred) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int s0 = blockIdx.x * TM;
    const int ns = min(TM, nv - s0);
    load_weights(sm, w);
    const float* rows[4];
    for (int lag = 0; lag < 4; ++lag) rows[lag] = ring + static_cast<size_t>((head - lag + 4) & 3) * kpad;
    gather_pairs(sm, false, nbr, nv, 1.f / sigma, [&](int si) { return si < ns ? s0 + si : -1; },
                 [&](int, int lag) { return rows[lag]; });
    __syncthreads();
    forward_tile(sm, false);
    const float* Y = reinterpret_cast<const float*>(sm + Smem::Y);
    for (int q = threadIdx.x; q < ns * NO; q += kThreads) {
        const int s = q / NO, o = q - s * NO;
        const int idx = o * nv + s0 + s;
        s_pred[idx] = __fmaf_rn(sigma, Y[q], rows[0][idx]);
    }
}

// Sum of the CTA partials in a fixed pairwise order, then (when lr > 0) one Adam step
// on the FP32 master weights and a refresh of the BF16 copies.  grad_out (optional)
// receives the summed gradient; loss_out (optional) the loss sum / (2B).
__global__ void mlp_update_kernel(MlpDev w, const float* __restrict__ parts, int nparts, float inv_2b,
                                  float lr, float beta1, float beta2, float eps, float bc1, float bc2,
                                  float* __restrict__ grad_out, float* __restrict__ loss_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NPARAM) return;
    float v[64];
    float g = 0.f;
    // pairwise tree over the partials, 64 at a time
    for (int c0 = 0; c0 < nparts; c0 += 64) {
        const int n = min(64, nparts - c0);
        for (int c = 0; c < n; ++c) v[c] = parts[static_cast<size_t>(c0 + c) * (NPARAM + 1) + p];
        for (int width = 1; width < n; width <<= 1)
            for (int i = 0; i + width < n; i += 2 * width) v[i] += v[i + width];
        g += v[0];
    }
    if (p == NPARAM) {
        if (loss_out) *loss_out = g * inv_2b;
        return;
    }
    if (grad_out) grad_out[p] = g;
    if (lr > 0.f) {
        const float m = beta1 * w.m[p] + (1.f - beta1) * g;
        const float s = beta2 * w.v[p] + (1.f - beta2) * g * g;
        w.m[p] = m;
        w.v[p] = s;
        const float mh = m / bc1, vh = s / bc2;
        const float np = w.master[p] - lr * mh / (sqrtf(vh) + eps);
        w.master[p] = np;
        if (p < OFF_B1) {
            const int r = p / NF, c = p - r * NF;
            w.w1_bf16[r * KP + c] = __float2bfloat16_rn(np);
        } else if (p >= OFF_W2 && p < OFF_B2) {
            w.w2_bf16[p - OFF_W2] = __float2bfloat16_rn(np);
        }
    }
}

__global__ void mlp_refresh_kernel(MlpDev w) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NH * KP) {
        const int r = p / KP, c = p - r * KP;
        w.w1_bf16[p] = __float2bfloat16_rn(c < NF ? w.master[OFF_W1 + r * NF + c] : 0.f);
    }
    if (p < NH * NH) w.w2_bf16[p] = __float2bfloat16_rn(w.master[OFF_W2 + p]);
}

}  // namespace

size_t mlp_smem_bytes() { return Smem::TOTAL; }

cudaError_t mlp_configure() {
    const int b = static_cast<int>(Smem::TOTAL);
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_train_seq_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_predict_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
    return e;
}

cudaError_t mlp_launch_refresh(const MlpDev& w, cudaStream_t st) {
    mlp_refresh_kernel<<<(NH * KP + 255) / 256, 256, 0, st>>>(w);
    return cudaGetLastError();
}

cudaError_t mlp_launch_train(const MlpDev& w, const float* X, const float* T, int B, float* parts,
                             cudaStream_t st) {
    mlp_train_kernel<<<(B + TM - 1) / TM, kThreads, Smem::TOTAL, st>>>(w, X, T, B, parts);
    return cudaGetLastError();
}

cudaError_t mlp_launch_train_seq(const MlpDev& w, const float* S, int n_frames, int nv,
                                 const int* nbr, const int2* samples, int B, float inv_sigma,
                                 float* parts, cudaStream_t st) {
    mlp_train_seq_kernel<<<(B + TM - 1) / TM, kThreads, Smem::TOTAL, st>>>(w, S, n_frames, nv, nbr,
                                                                           samples, B, inv_sigma, parts);
    return cudaGetLastError();
}

cudaError_t mlp_launch_forward(const MlpDev& w, const float* X, int B, float* Y, cudaStream_t st) {
    mlp_forward_kernel<<<(B + TM - 1) / TM, kThreads, Smem::TOTAL, st>>>(w, X, B, Y);
    return cudaGetLastError();
}

cudaError_t mlp_launch_predict(const MlpDev& w, const float* ring, int kpad, int head, int nv,
                               const int* nbr, float sigma, float* s_pred, cudaStream_t st) {
    if (nv == 0) return cudaSuccess;
    mlp_predict_kernel<<<(nv + TM - 1) / TM, kThreads, Smem::TOTAL, st>>>(w, ring, kpad, head, nv, nbr,
                                                                         sigma, s_pred);
    return cudaGetLastError();
}

cudaError_t mlp_launch_update(const MlpDev& w, const float* parts, int nparts, int B, float lr,
                              float beta1, float beta2, float eps, int step, float* grad_out,
                              float* loss_out, cudaStream_t st) {
    const float bc1 = 1.f - powf(beta1, static_cast<float>(step));
    const float bc2 = 1.f - powf(beta2, static_cast<float>(step));
    mlp_update_kernel<<<(NPARAM + 1 + 127) / 128, 128, 0, st>>>(w, parts, nparts, 0.5f / B, lr, beta1,
                                                               beta2, eps, bc1, bc2, grad_out, loss_out);
    return cudaGetLastError();
}
