// Load-time storage of the control matrix in the handle's slice-major layout, and
// the row-major split-K reconstruction of the allocation-free entry point.
//
// Split-K MVM (rtc_mvm_integrate_noalloc, on caller buffers [nact][kpad]): the
// MVM is bound by the bytes of M it streams from HBM (Sec. 1.1.1), so it runs on
// CUDA cores as a split-K GEMV:
//   - block (rb, ks) multiplies rows [4 rb, 4 rb + 4) over the ks-th K slice;
//     thread t takes the 16-byte chunks t, t+256, ... of the slice for all four
//     rows, so each s chunk (read through L1) serves four matrix chunks, and the
//     matrix is read with L1-bypassing non-coherent 16-byte loads;
//   - stored values are widened to FP32 just before the FMA (the widening dot
//     products of stream_mvm.cuh), as Sec. 2.3.4 widens its 16-bit matrix; the
//     FP8 and INT8 row scales are applied once, after the sum;
//   - partials are combined in a fixed order: xor butterfly within the warp,
//     a pairwise tree over the 8 warps, and, when K is split across blocks, a
//     pairwise tree over the ksplit block partials done by the last block to
//     finish that row group (arrival counter, self-resetting).  This is the GPU
//     form of the tree-like partial DM vector addition of Sec. 2.3.5, and the
//     result does not depend on block scheduling.

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "rtc_internal.h"
#include "stream_mvm.cuh"

namespace {

__device__ __forceinline__ uint4 ld_stream(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

using rtc_mvm::Esize;
using rtc_mvm::RowScaled;
using rtc_mvm::word_dot;

// Elements of the stored type per 16-byte chunk.
template <int DT> struct Epc { static constexpr int v = 16 / Esize<DT>::v; };

// acc += <16-byte chunk m, its Epc slopes sv>, word by word.
template <int DT>
__device__ __forceinline__ float chunk_dot(float acc, const uint4& m, const float* sv) {
    constexpr int EPW = 4 / Esize<DT>::v;
    acc = word_dot<DT>(acc, m.x, sv);
    acc = word_dot<DT>(acc, m.y, sv + EPW);
    acc = word_dot<DT>(acc, m.z, sv + 2 * EPW);
    return word_dot<DT>(acc, m.w, sv + 3 * EPW);
}

template <int DT>
__device__ __forceinline__ void load_s(const float* __restrict__ s, int chunk, float* sv) {
    const float4* p = reinterpret_cast<const float4*>(s) + chunk * (Epc<DT>::v / 4);
#pragma unroll
    for (int j = 0; j < Epc<DT>::v / 4; ++j) {
        const float4 v = __ldg(p + j);
        sv[4 * j + 0] = v.x;
        sv[4 * j + 1] = v.y;
        sv[4 * j + 2] = v.z;
        sv[4 * j + 3] = v.w;
    }
}

// Fixed pairwise tree over v[0 .. n): ((v0+v1)+(v2+v3))+...
__device__ __forceinline__ float tree_sum(float* v, int n) {
    for (int width = 1; width < n; width <<= 1)
        for (int i = 0; i + width < n; i += 2 * width) v[i] += v[i + width];
    return v[0];
}

template <int DT, int U>
__global__ void __launch_bounds__(kMvmThreads)
mvm_splitk_kernel(const uint4* __restrict__ M, int chunks_per_row, int nact,
                  const float* __restrict__ s, const float* __restrict__ row_scale, int ksplit,
                  float* __restrict__ partial, unsigned* __restrict__ counter,
                  float* __restrict__ a, float* __restrict__ dm_out, float gain, float leak) {
    constexpr int R = kMvmRows;
    constexpr int NW = kMvmThreads / 32;
    constexpr int E = Epc<DT>::v;
    __shared__ float red[R][NW];
    __shared__ bool last_block;

    const int rb = blockIdx.x;
    const int ks = blockIdx.y;
    const int row0 = rb * R;
    const int c_begin = static_cast<int>((static_cast<long long>(ks) * chunks_per_row) / ksplit);
    const int c_end = static_cast<int>((static_cast<long long>(ks + 1) * chunks_per_row) / ksplit);

    const uint4* rowp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int rr = min(row0 + r, nact - 1);   // rows past nact re-read the last row; discarded
        rowp[r] = M + static_cast<size_t>(rr) * chunks_per_row;
    }

    float acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.f;

    int c = c_begin + threadIdx.x;
    for (; c + (U - 1) * kMvmThreads < c_end; c += U * kMvmThreads) {
        uint4 m[U][R];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int r = 0; r < R; ++r) m[u][r] = ld_stream(rowp[r] + c + u * kMvmThreads);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            float sv[E];
            load_s<DT>(s, c + u * kMvmThreads, sv);
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = chunk_dot<DT>(acc[r], m[u][r], sv);
        }
    }
    for (; c < c_end; c += kMvmThreads) {
        uint4 m[R];
#pragma unroll
        for (int r = 0; r < R; ++r) m[r] = ld_stream(rowp[r] + c);
        float sv[E];
        load_s<DT>(s, c, sv);
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = chunk_dot<DT>(acc[r], m[r], sv);
    }

    // warp butterfly, then a pairwise tree over the warps
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float v = acc[r];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (lane == 0) red[r][warp] = v;
    }
    __syncthreads();

    const int t = threadIdx.x;
    float d = 0.f;
    if (t < R) {
        float v[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) v[w] = red[t][w];
        d = tree_sum(v, NW);
    }

    if (ksplit > 1) {
        if (t < R && row0 + t < nact) partial[static_cast<size_t>(ks) * nact + row0 + t] = d;
        __threadfence();
        __syncthreads();
        if (t == 0) last_block = (atomicAdd(counter + rb, 1u) == static_cast<unsigned>(ksplit - 1));
        __syncthreads();
        if (!last_block) return;
        __threadfence();
        if (t < R && row0 + t < nact) {
            float v[kMaxKsplit];
            for (int k = 0; k < ksplit; ++k)
                v[k] = __ldcg(partial + static_cast<size_t>(k) * nact + row0 + t);
            d = tree_sum(v, ksplit);
        }
        if (t == 0) counter[rb] = 0u;
    }

    if (t < R && row0 + t < nact) {
        const int row = row0 + t;
        if (RowScaled<DT>::v) d *= row_scale[row];
        const float an = fmaf(leak, a[row], gain * d);
        a[row] = an;
        if (dm_out) dm_out[row] = an;
    }
}

// --- load-time layout ------------------------------------------------------------

// Code of x / sc in the row-scaled formats (one correctly rounded FP32 division).
template <int DT>
__device__ __forceinline__ unsigned char encode_scaled(float x, float sc) {
    const float q = __fdiv_rn(x, sc);
    if (DT == RTC_FP8_E4M3) return __nv_cvt_float_to_fp8(q, __NV_SATFINITE, __NV_E4M3);
    const int i = max(-127, min(127, __float2int_rn(q)));       // nearest, ties to even
    return static_cast<unsigned char>(static_cast<signed char>(i));
}

// Per-row scale = max |M_r| / qmax (1 for a zero row), one block per row.
template <int DT>
__global__ void row_scale_kernel(const float* __restrict__ src, int ncol, float* __restrict__ scale) {
    constexpr float qmax = DT == RTC_FP8_E4M3 ? 448.0f : 127.0f;
    __shared__ float wmax[32];
    const int row = blockIdx.x;
    const float* in = src + static_cast<size_t>(row) * ncol;
    float m = 0.f;
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) m = fmaxf(m, fabsf(in[j]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float mm = 0.f;
        for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) mm = fmaxf(mm, wmax[w]);
        scale[row] = mm > 0.f ? __fdiv_rn(mm, qmax) : 1.0f;
    }
}

// One row per block: FP32 column c -> its slice's row in the stored type.
template <int DT>
__global__ void layout_f32_kernel(const float* __restrict__ src, int ncol, const int2* __restrict__ colmap,
                                  const long long* __restrict__ off, const int* __restrict__ rowbytes, int plane,
                                  const float* __restrict__ scale, unsigned char* __restrict__ dst) {
    const int row = blockIdx.x, nact = gridDim.x;
    const float sc = RowScaled<DT>::v ? scale[row] : 1.f;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const int2 sj = colmap[c];
        unsigned char* p =
            dst + rtc_mvm::slice_elem_offset(off[sj.x], rowbytes[sj.x], nact, row, sj.y * Esize<DT>::v, plane);
        const float v = src[static_cast<size_t>(row) * ncol + c];
        if (DT == RTC_F32) *reinterpret_cast<float*>(p) = v;
        else if (DT == RTC_BF16) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
        else if (DT == RTC_F16) *reinterpret_cast<__half*>(p) = __float2half_rn(v);
        else *p = encode_scaled<DT>(v, sc);
    }
}

// One row per block: an element of esize bytes, already in the stored type.
__global__ void layout_raw_kernel(const unsigned char* __restrict__ src, int ncol, int esize,
                                  const int2* __restrict__ colmap, const long long* __restrict__ off,
                                  const int* __restrict__ rowbytes, int plane, unsigned char* __restrict__ dst) {
    const int row = blockIdx.x, nact = gridDim.x;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const int2 sj = colmap[c];
        unsigned char* p = dst + rtc_mvm::slice_elem_offset(off[sj.x], rowbytes[sj.x], nact, row, sj.y * esize, plane);
        const unsigned char* q = src + (static_cast<size_t>(row) * ncol + c) * esize;
        for (int b = 0; b < esize; ++b) p[b] = q[b];
    }
}

__global__ void relayout_kernel(const unsigned char* __restrict__ src, const int2* __restrict__ src_map,
                                const long long* __restrict__ src_off, const int* __restrict__ src_rb,
                                int ncol, int esize, int src_plane, int dst_plane, const int2* __restrict__ dst_map,
                                const long long* __restrict__ dst_off, const int* __restrict__ dst_rb,
                                unsigned char* __restrict__ dst) {
    const int row = blockIdx.x, nact = gridDim.x;
    for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
        const int2 a = src_map[c], b = dst_map[c];
        const unsigned char* q =
            src + rtc_mvm::slice_elem_offset(src_off[a.x], src_rb[a.x], nact, row, a.y * esize, src_plane);
        unsigned char* p =
            dst + rtc_mvm::slice_elem_offset(dst_off[b.x], dst_rb[b.x], nact, row, b.y * esize, dst_plane);
        for (int k = 0; k < esize; ++k) p[k] = q[k];
    }
}

template <int DT>
void launch_raw_t(dim3 grid, const uint4* M, int kpad, int nact, const float* d_s, const float* d_scale,
                  int ksplit, float* d_partial, unsigned* d_count, float* d_a, float* d_dm_out,
                  float gain, float leak, cudaStream_t st) {
    mvm_splitk_kernel<DT, 2><<<grid, kMvmThreads, 0, st>>>(M, kpad / Epc<DT>::v, nact, d_s, d_scale, ksplit,
                                                           d_partial, d_count, d_a, d_dm_out, gain, leak);
}

}  // namespace

cudaError_t launch_mvm_raw(int store, const void* d_M, const float* d_scale, int nact, int kpad,
                           const float* d_s, int ksplit, float* d_partial, unsigned* d_count,
                           float* d_a, float* d_dm_out, float gain, float leak, cudaStream_t st) {
    dim3 grid((nact + kMvmRows - 1) / kMvmRows, ksplit);
    const uint4* M = static_cast<const uint4*>(d_M);
    switch (store) {
        case RTC_F32:
            launch_raw_t<RTC_F32>(grid, M, kpad, nact, d_s, d_scale, ksplit, d_partial, d_count, d_a, d_dm_out, gain, leak, st);
            break;
        case RTC_BF16:
            launch_raw_t<RTC_BF16>(grid, M, kpad, nact, d_s, d_scale, ksplit, d_partial, d_count, d_a, d_dm_out, gain, leak, st);
            break;
        case RTC_F16:
            launch_raw_t<RTC_F16>(grid, M, kpad, nact, d_s, d_scale, ksplit, d_partial, d_count, d_a, d_dm_out, gain, leak, st);
            break;
        case RTC_FP8_E4M3:
            launch_raw_t<RTC_FP8_E4M3>(grid, M, kpad, nact, d_s, d_scale, ksplit, d_partial, d_count, d_a, d_dm_out, gain, leak, st);
            break;
        case RTC_INT8:
            launch_raw_t<RTC_INT8>(grid, M, kpad, nact, d_s, d_scale, ksplit, d_partial, d_count, d_a, d_dm_out, gain, leak, st);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_layout(int src, int store, const void* d_src, int nact, int ncol,
                          const int2* d_colmap, const long long* d_off, const int* d_rowbytes, int plane,
                          float* d_scale, void* d_dst, cudaStream_t st) {
    if (nact <= 0 || ncol <= 0) return cudaSuccess;
    unsigned char* dst = static_cast<unsigned char*>(d_dst);
    if (src == store) {
        const int esize = store == RTC_F32 ? 4 : (store == RTC_BF16 || store == RTC_F16) ? 2 : 1;
        layout_raw_kernel<<<nact, 256, 0, st>>>(static_cast<const unsigned char*>(d_src), ncol, esize,
                                                d_colmap, d_off, d_rowbytes, plane, dst);
        return cudaGetLastError();
    }
    if (src != RTC_F32) return cudaErrorInvalidValue;
    const float* f = static_cast<const float*>(d_src);
    switch (store) {
        case RTC_BF16:
            layout_f32_kernel<RTC_BF16><<<nact, 256, 0, st>>>(f, ncol, d_colmap, d_off, d_rowbytes, plane, d_scale, dst);
            break;
        case RTC_F16:
            layout_f32_kernel<RTC_F16><<<nact, 256, 0, st>>>(f, ncol, d_colmap, d_off, d_rowbytes, plane, d_scale, dst);
            break;
        case RTC_FP8_E4M3:
            row_scale_kernel<RTC_FP8_E4M3><<<nact, 256, 0, st>>>(f, ncol, d_scale);
            layout_f32_kernel<RTC_FP8_E4M3><<<nact, 256, 0, st>>>(f, ncol, d_colmap, d_off, d_rowbytes, plane, d_scale, dst);
            break;
        case RTC_INT8:
            row_scale_kernel<RTC_INT8><<<nact, 256, 0, st>>>(f, ncol, d_scale);
            layout_f32_kernel<RTC_INT8><<<nact, 256, 0, st>>>(f, ncol, d_colmap, d_off, d_rowbytes, plane, d_scale, dst);
            break;
        default:
            return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_relayout(int esize, int old_plane, int new_plane, const void* d_old, const int2* d_old_colmap,
                            const long long* d_old_off, const int* d_old_rowbytes, int nact, int ncol,
                            const int2* d_new_colmap, const long long* d_new_off, const int* d_new_rowbytes,
                            void* d_new, cudaStream_t st) {
    if (nact <= 0 || ncol <= 0) return cudaSuccess;
    relayout_kernel<<<nact, 256, 0, st>>>(static_cast<const unsigned char*>(d_old), d_old_colmap, d_old_off,
                                          d_old_rowbytes, ncol, esize, old_plane, new_plane, d_new_colmap, d_new_off,
                                          d_new_rowbytes, static_cast<unsigned char*>(d_new));
    return cudaGetLastError();
}
