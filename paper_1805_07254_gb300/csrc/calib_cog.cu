// Pixel calibration, centre-of-gravity centroiding and slope packing
// (Sec. 2.1, Fig. 3 (a) and (b)).
//
// One block per (subaperture row, WFS).  The block stages the row's band of
// npx detector rows (npx * side uint16 pixels, contiguous in the frame) into
// shared memory with 16-byte loads, then each warp takes one valid
// subaperture of the band at a time: it calibrates the npx*npx pixels
//     p = (raw - dark) * gain,   gain = 1/flat,
// applies the threshold, and forms the flux and the two first moments about
// the box centre c = (npx-1)/2 with compensated (TwoSum) FP32 accumulation,
// reduced across the warp by a fixed xor butterfly.  Lane 0 writes
//     s[i] = Sx/F,  s[n_valid + i] = Sy/F   (0 when F <= 0),
// the x-then-y order of the Fig. 3 caption.
//
// Dark and gain values are kept per valid subaperture, contiguous
// (subap-major [n_valid][npx*npx]), so their loads are coalesced and only
// valid pixels are read.

#include "rtc_internal.h"

namespace {

struct CompSum {
    float s, c;
};

// TwoSum accumulation: the rounding error of every addition is kept in c.
__device__ __forceinline__ void comp_add(CompSum& a, float v) {
    float t = __fadd_rn(a.s, v);
    float bp = __fsub_rn(t, a.s);
    float e = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(v, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, e);
}

__device__ __forceinline__ void comp_warp_reduce(CompSum& a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        float os = __shfl_xor_sync(0xffffffffu, a.s, off);
        float oc = __shfl_xor_sync(0xffffffffu, a.c, off);
        a.c = __fadd_rn(a.c, oc);
        comp_add(a, os);
    }
}

// Copy n uint16 values from global src to shared memory, 16 bytes at a time
// where the source is aligned.  Returns the shared-memory address at which
// element 0 landed (shifted so that the aligned part stays aligned).
__device__ __forceinline__ const uint16_t* stage_band(const uint16_t* __restrict__ src, int n,
                                                      unsigned char* smem) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(src);
    const int shift = static_cast<int>(a & 15);          // bytes past the previous 16-B line
    uint16_t* dst = reinterpret_cast<uint16_t*>(smem + shift);
    int head = ((16 - shift) & 15) >> 1;                 // elements until src is 16-B aligned
    if (head > n) head = n;
    const int nvec = (n - head) >> 3;
    for (int q = threadIdx.x; q < head; q += blockDim.x) dst[q] = src[q];
    const uint4* vs = reinterpret_cast<const uint4*>(src + head);
    uint4* vd = reinterpret_cast<uint4*>(dst + head);
    for (int q = threadIdx.x; q < nvec; q += blockDim.x) vd[q] = __ldg(vs + q);
    for (int q = head + 8 * nvec + threadIdx.x; q < n; q += blockDim.x) dst[q] = src[q];
    return dst;
}

__global__ void __launch_bounds__(kCalibThreads)
calib_cog_kernel(const uint16_t* __restrict__ frame, int side, int npx, int n_valid,
                 const int32_t* __restrict__ bands, const int32_t* __restrict__ subcol,
                 const float* __restrict__ dark, const float* __restrict__ gainmap,
                 int thr_mode, float thr, float* __restrict__ s_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.x;
    const int w = blockIdx.y;
    const int row = bands[3 * b + 0];
    const int first = bands[3 * b + 1];
    const int count = bands[3 * b + 2];
    const size_t plane = static_cast<size_t>(side) * side;
    const uint16_t* src = frame + w * plane + static_cast<size_t>(row) * npx * side;
    const uint16_t* px = stage_band(src, npx * side, smem);
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int npp = npx * npx;
    const float cc = 0.5f * static_cast<float>(npx - 1);
    float* s_w = s_out + static_cast<size_t>(w) * 2 * n_valid;

    for (int k = warp; k < count; k += nwarps) {
        const int i = first + k;
        const int col0 = subcol[i] * npx;
        const size_t base = (static_cast<size_t>(w) * n_valid + i) * npp;
        const float* dk = dark + base;
        const float* gk = gainmap + base;
        CompSum F{0.f, 0.f}, Sx{0.f, 0.f}, Sy{0.f, 0.f};
        for (int q = lane; q < npp; q += 32) {
            const int y = q / npx;
            const int x = q - y * npx;
            const float raw = static_cast<float>(px[y * side + col0 + x]);
            float p = __fmul_rn(__fsub_rn(raw, __ldg(dk + q)), __ldg(gk + q));
            if (thr_mode == 0) {
                p = (p < thr) ? 0.f : p;
            } else {
                p = (p > thr) ? __fsub_rn(p, thr) : 0.f;
            }
            comp_add(F, p);
            comp_add(Sx, __fmul_rn(p, static_cast<float>(x) - cc));
            comp_add(Sy, __fmul_rn(p, static_cast<float>(y) - cc));
        }
        comp_warp_reduce(F);
        comp_warp_reduce(Sx);
        comp_warp_reduce(Sy);
        if (lane == 0) {
            const float f = F.s + F.c;
            const float sx = Sx.s + Sx.c;
            const float sy = Sy.s + Sy.c;
            const bool ok = f > 0.f;
            s_w[i] = ok ? sx / f : 0.f;
            s_w[n_valid + i] = ok ? sy / f : 0.f;
        }
    }
}

}  // namespace

size_t calib_cog_smem_bytes(const rtc_handle* h) {
    return static_cast<size_t>(h->cfg.npx) * h->side * sizeof(uint16_t) + 16;
}

cudaError_t calib_cog_configure(size_t smem_bytes) {
    return cudaFuncSetAttribute(calib_cog_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(smem_bytes));
}

cudaError_t launch_calib_cog(const rtc_handle* h, const uint16_t* d_frame, float* d_s,
                             cudaStream_t st) {
    if (h->nbands == 0) return cudaSuccess;
    dim3 grid(h->nbands, h->cfg.n_wfs);
    calib_cog_kernel<<<grid, kCalibThreads, calib_cog_smem_bytes(h), st>>>(
        d_frame, h->side, h->cfg.npx, h->n_valid, h->d_band, h->d_subcol, h->d_dark,
        h->d_gainmap, h->thr_mode, h->thr, d_s);
    return cudaGetLastError();
}
