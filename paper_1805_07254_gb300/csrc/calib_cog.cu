// Pixel calibration, centre-of-gravity centroiding and slope packing
// (Sec. 2.1, Fig. 3 (a) and (b)).
//
// One warp per valid subaperture (of one WFS).  The stage is latency-bound (a
// 740x740 frame plus its calibration data is ~4 MB), so every lane issues all of
// its loads -- raw pixels from the frame, dark and gain values from the
// subap-major calibration arrays -- before any arithmetic, and the whole frame
// costs about one HBM round trip.  Each lane then calibrates its pixels
//     p = (raw - dark) * gain,   gain = 1/flat,
// applies the threshold (the comparison on the FP32 value), and accumulates the
// flux and the two first moments about the box centre c = (npx-1)/2 with
// compensated (TwoSum) FP32 sums, reduced across the warp by a fixed xor
// butterfly.  Lane 0 writes
//     s[i] = Sx/F,  s[n_valid + i] = Sy/F   (0 when F <= 0),
// the x-then-y order of the Fig. 3 caption (per WFS block).
//
// Dark and gain are kept per valid subaperture, contiguous (subap-major
// [n_valid][npx*npx]), so their loads are coalesced and only valid pixels are
// read.

#include "rtc_internal.h"

namespace {

constexpr int kWarpsPerBlock = kCalibThreads / 32;
constexpr int kPixPerLane = 8;          // loads in flight per lane per pass (npx <= 16 in one pass)

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

// NPX > 0: box size known at compile time (divisions by constants, exact unrolling);
// NPX == 0: any box size, given at run time.
template <int NPX>
__global__ void __launch_bounds__(kCalibThreads)
calib_cog_kernel(const uint16_t* __restrict__ frame, int side, int npx_rt, int n_valid, int n_wfs,
                 const int2* __restrict__ rc, const float* __restrict__ dark,
                 const float* __restrict__ gainmap, int thr_mode, float thr,
                 float* __restrict__ s_out) {
    constexpr int kJ = NPX > 0 ? (NPX * NPX + 31) / 32 : kPixPerLane;
    const int npx = NPX > 0 ? NPX : npx_rt;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (gw >= n_valid * n_wfs) return;
    const int w = gw / n_valid;
    const int i = gw - w * n_valid;
    const int2 pos = rc[i];                                  // (row, col) on the grid
    const int npp = npx * npx;
    const float cc = 0.5f * static_cast<float>(npx - 1);
    const uint16_t* box = frame + static_cast<size_t>(w) * side * side +
                          static_cast<size_t>(pos.x) * npx * side + static_cast<size_t>(pos.y) * npx;
    const size_t base = (static_cast<size_t>(w) * n_valid + i) * npp;
    const float* dk = dark + base;
    const float* gk = gainmap + base;

    CompSum F{0.f, 0.f}, Sx{0.f, 0.f}, Sy{0.f, 0.f};
    for (int q0 = 0; q0 < npp; q0 += 32 * kJ) {
        float raw[kJ], dv[kJ], gv[kJ];
        int xs[kJ], ys[kJ];
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int q = q0 + lane + 32 * j;
            ys[j] = q / npx;
            xs[j] = q - ys[j] * npx;
            if (q < npp) {
                raw[j] = static_cast<float>(__ldg(box + ys[j] * side + xs[j]));
                dv[j] = __ldg(dk + q);
                gv[j] = __ldg(gk + q);
            }
        }
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            if (q0 + lane + 32 * j < npp) {
                float p = __fmul_rn(__fsub_rn(raw[j], dv[j]), gv[j]);
                if (thr_mode == 0) {
                    p = (p < thr) ? 0.f : p;
                } else {
                    p = (p > thr) ? __fsub_rn(p, thr) : 0.f;
                }
                comp_add(F, p);
                comp_add(Sx, __fmul_rn(p, static_cast<float>(xs[j]) - cc));
                comp_add(Sy, __fmul_rn(p, static_cast<float>(ys[j]) - cc));
            }
        }
    }
    comp_warp_reduce(F);
    comp_warp_reduce(Sx);
    comp_warp_reduce(Sy);
    if (lane == 0) {
        const float f = F.s + F.c;
        const float sx = Sx.s + Sx.c;
        const float sy = Sy.s + Sy.c;
        const bool ok = f > 0.f;
        float* s_w = s_out + static_cast<size_t>(w) * 2 * n_valid;
        s_w[i] = ok ? sx / f : 0.f;
        s_w[n_valid + i] = ok ? sy / f : 0.f;
    }
}

}  // namespace

cudaError_t launch_calib_cog(const rtc_handle* h, const uint16_t* d_frame, float* d_s,
                             cudaStream_t st) {
    const int warps = h->n_valid * h->cfg.n_wfs;
    if (warps == 0) return cudaSuccess;
    const int blocks = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
#define RTC_CALIB_ARGS                                                                           \
    d_frame, h->side, h->cfg.npx, h->n_valid, h->cfg.n_wfs, h->d_rc, h->d_dark, h->d_gainmap, \
        h->thr_mode, h->thr, d_s
    switch (h->cfg.npx) {
        case 8: calib_cog_kernel<8><<<blocks, kCalibThreads, 0, st>>>(RTC_CALIB_ARGS); break;
        case 10: calib_cog_kernel<10><<<blocks, kCalibThreads, 0, st>>>(RTC_CALIB_ARGS); break;
        case 16: calib_cog_kernel<16><<<blocks, kCalibThreads, 0, st>>>(RTC_CALIB_ARGS); break;
        default: calib_cog_kernel<0><<<blocks, kCalibThreads, 0, st>>>(RTC_CALIB_ARGS); break;
    }
#undef RTC_CALIB_ARGS
    return cudaGetLastError();
}
