// Stand-alone pixel stage: calibration, centre of gravity and slope packing for
// every valid subaperture of every WFS (Sec. 2.1, Fig. 3 (a)-(b)); one warp per
// subaperture (see pixel.cuh).  The fused frame kernel runs the same device code.

#include "pixel.cuh"

namespace {

constexpr int kWarpsPerBlock = kCalibThreads / 32;

template <int NPX>
__global__ void __launch_bounds__(kCalibThreads) calib_cog_kernel(rtc_pixel::PixelArgs p) {
    const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
    if (gw >= p.n_valid * p.n_wfs) return;
    rtc_pixel::subap_slopes<NPX, rtc_pixel::kPixelReadOnly, 32>(p, p.frame, p.s, gw, true,
                                                                threadIdx.x & 31);
}

}  // namespace

rtc_pixel::PixelArgs pixel_args(const rtc_handle* h, const uint16_t* d_frame, float* d_s) {
    return rtc_pixel::PixelArgs{d_frame,    h->side,     h->cfg.npx, h->n_valid, h->cfg.n_wfs,
                                h->d_rc,    h->d_dark,   h->d_gainmap, h->thr_mode, h->thr, d_s};
}

cudaError_t launch_calib_cog(const rtc_handle* h, const uint16_t* d_frame, float* d_s,
                             cudaStream_t st) {
    const int warps = h->n_valid * h->cfg.n_wfs;
    if (warps == 0) return cudaSuccess;
    const int blocks = (warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
    const rtc_pixel::PixelArgs p = pixel_args(h, d_frame, d_s);
    switch (h->cfg.npx) {
        case 8: calib_cog_kernel<8><<<blocks, kCalibThreads, 0, st>>>(p); break;
        case 10: calib_cog_kernel<10><<<blocks, kCalibThreads, 0, st>>>(p); break;
        case 16: calib_cog_kernel<16><<<blocks, kCalibThreads, 0, st>>>(p); break;
        default: calib_cog_kernel<0><<<blocks, kCalibThreads, 0, st>>>(p); break;
    }
    return cudaGetLastError();
}
