// Device code of the pixel stage (Sec. 2.1, Fig. 3 (a)-(b)), shared by the
// stand-alone centroid kernel and the fused frame kernel.
//
// One warp takes one valid subaperture of one WFS.  The stage is latency-bound
// (a 740x740 frame plus its calibration data is ~4 MB), so every lane issues all
// of its loads -- raw pixels from the frame, dark and gain values from the
// subap-major calibration arrays -- before any arithmetic.  Each lane then
// calibrates its pixels
//     p = (raw - dark) * gain,   gain = 1/flat,
// applies the threshold (the comparison on the FP32 value), and accumulates the
// flux and the two first moments about the box centre c = (npx-1)/2 with
// compensated (TwoSum) FP32 sums, reduced across the warp by a fixed xor
// butterfly.  Lane 0 writes
//     s[i] = Sx/F,  s[n_valid + i] = Sy/F   (0 when F <= 0),
// the x-then-y order of the Fig. 3 caption (per WFS block).
#pragma once

#include "rtc_internal.h"

namespace rtc_pixel {

constexpr int kPixPerLane = 8;   // loads in flight per lane per pass for a run-time box size

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

// Reduce over aligned groups of L lanes (L = 16 or 32) with a fixed xor butterfly.
template <int L>
__device__ __forceinline__ void comp_group_reduce(CompSum& a) {
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) {
        float os = __shfl_xor_sync(0xffffffffu, a.s, off);
        float oc = __shfl_xor_sync(0xffffffffu, a.c, off);
        a.c = __fadd_rn(a.c, oc);
        comp_add(a, os);
    }
}

struct PixelArgs {
    const uint16_t* frame;   // [n_wfs][side][side]
    int side, npx, n_valid, n_wfs;
    const int2* rc;          // [n_valid] (row, col)
    const float* dark;       // [n_wfs][n_valid][npx*npx]
    const float* gainmap;    // [n_wfs][n_valid][npx*npx]
    int thr_mode;
    float thr;
    float* s;                // [n_wfs][2][n_valid]
};

// How raw pixels are read: through the read-only path (a frame that does not change
// while the kernel runs), fetched fresh every time (a frame buffer that a host
// producer rewrites while a persistent kernel keeps running), or through L2 (a
// device buffer that other blocks of the same kernel rewrite frame after frame).
enum PixelLoad { kPixelReadOnly = 0, kPixelVolatile = 1, kPixelL2 = 2 };

template <int LD>
__device__ __forceinline__ uint16_t load_pixel(const uint16_t* ptr) {
    if (LD == kPixelVolatile) return __ldcv(ptr);
    if (LD == kPixelL2) return __ldcg(ptr);
    return __ldg(ptr);
}

struct NoHook {
    __device__ void operator()() const {}
};

// Slopes of subaperture gi (= w * n_valid + i) by an aligned group of L lanes
// (L = 32: the whole warp; L = 16: each half-warp takes its own subaperture).
// Every lane of the warp must call it (the reductions shuffle across the warp);
// a group with valid == false computes nothing and writes nothing.
// NPX > 0: box size known at compile time; NPX == 0: p.npx at run time.
// frame and s_out: this frame's pixels and slope vector (PixelArgs' own fields are
// not used, so that a persistent kernel can switch buffers per frame cheaply).
// loaded(): called by every lane after each pass has issued its loads (the
// passes are the same for every lane, valid or not).  Returns (x, y) slopes on the
// group's first lane (zeros elsewhere).
//
// subap_slopes_at takes the subaperture's grid position (subap_pos) from the
// caller, who may have loaded it early; subap_slopes loads it itself.
__device__ __forceinline__ int2 subap_pos(const PixelArgs& p, int gi, bool valid) {
    const int w = valid ? gi / p.n_valid : 0;
    return valid ? p.rc[gi - w * p.n_valid] : make_int2(0, 0);
}

template <int NPX, int LD, int L, typename Hook = NoHook>
__device__ __forceinline__ float2 subap_slopes_at(const PixelArgs& p, const uint16_t* __restrict__ frame,
                                                float* __restrict__ s_out, int gi, bool valid, int lane,
                                                int2 pos, const Hook& loaded = Hook()) {
    constexpr int kJ = NPX > 0 ? (NPX * NPX + L - 1) / L : kPixPerLane;
    const int npx = NPX > 0 ? NPX : p.npx;
    const int l = lane & (L - 1);
    const int w = valid ? gi / p.n_valid : 0;
    const int i = valid ? gi - w * p.n_valid : 0;
    const int npp = npx * npx;
    const float cc = 0.5f * static_cast<float>(npx - 1);
    const uint16_t* box = frame + static_cast<size_t>(w) * p.side * p.side +
                          static_cast<size_t>(pos.x) * npx * p.side + static_cast<size_t>(pos.y) * npx;
    const size_t base = (static_cast<size_t>(w) * p.n_valid + i) * npp;
    const float* dk = p.dark + base;
    const float* gk = p.gainmap + base;

    CompSum F{0.f, 0.f}, Sx{0.f, 0.f}, Sy{0.f, 0.f};
    for (int q0 = 0; q0 < npp; q0 += L * kJ) {
        float raw[kJ], dv[kJ], gv[kJ];
        // the calibration data first: its addresses do not wait for the position
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int q = q0 + l + L * j;
            dv[j] = gv[j] = 0.f;
            if (valid && q < npp) {
                dv[j] = __ldg(dk + q);
                gv[j] = __ldg(gk + q);
            }
        }
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int q = q0 + l + L * j;
            raw[j] = 0.f;
            if (valid && q < npp) {
                const int y = q / npx;
                raw[j] = static_cast<float>(load_pixel<LD>(box + y * p.side + (q - y * npx)));
            }
        }
        loaded();
#pragma unroll
        for (int j = 0; j < kJ; ++j) {
            const int q = q0 + l + L * j;
            if (valid && q < npp) {
                const int y = q / npx;
                const int x = q - y * npx;
                float v = __fmul_rn(__fsub_rn(raw[j], dv[j]), gv[j]);
                if (p.thr_mode == 0) {
                    v = (v < p.thr) ? 0.f : v;
                } else {
                    v = (v > p.thr) ? __fsub_rn(v, p.thr) : 0.f;
                }
                comp_add(F, v);
                comp_add(Sx, __fmul_rn(v, static_cast<float>(x) - cc));
                comp_add(Sy, __fmul_rn(v, static_cast<float>(y) - cc));
            }
        }
    }
    comp_group_reduce<L>(F);
    comp_group_reduce<L>(Sx);
    comp_group_reduce<L>(Sy);
    float2 res = make_float2(0.f, 0.f);
    if (l == 0 && valid) {
        const float f = F.s + F.c;
        const float sx = Sx.s + Sx.c;
        const float sy = Sy.s + Sy.c;
        const bool ok = f > 0.f;
        res = make_float2(ok ? sx / f : 0.f, ok ? sy / f : 0.f);
        float* s_w = s_out + static_cast<size_t>(w) * 2 * p.n_valid;
        s_w[i] = res.x;
        s_w[p.n_valid + i] = res.y;
    }
    return res;
}

template <int NPX, int LD, int L, typename Hook = NoHook>
__device__ __forceinline__ float2 subap_slopes(const PixelArgs& p, const uint16_t* __restrict__ frame,
                                             float* __restrict__ s_out, int gi, bool valid, int lane,
                                             const Hook& loaded = Hook()) {
    return subap_slopes_at<NPX, LD, L>(p, frame, s_out, gi, valid, lane, subap_pos(p, gi, valid), loaded);
}

// ---- frame ingest from host memory ---------------------------------------------
// A block copies exactly the pixel rows its subapertures cover from a frame in
// mapped host memory into a device staging buffer, as a host-built, sorted list of
// copy units (16 bytes for ELT frames): every load in flight before the stores,
// bypassing the caches (the host rewrites its buffers between uses).  Two blocks may
// both copy a unit that straddles their subapertures; they write the same bytes.

// Units a thread keeps in registers (a persistent loop keeps them across frames); a
// block with more than kUnitRegs * NT units reads the rest from the table.
constexpr int kUnitRegs = 2;
constexpr unsigned kNoUnit = ~0u;

// The block's copy units of one frame: host frame -> staging, all loads issued
// before the stores.  NT threads take part; ur: the thread's first units (kNoUnit
// for none), fo: its first unit beyond them, f1: the block's end.
template <typename V, int NT>
__device__ __forceinline__ void copy_units(const uint16_t* frame, uint16_t* stage, const unsigned* units,
                                           int f1, const unsigned (&ur)[kUnitRegs], int fo) {
    const V* src = reinterpret_cast<const V*>(frame);
    V* dst = reinterpret_cast<V*>(stage);
    V v[kUnitRegs];
#pragma unroll
    for (int j = 0; j < kUnitRegs; ++j)
        if (ur[j] != kNoUnit) v[j] = __ldcv(src + ur[j]);
    // units beyond the registers, two per thread in flight
    for (int f = fo; f < f1; f += 2 * NT) {
        unsigned u[2];
        V w[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int fj = f + j * NT;
            u[j] = fj < f1 ? __ldg(units + fj) : kNoUnit;
        }
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (u[j] != kNoUnit) w[j] = __ldcv(src + u[j]);
#pragma unroll
        for (int j = 0; j < 2; ++j)
            if (u[j] != kNoUnit) __stcg(dst + u[j], w[j]);
    }
#pragma unroll
    for (int j = 0; j < kUnitRegs; ++j)
        if (ur[j] != kNoUnit) __stcg(dst + ur[j], v[j]);
}

// The pixel rows of block `blk` from a host frame into staging (a block's entry of
// the ingest table: first unit, end unit).  `unit`: bytes per copy unit (16, 4, 2).
template <int NT>
__device__ __forceinline__ void ingest_block(const uint16_t* frame, uint16_t* stage, const unsigned* units,
                                             int4 bk, int unit, int tid) {
    unsigned ur[kUnitRegs];
#pragma unroll
    for (int j = 0; j < kUnitRegs; ++j) {
        const int f = bk.x + tid + j * NT;
        ur[j] = f < bk.y ? __ldg(units + f) : kNoUnit;
    }
    const int fo = bk.x + tid + kUnitRegs * NT;
    if (unit == 16) copy_units<uint4, NT>(frame, stage, units, bk.y, ur, fo);
    else if (unit == 4) copy_units<unsigned, NT>(frame, stage, units, bk.y, ur, fo);
    else copy_units<unsigned short, NT>(frame, stage, units, bk.y, ur, fo);
}

}  // namespace rtc_pixel

// Pixel-stage arguments of a handle for one frame (defined in calib_cog.cu).
rtc_pixel::PixelArgs pixel_args(const rtc_handle* h, const uint16_t* d_frame, float* d_s);
