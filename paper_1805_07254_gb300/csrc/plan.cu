// Host-side planning, without a handle or a device: the slice cut of the
// asymmetric subaperture allocation (Sec. 2.3.3, Fig. 6 (d)) and the persistent
// loop's per-block ingest table for a banded readout (Sec. 2.2).  rtc_api.cu and
// loop_kernel.cu use these; rtc_plan_slices / rtc_plan_ingest expose them.

#include <algorithm>
#include <vector>

#include "rtc_internal.h"

namespace {

// The per-block cost model of the cut.  A block that owns n subapertures needs,
// after the last of their pixel rows has arrived, about
//     a + n * 2 nact (esz kAllocPsPerByte + kAllocPsPerElem) ps:
// the fixed part a is the same for every block and drops out of the cut; the
// rest is one SM streaming and multiplying the n subapertures' matrix columns.
// Fitted to ELT blocks running alone on a GB300 SM (506 / 324 / 262 ns per
// subaperture for FP32 / BF16 / FP8 columns of 4421 rows) and raised by ~1.3x,
// since blocks of neighbouring bands overlap in time and share the memory system.
constexpr long long kAllocPsPerByte = 12;
constexpr long long kAllocPsPerElem = 27;
constexpr int kAllocMaxWidth = 2;           // largest slice, in mean slice widths

// Band of pixel row y (of every WFS) when H rows are read out in nb bands: row y
// belongs to band j when floor(H j / nb) <= y < floor(H (j+1) / nb).
long long band_of_row(long long y, int nb, int side) {
    return ((y + 1) * nb - 1) / side;
}

}  // namespace

std::vector<int> plan_slices(const int32_t* rc, int nv, int nw, int npx, int side, int nact, int esz,
                             int max_slices, int n_bands, long long interval_ns) {
    const int nt = nv * nw;
    const int S = std::max(1, std::min(max_slices, nt));
    std::vector<int> g0(S + 1);
    for (int s = 0; s <= S; ++s) g0[s] = static_cast<int>(static_cast<long long>(nt) * s / S);
    if (n_bands <= 1 || nt <= S) return g0;
    // arrival of each subaperture: the band of its last pixel row
    std::vector<long long> t(nt);
    long long t_last = 0;
    for (int gi = 0; gi < nt; ++gi) {
        const int i = gi % nv;
        const long long last_row = static_cast<long long>(rc[2 * i]) * npx + npx - 1;
        t[gi] = band_of_row(last_row, n_bands, side) * interval_ns;
        t_last = std::max(t_last, t[gi]);
    }
    const long long c = 2ll * nact * (esz * kAllocPsPerByte + kAllocPsPerElem) / 1000 + 1;
    const int wmax = std::max(1, (kAllocMaxWidth * nt + S - 1) / S);
    // slices cut from the end for a common finish time T; returns their count
    auto cut = [&](long long T, std::vector<int>* starts) {
        int p = nt, k = 0;
        while (p > 0) {
            int n = 0;
            long long tmax = 0;
            while (p - n > 0 && n < wmax) {
                const long long tm = std::max(tmax, t[p - n - 1]);
                if (n > 0 && tm + c * (n + 1) > T) break;
                tmax = tm;
                ++n;
            }
            p -= n;
            ++k;
            if (starts) starts->push_back(p);
        }
        return k;
    };
    long long lo = t_last + c, hi = t_last + c * nt;   // cut(hi) <= ceil(nt / wmax) <= S
    if (cut(lo, nullptr) > S) {
        while (hi - lo > 1) {
            const long long mid = lo + (hi - lo) / 2;
            if (cut(mid, nullptr) <= S) hi = mid;
            else lo = mid;
        }
        lo = hi;
    }
    std::vector<int> starts;
    cut(lo, &starts);
    std::reverse(starts.begin(), starts.end());
    starts.push_back(nt);
    return starts;
}

void plan_ingest(const int32_t* rc, int nv, int npx, int side, const int* g0, int S, int G, int unit,
                 int n_bands, std::vector<unsigned>& units, std::vector<int>& blk) {
    units.clear();
    blk.assign(4 * static_cast<size_t>(G), 0);
    std::vector<unsigned> mine;
    for (int b = 0; b < G; ++b) {
        const int gb0 = g0[static_cast<long long>(S) * b / G];
        const int gb1 = g0[static_cast<long long>(S) * (b + 1) / G];
        mine.clear();
        long long last_row = 0;
        for (int gi = gb0; gi < gb1;) {
            const int w = gi / nv, i = gi - w * nv;
            const int r = rc[2 * i], c = rc[2 * i + 1];
            // a run of neighbours in one row of the subaperture grid
            int n = 1;
            while (gi + n < gb1 && (gi + n) / nv == w && rc[2 * (i + n)] == r && rc[2 * (i + n) + 1] == c + n)
                ++n;
            for (int y = 0; y < npx; ++y) {
                const long long row = static_cast<long long>(w) * side + static_cast<long long>(r) * npx + y;
                const long long b0 = (row * side + static_cast<long long>(c) * npx) * 2;
                const long long b1 = b0 + static_cast<long long>(n) * npx * 2;
                for (long long u = b0 / unit; u <= (b1 - 1) / unit; ++u) mine.push_back(static_cast<unsigned>(u));
            }
            last_row = std::max(last_row, static_cast<long long>(r) * npx + npx - 1);
            gi += n;
        }
        std::sort(mine.begin(), mine.end());
        mine.erase(std::unique(mine.begin(), mine.end()), mine.end());
        blk[4 * b] = static_cast<int>(units.size());
        blk[4 * b + 1] = static_cast<int>(units.size() + mine.size());
        blk[4 * b + 2] = static_cast<int>(band_of_row(last_row, std::max(n_bands, 1), side));
        units.insert(units.end(), mine.begin(), mine.end());
    }
}

namespace {

bool subaps_ok(const int32_t* rc, int nv, int nsub) {
    if (!rc || nv < 1) return false;
    for (int i = 0; i < nv; ++i)
        if (rc[2 * i] < 0 || rc[2 * i] >= nsub || rc[2 * i + 1] < 0 || rc[2 * i + 1] >= nsub) return false;
    return true;
}

int esize(int dt) {
    switch (dt) {
        case RTC_F32: return 4;
        case RTC_BF16:
        case RTC_F16: return 2;
        case RTC_FP8_E4M3:
        case RTC_INT8: return 1;
        default: return 0;
    }
}

}  // namespace

extern "C" int rtc_plan_slices(const int32_t* rc, int32_t n_valid, int32_t n_wfs, int32_t nsub, int32_t npx,
                               int32_t nact, int32_t store, int32_t max_slices, int32_t n_bands,
                               double band_interval_us, int32_t* g0_out, int32_t* n_slices) {
    if (!subaps_ok(rc, n_valid, nsub) || n_wfs < 1 || npx < 1 || nact < 1 || esize(store) == 0 ||
        max_slices < 1 || n_bands < 0 || n_bands > nsub * npx || !(band_interval_us >= 0.0) ||
        !(band_interval_us <= 1e6) || !g0_out || !n_slices)
        return RTC_EINVAL;
    const std::vector<int> g0 = plan_slices(rc, n_valid, n_wfs, npx, nsub * npx, nact, esize(store), max_slices,
                                            n_bands, static_cast<long long>(band_interval_us * 1e3 + 0.5));
    for (size_t s = 0; s < g0.size(); ++s) g0_out[s] = g0[s];
    *n_slices = static_cast<int32_t>(g0.size() - 1);
    return RTC_OK;
}

extern "C" int rtc_plan_ingest(const int32_t* rc, int32_t n_valid, int32_t n_wfs, int32_t nsub, int32_t npx,
                               const int32_t* g0, int32_t n_slices, int32_t blocks, int32_t unit_bytes,
                               int32_t n_bands, int32_t* blk_out, uint32_t* units_out, int64_t units_cap,
                               int64_t* n_units) {
    if (!subaps_ok(rc, n_valid, nsub) || n_wfs < 1 || npx < 1 || !g0 || n_slices < 1 || blocks < 1 ||
        blocks > n_slices || (unit_bytes != 2 && unit_bytes != 4 && unit_bytes != 16) || n_bands < 0 ||
        n_bands > nsub * npx || !blk_out || !n_units)
        return RTC_EINVAL;
    const int nt = n_valid * n_wfs;
    if (g0[0] != 0 || g0[n_slices] != nt) return RTC_EINVAL;
    for (int s = 0; s < n_slices; ++s)
        if (g0[s + 1] <= g0[s]) return RTC_EINVAL;
    const long long frame_bytes = static_cast<long long>(n_wfs) * nsub * npx * nsub * npx * 2;
    if (frame_bytes % unit_bytes != 0 || frame_bytes / unit_bytes > 0xffffffffll) return RTC_EINVAL;
    std::vector<unsigned> units;
    std::vector<int> blk;
    plan_ingest(rc, n_valid, npx, nsub * npx, g0, n_slices, blocks, unit_bytes, n_bands, units, blk);
    *n_units = static_cast<int64_t>(units.size());
    for (size_t i = 0; i < blk.size(); ++i) blk_out[i] = blk[i];
    if (units_out) {
        if (units_cap < static_cast<int64_t>(units.size())) return RTC_EINVAL;
        std::copy(units.begin(), units.end(), units_out);
    }
    return RTC_OK;
}
