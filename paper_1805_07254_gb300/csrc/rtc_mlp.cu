// C-ABI of the slope predictor (include/rtc.h): network objects for training and
// evaluation, and the predictor of a controller handle.  Errors of the rtc_mlp_*
// calls are reported by rtc_last_error(NULL).

#include <math.h>
#include <string.h>

#include <vector>

#include "mlp.h"
#include "rtc_internal.h"

struct rtc_mlp {
    int device = 0;
    MlpDev w{};
    float* parts = nullptr;      // [nparts_cap][RTC_MLP_NPARAMS + 1] CTA partials
    int nparts_cap = 0;
    int* d_nbr = nullptr;        // [nv][25] neighbour table (rtc_mlp_set_geometry)
    int nv = 0;
    int step = 0;                // Adam steps taken
};

namespace {

constexpr int kTile = 64;        // samples per CTA of the MLP kernels

int mfail(int code, const char* msg) {
    rtc_set_global_error(msg);
    return code;
}

struct Dev {
    int prev = -1;
    explicit Dev(int d) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != d) cudaSetDevice(d);
    }
    ~Dev() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int ensure_parts(rtc_mlp* m, int B) {
    const int need = (B + kTile - 1) / kTile;
    if (need <= m->nparts_cap) return RTC_OK;
    if (m->parts) cudaFree(m->parts);
    m->parts = nullptr;
    m->nparts_cap = 0;
    if (cudaMalloc(&m->parts, static_cast<size_t>(need) * (RTC_MLP_NPARAMS + 1) * sizeof(float)) != cudaSuccess)
        return mfail(RTC_ENOMEM, "cannot allocate the gradient partials");
    m->nparts_cap = need;
    return RTC_OK;
}

}  // namespace

// ---- shared with the handle's predictor ---------------------------------------------

int mlp_alloc(MlpDev& w) {
    w = MlpDev{};
    const size_t n = RTC_MLP_NPARAMS * sizeof(float);
    if (cudaMalloc(&w.master, n) != cudaSuccess || cudaMalloc(&w.m, n) != cudaSuccess ||
        cudaMalloc(&w.v, n) != cudaSuccess ||
        cudaMalloc(&w.w1_bf16, 64 * 208 * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&w.w2_bf16, 64 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess)
        return RTC_ENOMEM;
    if (cudaMemset(w.master, 0, n) != cudaSuccess || cudaMemset(w.m, 0, n) != cudaSuccess ||
        cudaMemset(w.v, 0, n) != cudaSuccess ||
        cudaMemset(w.w1_bf16, 0, 64 * 208 * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMemset(w.w2_bf16, 0, 64 * 64 * sizeof(__nv_bfloat16)) != cudaSuccess)
        return RTC_EDEVICE;
    return RTC_OK;
}

void mlp_free(MlpDev& w) {
    if (w.master) cudaFree(w.master);
    if (w.m) cudaFree(w.m);
    if (w.v) cudaFree(w.v);
    if (w.w1_bf16) cudaFree(w.w1_bf16);
    if (w.w2_bf16) cudaFree(w.w2_bf16);
    w = MlpDev{};
}

// Copy host parameters in, clear the Adam state and refresh the BF16 copies.
int mlp_upload(MlpDev& w, const float* params, cudaStream_t st) {
    const size_t n = RTC_MLP_NPARAMS * sizeof(float);
    if (cudaMemcpyAsync(w.master, params, n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(w.m, 0, n, st) != cudaSuccess || cudaMemsetAsync(w.v, 0, n, st) != cudaSuccess ||
        mlp_launch_refresh(w, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
        return RTC_EDEVICE;
    return RTC_OK;
}

// 5x5 neighbour table: index of the valid subaperture at (r + dr, c + dc), else -1.
std::vector<int> mlp_neighbours(const int32_t* rc, int nv, int nsub) {
    std::vector<int> grid(static_cast<size_t>(nsub) * nsub, -1);
    for (int i = 0; i < nv; ++i) grid[static_cast<size_t>(rc[2 * i]) * nsub + rc[2 * i + 1]] = i;
    std::vector<int> nbr(static_cast<size_t>(nv) * 25, -1);
    for (int i = 0; i < nv; ++i)
        for (int dr = -2; dr <= 2; ++dr)
            for (int dc = -2; dc <= 2; ++dc) {
                const int r = rc[2 * i] + dr, c = rc[2 * i + 1] + dc;
                if (r >= 0 && r < nsub && c >= 0 && c < nsub)
                    nbr[static_cast<size_t>(i) * 25 + (dr + 2) * 5 + (dc + 2)] = grid[static_cast<size_t>(r) * nsub + c];
            }
    return nbr;
}

// ---- C ABI ---------------------------------------------------------------------------

extern "C" {

int rtc_mlp_create(int32_t device, rtc_mlp** out) {
    if (!out) return mfail(RTC_EINVAL, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return mfail(RTC_EINVAL, "device not available");
    Dev d(device);
    if (mlp_configure() != cudaSuccess) return mfail(RTC_EDEVICE, "cannot configure the MLP kernels");
    rtc_mlp* m = new rtc_mlp();
    m->device = device;
    const int rc = mlp_alloc(m->w);
    if (rc != RTC_OK) {
        mlp_free(m->w);
        delete m;
        return mfail(rc, "cannot allocate the network");
    }
    *out = m;
    return RTC_OK;
}

int rtc_mlp_destroy(rtc_mlp* m) {
    if (!m) return RTC_OK;
    if (release_or_defer([m] { rtc_mlp_destroy(m); })) return RTC_OK;
    Dev d(m->device);
    cudaDeviceSynchronize();
    mlp_free(m->w);
    if (m->parts) cudaFree(m->parts);
    if (m->d_nbr) cudaFree(m->d_nbr);
    delete m;
    return RTC_OK;
}

int rtc_mlp_set_params(rtc_mlp* m, const float* params, int64_t n) {
    if (!m || !params || n != RTC_MLP_NPARAMS) return mfail(RTC_EINVAL, "need RTC_MLP_NPARAMS host floats");
    for (int64_t i = 0; i < n; ++i)
        if (!isfinite(params[i])) return mfail(RTC_EINVAL, "parameters must be finite");
    Dev d(m->device);
    if (mlp_upload(m->w, params, 0) != RTC_OK) return mfail(RTC_EDEVICE, "parameter upload failed");
    m->step = 0;
    return RTC_OK;
}

int rtc_mlp_get_params(rtc_mlp* m, float* params, int64_t n) {
    if (!m || !params || n != RTC_MLP_NPARAMS) return mfail(RTC_EINVAL, "need RTC_MLP_NPARAMS host floats");
    Dev d(m->device);
    if (cudaMemcpy(params, m->w.master, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess)
        return mfail(RTC_EDEVICE, "parameter download failed");
    return RTC_OK;
}

int rtc_mlp_set_geometry(rtc_mlp* m, const int32_t* rc, int32_t n_valid, int32_t nsub) {
    if (!m || (!rc && n_valid > 0) || n_valid < 0 || nsub <= 0) return mfail(RTC_EINVAL, "bad geometry");
    for (int i = 0; i < n_valid; ++i)
        if (rc[2 * i] < 0 || rc[2 * i] >= nsub || rc[2 * i + 1] < 0 || rc[2 * i + 1] >= nsub)
            return mfail(RTC_EINVAL, "subaperture outside the grid");
    Dev d(m->device);
    const std::vector<int> nbr = mlp_neighbours(rc, n_valid, nsub);
    if (m->d_nbr) cudaFree(m->d_nbr);
    m->d_nbr = nullptr;
    m->nv = 0;
    if (n_valid > 0) {
        if (cudaMalloc(&m->d_nbr, nbr.size() * sizeof(int)) != cudaSuccess)
            return mfail(RTC_ENOMEM, "cannot allocate the neighbour table");
        if (cudaMemcpy(m->d_nbr, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess)
            return mfail(RTC_EDEVICE, "neighbour table upload failed");
    }
    m->nv = n_valid;
    return RTC_OK;
}

int rtc_mlp_forward(rtc_mlp* m, const float* d_X, int32_t B, float* d_Y, void* stream) {
    if (!m || B < 0 || (B > 0 && (!d_X || !d_Y))) return mfail(RTC_EINVAL, "bad arguments");
    if (B == 0) return RTC_OK;
    Dev d(m->device);
    if (mlp_launch_forward(m->w, d_X, B, d_Y, static_cast<cudaStream_t>(stream)) != cudaSuccess)
        return mfail(RTC_EDEVICE, "forward launch failed");
    return RTC_OK;
}

int rtc_mlp_gradient(rtc_mlp* m, const float* d_X, const float* d_T, int32_t B, float* d_grad,
                     float* d_loss, void* stream) {
    if (!m || B <= 0 || !d_X || !d_T || !d_grad) return mfail(RTC_EINVAL, "bad arguments");
    Dev d(m->device);
    int rc = ensure_parts(m, B);
    if (rc != RTC_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (mlp_launch_train(m->w, d_X, d_T, B, m->parts, st) != cudaSuccess ||
        mlp_launch_update(m->w, m->parts, (B + kTile - 1) / kTile, B, 0.f, 0.9f, 0.999f, 1e-8f, 1,
                          d_grad, d_loss, st) != cudaSuccess)
        return mfail(RTC_EDEVICE, "gradient launch failed");
    return RTC_OK;
}

int rtc_mlp_train_step(rtc_mlp* m, const float* d_X, const float* d_T, int32_t B, float lr,
                       float* d_loss, void* stream) {
    if (!m || B <= 0 || !d_X || !d_T || !(lr > 0.f)) return mfail(RTC_EINVAL, "bad arguments");
    Dev d(m->device);
    int rc = ensure_parts(m, B);
    if (rc != RTC_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    m->step += 1;
    if (mlp_launch_train(m->w, d_X, d_T, B, m->parts, st) != cudaSuccess ||
        mlp_launch_update(m->w, m->parts, (B + kTile - 1) / kTile, B, lr, 0.9f, 0.999f, 1e-8f,
                          m->step, nullptr, d_loss, st) != cudaSuccess)
        return mfail(RTC_EDEVICE, "training launch failed");
    return RTC_OK;
}

int rtc_mlp_train_seq(rtc_mlp* m, const float* d_S, int32_t n_frames, const int32_t* d_samples,
                      int32_t B, float sigma, float lr, float* d_loss, void* stream) {
    if (!m || !d_S || !d_samples || B <= 0 || n_frames < 5 || !(sigma > 0.f) || !(lr > 0.f))
        return mfail(RTC_EINVAL, "bad arguments");
    if (!m->d_nbr) return mfail(RTC_ESTATE, "rtc_mlp_set_geometry first");
    Dev d(m->device);
    int rc = ensure_parts(m, B);
    if (rc != RTC_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    m->step += 1;
    if (mlp_launch_train_seq(m->w, d_S, n_frames, m->nv, m->d_nbr,
                             reinterpret_cast<const int2*>(d_samples), B, 1.f / sigma, m->parts,
                             st) != cudaSuccess ||
        mlp_launch_update(m->w, m->parts, (B + kTile - 1) / kTile, B, lr, 0.9f, 0.999f, 1e-8f,
                          m->step, nullptr, d_loss, st) != cudaSuccess)
        return mfail(RTC_EDEVICE, "training launch failed");
    return RTC_OK;
}

}  // extern "C"

extern "C" int rtc_mlp_predict_seq(rtc_mlp* m, const float* d_S, int32_t n_frames, float sigma,
                                   float* d_out, void* stream) {
    if (!m || !d_S || !d_out || n_frames < 0 || !(sigma > 0.f)) return mfail(RTC_EINVAL, "bad arguments");
    if (!m->d_nbr && m->nv > 0) return mfail(RTC_ESTATE, "rtc_mlp_set_geometry first");
    Dev d(m->device);
    const size_t row = 2 * static_cast<size_t>(m->nv);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int k = 3; k <= n_frames - 2; ++k) {
        // rows k-3 .. k of the sequence play the history ring with the newest in slot 3
        if (mlp_launch_predict(m->w, d_S + (k - 3) * row, static_cast<int>(row), 3, m->nv, m->d_nbr,
                               sigma, d_out + (k + 1) * row, st) != cudaSuccess)
            return mfail(RTC_EDEVICE, "prediction launch failed");
    }
    return RTC_OK;
}
