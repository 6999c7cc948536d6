// extern "C" entry points declared in include/oat.h: argument checks, device selection,
// error reporting.  All arithmetic lives in the kernels (forward.cu, adjoint.cu) and the
// plan builder (plan.cpp).
#include <cstdint>
#include <cmath>
#include <mutex>
#include <string>

#include "oat_internal.h"
#include "../../include/oat_probe.h"

namespace oat {

int plan_create(const oat_geometry *g, int device, Plan **out);
void plan_destroy(Plan *p);

static thread_local std::string g_last_error;

int set_error(int code, const std::string &msg) {
    g_last_error = msg;
    return code;
}

int current_sm_count() {
    static std::mutex mu;
    static int cache[256] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return 1; }
    std::lock_guard<std::mutex> lock(mu);
    if (cache[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
            cudaGetLastError();
            return 1;
        }
        cache[dev] = n;
    }
    return cache[dev];
}

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    cudaError_t err = cudaSuccess;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) err = cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace oat

using namespace oat;

extern "C" {

int oat_version(void) { return 10000; }

const char *oat_last_error(void) { return g_last_error.c_str(); }

int oat_plan_create(const oat_geometry *geom, int device, oat_plan *out) {
    if (!out) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_create: out is NULL");
    *out = nullptr;
    Plan *p = nullptr;
    int rc = plan_create(geom, device, &p);
    if (rc != OAT_OK) return rc;
    *out = reinterpret_cast<oat_plan>(p);
    g_last_error.clear();
    return OAT_OK;
}

int oat_plan_destroy(oat_plan plan) {
    plan_destroy(reinterpret_cast<Plan *>(plan));
    return OAT_OK;
}

int oat_project(oat_plan plan, const float *d_vol, void *d_data, void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !d_vol || !d_data) return set_error(OAT_ERR_INVALID_ARG, "oat_project: NULL plan or buffer");
    if (!aligned16(d_vol) || !aligned16(d_data))
        return set_error(OAT_ERR_INVALID_ARG, "oat_project: buffers must be 16-byte aligned");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_project: ") + cudaGetErrorString(dg.err));
    return launch_project(*p, d_vol, d_data, (cudaStream_t)stream);
}

int oat_backproject(oat_plan plan, const void *d_data, float *d_vol, void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !d_vol || !d_data) return set_error(OAT_ERR_INVALID_ARG, "oat_backproject: NULL plan or buffer");
    if (!aligned16(d_vol) || !aligned16(d_data))
        return set_error(OAT_ERR_INVALID_ARG, "oat_backproject: buffers must be 16-byte aligned");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_backproject: ") + cudaGetErrorString(dg.err));
    return launch_backproject(*p, d_data, d_vol, (cudaStream_t)stream);
}

int oat_backproject_noalloc(oat_plan plan, const void *d_data, float *d_vol, void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !d_vol || !d_data) return set_error(OAT_ERR_INVALID_ARG, "oat_backproject_noalloc: NULL plan or buffer");
    if (!aligned16(d_vol) || !aligned16(d_data))
        return set_error(OAT_ERR_INVALID_ARG, "oat_backproject_noalloc: buffers must be 16-byte aligned");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess)
        return set_error(OAT_ERR_CUDA, std::string("oat_backproject_noalloc: ") + cudaGetErrorString(dg.err));
    return launch_backproject_static(*p, d_data, d_vol, (cudaStream_t)stream);
}

int oat_plan_set_fbp_weights(oat_plan plan, const double *weights) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !weights) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_fbp_weights: NULL plan or weights");
    for (int q = 0; q < p->Q; ++q)
        if (!std::isfinite(weights[q])) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_fbp_weights: non-finite weight");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess)
        return set_error(OAT_ERR_CUDA, std::string("oat_plan_set_fbp_weights: ") + cudaGetErrorString(dg.err));
    for (int q = 0; q < p->Q; ++q) p->fbp_host[2 * (size_t)q].w = (float)weights[q];
    cudaError_t e = cudaMemcpy(p->d_fbp, p->fbp_host.data(), sizeof(float4) * p->fbp_host.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_set_fbp_weights: ") + cudaGetErrorString(e));
    p->fbp_weights = true;
    return OAT_OK;
}

int oat_fbp(oat_plan plan, const void *d_data, float *d_vol, void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !d_vol || !d_data) return set_error(OAT_ERR_INVALID_ARG, "oat_fbp: NULL plan or buffer");
    if (!aligned16(d_vol) || !aligned16(d_data)) return set_error(OAT_ERR_INVALID_ARG, "oat_fbp: buffers must be 16-byte aligned");
    if (!p->fbp_weights) return set_error(OAT_ERR_INVALID_ARG, "oat_fbp: weights not set (oat_plan_set_fbp_weights)");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_fbp: ") + cudaGetErrorString(dg.err));
    return launch_fbp(*p, d_data, d_vol, (cudaStream_t)stream);
}

int oat_fbp_sample_positions(oat_plan plan, const int *d_nodes, const int *d_transducers, int n, double *d_out,
                             void *stream) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || n < 0 || (n > 0 && (!d_nodes || !d_transducers || !d_out)))
        return set_error(OAT_ERR_INVALID_ARG, "oat_fbp_sample_positions: NULL plan or buffer, or n < 0");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess)
        return set_error(OAT_ERR_CUDA, std::string("oat_fbp_sample_positions: ") + cudaGetErrorString(dg.err));
    return launch_fbp_kpos(*p, d_nodes, d_transducers, n, d_out, (cudaStream_t)stream);
}

int oat_plan_set_eir(oat_plan plan, const double *h, int n_taps, int first_index) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_eir: NULL plan");
    if (n_taps < 0 || (n_taps > 0 && !h)) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_eir: bad tap array");
    for (int i = 0; i < n_taps; ++i)
        if (!std::isfinite(h[i])) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_eir: non-finite tap");
    if (first_index < -(1 << 30) || first_index > (1 << 30))
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_eir: first_index out of range (|m0| <= 2^30)");
    DeviceGuard dg(p->device);
    if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_set_eir: ") + cudaGetErrorString(dg.err));
    if (n_taps == 0) {
        p->eir_n = 0;
        return OAT_OK;
    }
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    if (sizeof(double) * ((size_t)p->K + (size_t)n_taps) > (size_t)optin)
        return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_eir: n_samples + n_taps doubles exceed the shared memory of a block");
    cudaError_t e = cudaSuccess;
    if (!p->d_eir_z) {
        e = cudaMalloc(&p->d_eir_z, sizeof(float) * (size_t)p->Q * p->K);
        if (e != cudaSuccess) {
            p->d_eir_z = nullptr;
            cudaGetLastError();
            return set_error(e == cudaErrorMemoryAllocation ? OAT_ERR_OOM : OAT_ERR_CUDA,
                             std::string("oat_plan_set_eir: cudaMalloc: ") + cudaGetErrorString(e));
        }
        p->scratch_bytes += (long long)(sizeof(float) * (size_t)p->Q * p->K);
    }
    if (p->d_eir) { cudaFree(p->d_eir); p->d_eir = nullptr; }
    e = cudaMalloc(&p->d_eir, sizeof(double) * (size_t)n_taps);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_eir, h, sizeof(double) * (size_t)n_taps, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        if (p->d_eir) { cudaFree(p->d_eir); p->d_eir = nullptr; }
        p->eir_n = 0;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? OAT_ERR_OOM : OAT_ERR_CUDA,
                         std::string("oat_plan_set_eir: ") + cudaGetErrorString(e));
    }
    p->eir_n = n_taps;
    p->eir_m0 = first_index;
    return set_eir_attributes(*p);
}

int oat_plan_query(oat_plan plan, int want_count, oat_stats *st) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || !st) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_query: NULL plan or stats");
    st->n_radius_classes = p->n_cls;
    st->n_rings = p->n_rings;
    st->points_ball = p->points_ball;
    st->points_grid = -1;
    st->table_bytes = p->table_bytes;
    st->scratch_bytes = p->scratch_bytes;
    st->work_items = p->fwd.items;
    if (want_count) {
        DeviceGuard dg(p->device);
        if (dg.err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_query: ") + cudaGetErrorString(dg.err));
        long long n = 0;
        int rc = oat::count_grid_points(*p, &n);
        if (rc != OAT_OK) return rc;
        st->points_grid = n;
    }
    return OAT_OK;
}

int oat_plan_set_profiling(oat_plan plan, int enable) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_set_profiling: NULL plan");
    if (enable && p->ev[0].empty()) {
        DeviceGuard dg(p->device);
        for (int w = 0; w < 3; ++w) {
            p->ev[w].resize(2 * kMaxEvents);
            for (auto &e : p->ev[w]) {
                cudaError_t err = cudaEventCreate(&e);
                if (err != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_set_profiling: ") + cudaGetErrorString(err));
            }
        }
    }
    p->profiling = enable != 0;
    return OAT_OK;
}

int oat_plan_kernel_time(oat_plan plan, int which, int reset, double *ms, long long *launches) {
    Plan *p = reinterpret_cast<Plan *>(plan);
    if (!p || which < 0 || which > 2) return set_error(OAT_ERR_INVALID_ARG, "oat_plan_kernel_time: bad plan or kernel index");
    DeviceGuard dg(p->device);
    for (int i = 0; i + 1 < p->ev_used[which]; i += 2) {
        cudaError_t e = cudaEventSynchronize(p->ev[which][i + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->ev[which][i], p->ev[which][i + 1]);
        if (e != cudaSuccess) return set_error(OAT_ERR_CUDA, std::string("oat_plan_kernel_time: ") + cudaGetErrorString(e));
        p->ms_acc[which] += t;
        p->launches[which] += 1;
    }
    p->ev_used[which] = 0;
    if (ms) *ms = p->ms_acc[which];
    if (launches) *launches = p->launches[which];
    if (reset) { p->ms_acc[which] = 0; p->launches[which] = 0; }
    return OAT_OK;
}

}  // extern "C"
