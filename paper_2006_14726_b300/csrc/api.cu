// api.cu -- host-side plumbing of the C ABI: error strings, status word, version, struct sizes.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace wrs {

static thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(WRS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace wrs

extern "C" {

const char* wrs_version(void) { return "wrs 0.3 (sm_103a)"; }

const char* wrs_last_error(void) { return wrs::g_err; }

size_t wrs_session_size(void) { return sizeof(wrs_session); }

size_t wrs_camera_size(void) { return sizeof(wrs_camera); }

float wrs_window_weight(float decay, uint32_t age) {
    if (!(decay > 0.0f && decay <= 1.0f)) return __builtin_nanf("");
    float w = 1.0f;
    for (uint32_t g = 0; g < age; g++) w = w * decay;  // one binary32 rounding per frame of age
    return w;
}

int wrs_check_status(int32_t* status, wrs_stream_t stream) {
    if (!status) return wrs::fail(WRS_ERR_ARG, "wrs_check_status: status is NULL");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int32_t h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return wrs::cuda_fail(e, "wrs_check_status");
    if (h == 0) {
        wrs::g_err[0] = 0;
        return WRS_OK;
    }
    return wrs::fail(WRS_ERR_DEVICE, "device status 0x%x:%s%s%s%s", (unsigned)h,
                     (h & WRS_STATUS_STACK_OVERFLOW) ? " traversal stack overflow" : "",
                     (h & WRS_STATUS_CHUNK_OVERFLOW) ? " backward chunk table overflow" : "",
                     (h & WRS_STATUS_MALFORMED_TREE) ? " malformed tree" : "",
                     (h & WRS_STATUS_SPLAT_OVERFLOW) ? " splat capacity overflow" : "");
}

}  // extern "C"

namespace wrs {
// Camera validation shared by the entry points.
int check_camera(const wrs_camera* c, const char* fn) {
    if (!c) return fail(WRS_ERR_ARG, "%s: camera is NULL", fn);
    if (c->width <= 0 || c->height <= 0 || c->width > 32768 || c->height > 32768)
        return fail(WRS_ERR_ARG, "%s: camera size %dx%d out of range (1..32768)", fn, c->width,
                    c->height);
    const float* v = c->eye;
    for (int k = 0; k < 12; k++)
        if (!(v[k] == v[k]) || v[k] > 3.0e38f || v[k] < -3.0e38f)
            return fail(WRS_ERR_ARG, "%s: camera vector component %d is not finite", fn, k);
    if (!(c->tan_half_fovy > 0.0f && c->tan_half_fovy < 1.0e6f))
        return fail(WRS_ERR_ARG, "%s: tan_half_fovy must be positive and finite", fn);
    return WRS_OK;
}
}  // namespace wrs
