// Reconstruction from host buffers through a fixed device staging area that
// the library owns statically, for callers that must not allocate device
// memory (see ants_reconstruct_host_noalloc in include/ants.h).
//
// The staging area is a file-scope __device__ array.  Host code cannot use
// its name as a device address, so the first call on each device looks the
// address up with cudaGetSymbolAddress (with that device current) and keeps
// it; every later call on that device reuses it.  With lazy module loading
// (the CUDA default) that lookup is also what loads this file's module and so
// reserves the area on the device; a call with n_events = 0 does only that.
#include <mutex>

#include "internal.cuh"

namespace ants {

namespace {

constexpr size_t kStageBytes = (size_t)ANTS_NOALLOC_STAGE_BYTES;
constexpr size_t kAlign = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_stage[kStageBytes];

void *g_stage_addr[kMaxDevices];
std::mutex g_stage_mutex;

size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// bytes of the staging area used by n events of n_s sensors
size_t stage_bytes(long n, int n_s, bool with_start)
{
    size_t b = round_up((size_t)n * n_s * sizeof(float));           // signals
    if (with_start) b += round_up((size_t)n * 3 * sizeof(float));   // start positions
    b += round_up((size_t)n * 3 * sizeof(float));                   // xyz
    b += 2 * round_up((size_t)n * sizeof(float));                   // E, logL
    b += round_up((size_t)n * sizeof(int32_t));                     // status
    return b;
}

int stage_address(int device, unsigned char **out)
{
    if (device < 0 || device >= kMaxDevices) return fail(ANTS_E_ARG, "noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_stage_mutex);
    if (!g_stage_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_stage);  // device `device` is current
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(staging area)");
        g_stage_addr[device] = p;
    }
    *out = static_cast<unsigned char *>(g_stage_addr[device]);
    return ANTS_OK;
}

}  // namespace

}  // namespace ants

namespace ants {
namespace {

// largest n_events whose staging need fits the area
long noalloc_capacity(int n_sensors, bool with_start)
{
    if (n_sensors < 1) return 0;
    // largest n with stage_bytes(n) <= kStageBytes (bytes grow monotonically in n)
    long lo = 0, hi = (long)(kStageBytes / ((size_t)n_sensors * sizeof(float) + 24)) + 1;
    while (lo < hi) {
        long mid = (lo + hi + 1) / 2;
        if (stage_bytes(mid, n_sensors, with_start) <= kStageBytes) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

}  // namespace
}  // namespace ants

extern "C" ANTS_API int ants_reconstruct_host_noalloc(ants_ctx *ctx, const ants_lrf *lrf, int method,
                                                      const void *params, const void *signals_host,
                                                      int signal_dtype, long n_events, int n_sensors,
                                                      const float *start_xyz_host, float *xyz_host, float *E_host,
                                                      float *logL_host, int32_t *status_host)
{
    using namespace ants;
    begin_call();
    if (!ctx || !lrf || !params) return fail(ANTS_E_ARG, "ants_reconstruct_host_noalloc: NULL ctx, lrf or params");
    if (lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_reconstruct_host_noalloc: lrf belongs to another context");
    if (n_events < 0) return fail(ANTS_E_ARG, "ants_reconstruct_host_noalloc: n_events < 0");
    if (n_sensors != lrf->n_s)
        return fail(ANTS_E_SHAPE, "ants_reconstruct_host_noalloc: n_sensors %d but the LRF has %d", n_sensors,
                    lrf->n_s);
    if (signal_dtype != ANTS_F32)
        return fail(ANTS_E_UNIMPLEMENTED, "ants_reconstruct_host_noalloc: dtype %d", signal_dtype);
    if (method != ANTS_CGS_PLAIN)
        return fail(ANTS_E_UNIMPLEMENTED, "ants_reconstruct_host_noalloc: method %d", method);
    const ants_cgs_params *p = (const ants_cgs_params *)params;
    int rc = check_cgs_params(lrf, p);
    if (rc != ANTS_OK) return rc;
    const bool with_start = start_xyz_host != nullptr;
    const long cap = noalloc_capacity(n_sensors, with_start);
    if (n_events > cap)
        return fail(ANTS_E_ARG,
                    "ants_reconstruct_host_noalloc: %ld events exceed the static staging capacity of %ld events "
                    "for %d sensors (%zu bytes)",
                    n_events, cap, n_sensors, kStageBytes);
    if (n_events > 0 && (!signals_host || !xyz_host || !E_host || !logL_host || !status_host))
        return fail(ANTS_E_ARG, "ants_reconstruct_host_noalloc: NULL signal or output buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    unsigned char *base = nullptr;
    rc = stage_address(ctx->device, &base);  // set-up on the first call, also with n_events = 0
    if (rc != ANTS_OK) return rc;
    if (n_events == 0) return ANTS_OK;

    // carve the staging area; nothing in it has to start at zero (every region
    // is written before it is read)
    const long n = n_events;
    unsigned char *cur = base;
    float *d_sig = reinterpret_cast<float *>(cur);
    cur += round_up((size_t)n * n_sensors * sizeof(float));
    float *d_start = nullptr;
    if (with_start) {
        d_start = reinterpret_cast<float *>(cur);
        cur += round_up((size_t)n * 3 * sizeof(float));
    }
    float *d_xyz = reinterpret_cast<float *>(cur);
    cur += round_up((size_t)n * 3 * sizeof(float));
    float *d_E = reinterpret_cast<float *>(cur);
    cur += round_up((size_t)n * sizeof(float));
    float *d_logL = reinterpret_cast<float *>(cur);
    cur += round_up((size_t)n * sizeof(float));
    int32_t *d_status = reinterpret_cast<int32_t *>(cur);

    cudaStream_t s = ctx->stream[0];
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_sig, signals_host, (size_t)n * n_sensors * sizeof(float),
                                  cudaMemcpyHostToDevice, s), "noalloc: H2D signals");
    if (with_start)
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_start, start_xyz_host, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice,
                                      s), "noalloc: H2D start");
    rc = launch_cgs_plain(ctx, lrf, *p, d_sig, n, d_start, d_xyz, d_E, d_logL, d_status, nullptr, s);
    if (rc != ANTS_OK) return rc;
    ANTS_CUDA_TRY(cudaMemcpyAsync(xyz_host, d_xyz, (size_t)n * 3 * sizeof(float), cudaMemcpyDeviceToHost, s),
                  "noalloc: D2H xyz");
    ANTS_CUDA_TRY(cudaMemcpyAsync(E_host, d_E, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s),
                  "noalloc: D2H E");
    ANTS_CUDA_TRY(cudaMemcpyAsync(logL_host, d_logL, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s),
                  "noalloc: D2H logL");
    ANTS_CUDA_TRY(cudaMemcpyAsync(status_host, d_status, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                  "noalloc: D2H status");
    ANTS_CUDA_TRY(cudaStreamSynchronize(s), "noalloc: stream");
    return ANTS_OK;
}
