// libants: handles, errors, LRF storage and evaluation, host-buffer driver.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include <cuda_fp16.h>

#include "internal.cuh"
#include "bspline.cuh"

namespace ants {

static thread_local std::string t_err;
static thread_local long t_launches = 0;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(ANTS_E_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

void begin_call()
{
    t_err.clear();
    t_launches = 0;
    // a failed runtime call outside any entry point (or in a free function)
    // must not surface as this call's error; sticky errors persist anyway
    (void)cudaGetLastError();
}

void count_launch(long n) { t_launches += n; }

int lrf_dims(int type)
{
    // spline axes: radial r; XY and composite (its box) x, y; axial+z r, z;
    // sliced x, y (+ the plane range); XYZ x, y, z
    return type == ANTS_LRF_RADIAL ? 1 : (type == ANTS_LRF_XYZ ? 3 : 2);
}

void *ctx_scratch(ants_ctx *ctx, int slot, size_t bytes)
{
    if (slot < 0 || slot >= kScratchSlots) {
        fail(ANTS_E_INTERNAL, "scratch slot %d", slot);
        return nullptr;
    }
    if (ctx->scratch_cap[slot] >= bytes && ctx->scratch[slot]) return ctx->scratch[slot];
    cudaFree(ctx->scratch[slot]);
    ctx->scratch[slot] = nullptr;
    ctx->scratch_cap[slot] = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&ctx->scratch[slot], want);
    if (e != cudaSuccess) {
        fail(ANTS_E_OOM, "device scratch of %zu bytes: %s", want, cudaGetErrorString(e));
        ctx->scratch[slot] = nullptr;
        return nullptr;
    }
    ctx->scratch_cap[slot] = want;
    return ctx->scratch[slot];
}

__global__ void widen_half_kernel(const __half *__restrict__ h, size_t n, float *__restrict__ f)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        f[i] = __half2float(h[i]);
}

int widen_half(const __half *h, size_t n, float *f, cudaStream_t s)
{
    if (n == 0) return ANTS_OK;
    size_t blocks = (n + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    widen_half_kernel<<<(unsigned)blocks, 256, 0, s>>>(h, n, f);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? ANTS_OK : cuda_fail(e, "widen FP16 signals");
}

}  // namespace ants

using namespace ants;

namespace ants {
namespace {

__global__ void bounds_selftest_kernel(int *word)
{
    if (ANTS_IN_RANGE(word, 7, 5, 9999)) {
        // an access would go here; the check keeps it from happening
    }
}

}  // namespace
}  // namespace ants

namespace ants {

int check_bounds(const ants_ctx *ctx, cudaStream_t s)
{
#ifdef ANTS_DEBUG_BOUNDS
    int site = 0;
    ANTS_CUDA_TRY(cudaStreamSynchronize(s), "index check: synchronize");
    ANTS_CUDA_TRY(cudaMemcpy(&site, ctx->d_bounds, sizeof(int), cudaMemcpyDeviceToHost), "index check: read");
    if (site) return fail(ANTS_E_INTERNAL, "index check: an index out of range at site %d", site);
#else
    (void)ctx;
    (void)s;
#endif
    return ANTS_OK;
}

}  // namespace ants

extern "C" {

ANTS_API const char *ants_last_error(void) { return t_err.c_str(); }

ANTS_API int ants_version(void) { return 1; }

ANTS_API long ants_last_launch_count(void) { return t_launches; }

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------

ANTS_API int ants_ctx_create(int device, ants_ctx **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_ctx_create: out is NULL");
    *out = nullptr;
    int n_dev = 0;
    ANTS_CUDA_TRY(cudaGetDeviceCount(&n_dev), "cudaGetDeviceCount");
    if (device < 0 || device >= n_dev)
        return fail(ANTS_E_ARG, "ants_ctx_create: device %d not in [0, %d)", device, n_dev);
    ANTS_CUDA_TRY(cudaSetDevice(device), "cudaSetDevice");
    ants_ctx *c = new (std::nothrow) ants_ctx();
    if (!c) return fail(ANTS_E_OOM, "ants_ctx_create: out of host memory");
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaGetDeviceProperties"); }
    c->n_sm = prop.multiProcessorCount;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    for (int k = 0; k < 2; ++k) {
        e = cudaStreamCreateWithFlags(&c->stream[k], cudaStreamNonBlocking);
        if (e != cudaSuccess) { ants_ctx_destroy(c); return cuda_fail(e, "cudaStreamCreate"); }
    }
    e = cudaMalloc(&c->d_fault, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_fault, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_bounds, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_bounds, 0, sizeof(int));
    if (e != cudaSuccess) { ants_ctx_destroy(c); return cuda_fail(e, "fault word"); }
    *out = c;
    return ANTS_OK;
}

static void free_host_buffers(ants_ctx *c)
{
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->d_sig[k]);
        cudaFree(c->d_start[k]);
        cudaFree(c->d_out[k]);
        cudaFree(c->d_status[k]);
        c->d_sig[k] = nullptr;
        c->d_start[k] = nullptr;
        c->d_out[k] = nullptr;
        c->d_status[k] = nullptr;
    }
    c->host_cap_events = 0;
    c->host_cap_sensors = 0;
}

ANTS_API void ants_ctx_destroy(ants_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    free_host_buffers(ctx);
    for (int k = 0; k < kScratchSlots; ++k) cudaFree(ctx->scratch[k]);
    cudaFree(ctx->d_fault);
    cudaFree(ctx->d_bounds);
    for (int k = 0; k < 2; ++k)
        if (ctx->stream[k]) cudaStreamDestroy(ctx->stream[k]);
    delete ctx;
}

ANTS_API int ants_ctx_fault(ants_ctx *ctx, int *fault)
{
    begin_call();
    if (!ctx || !fault) return fail(ANTS_E_ARG, "ants_ctx_fault: NULL argument");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaDeviceSynchronize(), "ants_ctx_fault: synchronize");
    ANTS_CUDA_TRY(cudaMemcpy(fault, ctx->d_fault, sizeof(int), cudaMemcpyDeviceToHost), "ants_ctx_fault: read");
    ANTS_CUDA_TRY(cudaMemset(ctx->d_fault, 0, sizeof(int)), "ants_ctx_fault: clear");
    return *fault ? fail(ANTS_E_TIMEOUT, "a device-side wait ran out of time") : ANTS_OK;
}

ANTS_API int ants_build_flags(void)
{
#ifdef ANTS_DEBUG_BOUNDS
    return ANTS_BUILD_DEBUG_BOUNDS;
#else
    return 0;
#endif
}

ANTS_API int ants_debug_bounds_site(ants_ctx *ctx, int *site)
{
    begin_call();
    if (!ctx || !site) return fail(ANTS_E_ARG, "ants_debug_bounds_site: NULL argument");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaDeviceSynchronize(), "ants_debug_bounds_site: synchronize");
    ANTS_CUDA_TRY(cudaMemcpy(site, ctx->d_bounds, sizeof(int), cudaMemcpyDeviceToHost), "ants_debug_bounds_site: read");
    ANTS_CUDA_TRY(cudaMemset(ctx->d_bounds, 0, sizeof(int)), "ants_debug_bounds_site: clear");
    return ANTS_OK;
}


ANTS_API int ants_selftest_bounds(ants_ctx *ctx)
{
    using namespace ants;
    begin_call();
    if (!ctx) return fail(ANTS_E_ARG, "ants_selftest_bounds: NULL context");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    bounds_selftest_kernel<<<1, 1>>>(ctx->d_bounds);
    ANTS_CUDA_TRY(cudaGetLastError(), "bounds self-test launch");
    ANTS_CUDA_TRY(cudaDeviceSynchronize(), "bounds self-test");
    return ANTS_OK;
}



// ---------------------------------------------------------------------------
// detector
// ---------------------------------------------------------------------------

ANTS_API int ants_detector_create(int n_sensors, const double *sensor_xy_host,
                                  const double *rel_gain_host, ants_detector **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_detector_create: out is NULL");
    *out = nullptr;
    if (n_sensors < 1 || n_sensors > 1024)
        return fail(ANTS_E_ARG, "ants_detector_create: n_sensors %d not in [1, 1024]", n_sensors);
    if (!sensor_xy_host) return fail(ANTS_E_ARG, "ants_detector_create: sensor_xy_host is NULL");
    for (int i = 0; i < 2 * n_sensors; ++i)
        if (!std::isfinite(sensor_xy_host[i]))
            return fail(ANTS_E_ARG, "ants_detector_create: sensor position %d not finite", i / 2);
    if (rel_gain_host)
        for (int i = 0; i < n_sensors; ++i)
            if (!(rel_gain_host[i] > 0.0) || !std::isfinite(rel_gain_host[i]))
                return fail(ANTS_E_ARG, "ants_detector_create: gain of sensor %d must be > 0", i);
    ants_detector *d = new (std::nothrow) ants_detector();
    if (!d) return fail(ANTS_E_OOM, "ants_detector_create: out of host memory");
    d->n_s = n_sensors;
    d->xy.assign(sensor_xy_host, sensor_xy_host + 2 * n_sensors);
    d->gain.assign(n_sensors, 1.0);
    if (rel_gain_host) d->gain.assign(rel_gain_host, rel_gain_host + n_sensors);
    *out = d;
    return ANTS_OK;
}

ANTS_API void ants_detector_free(ants_detector *det) { delete det; }

// ---------------------------------------------------------------------------
// LRF
// ---------------------------------------------------------------------------

static int upload_lrf(ants_lrf *L)
{
    std::vector<float> c(L->coef.size()), xy(L->sxy.size()), g(L->n_s), w(L->n_s);
    // positive: every coefficient > 0 and max <= 2^100 min, so every LRF value
    // (between the smallest and the largest coefficient) is > 0 and every
    // ratio of two values is a normal float
    int positive = 1;
    float cmin = INFINITY, cmax = 0.0f;
    for (size_t k = 0; k < c.size(); ++k) {
        c[k] = (float)L->coef[k];
        if (!(c[k] > 0.0f)) positive = 0;
        cmin = std::min(cmin, c[k]);
        cmax = std::max(cmax, c[k]);
    }
    if (positive && !(cmax <= std::ldexp(cmin, 100))) positive = 0;
    for (size_t k = 0; k < xy.size(); ++k) xy[k] = (float)L->sxy[k];
    for (int i = 0; i < L->n_s; ++i) {
        g[i] = (float)L->gain[i];
        w[i] = (float)(1.0 / L->rel_gain[i]);
    }
    ANTS_CUDA_TRY(cudaSetDevice(L->ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaMalloc(&L->d_coef, c.size() * sizeof(float)), "cudaMalloc(lrf coef)");
    ANTS_CUDA_TRY(cudaMalloc(&L->d_sxy, xy.size() * sizeof(float)), "cudaMalloc(lrf sxy)");
    ANTS_CUDA_TRY(cudaMalloc(&L->d_gain, g.size() * sizeof(float)), "cudaMalloc(lrf gain)");
    ANTS_CUDA_TRY(cudaMalloc(&L->d_cogw, w.size() * sizeof(float)), "cudaMalloc(lrf cogw)");
    ANTS_CUDA_TRY(cudaMemcpy(L->d_coef, c.data(), c.size() * sizeof(float), cudaMemcpyHostToDevice),
                  "upload coef");
    ANTS_CUDA_TRY(cudaMemcpy(L->d_sxy, xy.data(), xy.size() * sizeof(float), cudaMemcpyHostToDevice),
                  "upload sxy");
    ANTS_CUDA_TRY(cudaMemcpy(L->d_gain, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice),
                  "upload gain");
    ANTS_CUDA_TRY(cudaMemcpy(L->d_cogw, w.data(), w.size() * sizeof(float), cudaMemcpyHostToDevice),
                  "upload cog weights");
    LrfDev &D = L->dev;
    D.dbg = L->ctx->d_bounds;
    D.coef2 = nullptr;
    D.coef2_pf = nullptr;
    D.coef_t = nullptr;
    D.set_of = nullptr;
    D.op_of = nullptr;
    D.n_sets = L->n_sets;
    D.sym_c[0] = (float)L->sym_c[0];
    D.sym_c[1] = (float)L->sym_c[1];
    if (!L->ops.empty()) {
        ANTS_CUDA_TRY(cudaMalloc(&L->d_op_of, L->ops.size() * sizeof(int)), "cudaMalloc(lrf operations)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_op_of, L->ops.data(), L->ops.size() * sizeof(int), cudaMemcpyHostToDevice),
                      "upload operations");
        D.op_of = L->d_op_of;
    }
    if (!L->groups.empty()) {
        ANTS_CUDA_TRY(cudaMalloc(&L->d_set_of, L->groups.size() * sizeof(int)), "cudaMalloc(lrf groups)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_set_of, L->groups.data(), L->groups.size() * sizeof(int), cudaMemcpyHostToDevice),
                      "upload groups");
        D.set_of = L->d_set_of;
    }
    D.n_pairs = (L->n_s + 1) / 2;
    D.pair_stride = 0;
    if (L->type == ANTS_LRF_XY && L->ops.empty()) {
        const int ps = L->n_coef;
        std::vector<float2> c2((size_t)D.n_pairs * ps);
        for (int p = 0; p < D.n_pairs; ++p)
            for (int k = 0; k < ps; ++k) {
                int i0 = 2 * p, i1 = 2 * p + 1;
                c2[(size_t)p * ps + k] = make_float2(c[(size_t)i0 * ps + k], i1 < L->n_s ? c[(size_t)i1 * ps + k] : 0.0f);
            }
        ANTS_CUDA_TRY(cudaMalloc(&L->d_coef2, c2.size() * sizeof(float2)), "cudaMalloc(lrf coef pairs)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_coef2, c2.data(), c2.size() * sizeof(float2), cudaMemcpyHostToDevice),
                      "upload coef pairs");
        D.coef2 = L->d_coef2;
        D.pair_stride = ps;
        std::vector<float2> cpf(c2.size());
        for (int p = 0; p < D.n_pairs; ++p)
            for (int k = 0; k < ps; ++k) cpf[(size_t)k * D.n_pairs + p] = c2[(size_t)p * ps + k];
        ANTS_CUDA_TRY(cudaMalloc(&L->d_coef2_pf, cpf.size() * sizeof(float2)), "cudaMalloc(lrf coef pairs, pair-fastest)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_coef2_pf, cpf.data(), cpf.size() * sizeof(float2), cudaMemcpyHostToDevice),
                      "upload coef pairs (pair-fastest)");
        D.coef2_pf = L->d_coef2_pf;
        std::vector<float> ct(c.size());
        for (int i = 0; i < L->n_s; ++i)
            for (int k = 0; k < ps; ++k) ct[(size_t)k * L->n_s + i] = c[(size_t)i * ps + k];
        ANTS_CUDA_TRY(cudaMalloc(&L->d_coeft, ct.size() * sizeof(float)), "cudaMalloc(lrf coef sensor-minor)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_coeft, ct.data(), ct.size() * sizeof(float), cudaMemcpyHostToDevice),
                      "upload coef sensor-minor");
        D.coef_t = L->d_coeft;
    }
    D.rpoly = nullptr;
    if (L->type == ANTS_LRF_RADIAL || L->type == ANTS_LRF_COMPOSITE) {
        // uniform cubic B-spline on interval j: sum_a c[j+a] B_a(t) expanded in
        // powers of t (FP64, then rounded once to FP32); a composite set's
        // axial part leads its coefficients
        const int ni = L->type == ANTS_LRF_COMPOSITE ? L->n_int_r : L->n_int[0];
        std::vector<float4> rp((size_t)L->n_sets * ni);
        for (int set = 0; set < L->n_sets; ++set)
            for (int j = 0; j < ni; ++j) {
                const double *c = L->coef.data() + (size_t)set * L->n_coef + j;
                const double p0 = (c[0] + 4.0 * c[1] + c[2]) / 6.0;
                const double p1 = (c[2] - c[0]) / 2.0;
                const double p2 = (c[0] - 2.0 * c[1] + c[2]) / 2.0;
                const double p3 = (-c[0] + 3.0 * c[1] - 3.0 * c[2] + c[3]) / 6.0;
                rp[(size_t)set * ni + j] = make_float4((float)p0, (float)p1, (float)p2, (float)p3);
            }
        ANTS_CUDA_TRY(cudaMalloc(&L->d_rpoly, rp.size() * sizeof(float4)), "cudaMalloc(lrf radial polynomials)");
        ANTS_CUDA_TRY(cudaMemcpy(L->d_rpoly, rp.data(), rp.size() * sizeof(float4), cudaMemcpyHostToDevice),
                      "upload radial polynomials");
        D.rpoly = L->d_rpoly;
    }
    D.type = L->type;
    D.n_s = L->n_s;
    D.shared = L->shared;
    D.n_coef = L->n_coef;
    for (int a = 0; a < 3; ++a) {
        D.n_int[a] = L->n_int[a];
        D.lo[a] = (float)L->lo[a];
        D.hi[a] = (float)L->hi[a];
        D.inv_h[a] = L->n_int[a] > 0 ? (float)((double)L->n_int[a] / (L->hi[a] - L->lo[a])) : 0.0f;
    }
    D.stride_y = L->n_int[0] + 3;
    D.stride_z = (L->n_int[0] + 3) * (L->type == ANTS_LRF_RADIAL ? 1 : L->n_int[1] + 3);
    D.n_int_r = L->n_int_r;
    D.hi_r = (float)L->hi_r;
    D.inv_h_r = L->n_int_r > 0 ? (float)((double)L->n_int_r / L->hi_r) : 0.0f;
    D.n_planes = L->n_planes;
    D.n_coef_xy = (L->n_int[0] + 3) * (L->n_int[1] + 3);
    if (L->type == ANTS_LRF_SLICED) D.inv_h[2] = (float)((double)(L->n_planes - 1) / (L->hi[2] - L->lo[2]));
    D.positive = positive;
    D.coef = L->d_coef;
    D.sxy = L->d_sxy;
    D.gain = L->d_gain;
    D.cog_w = L->d_cogw;
    return ANTS_OK;
}

ANTS_API void ants_lrf_free(ants_lrf *lrf)
{
    if (!lrf) return;
    cudaSetDevice(lrf->device);
    cudaFree(lrf->d_coef);
    cudaFree(lrf->d_sxy);
    cudaFree(lrf->d_gain);
    cudaFree(lrf->d_cogw);
    cudaFree(lrf->d_coef2);
    cudaFree(lrf->d_coeft);
    cudaFree(lrf->d_coef2_pf);
    cudaFree(lrf->d_set_of);
    cudaFree(lrf->d_op_of);
    cudaFree(lrf->d_rpoly);
    delete lrf;
    (void)cudaGetLastError();
}

}  // extern "C"

namespace ants {

int lrf_create_impl(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int, const double *lo,
                    const double *hi, int shared, const double *coef_host, const double *gain_host, int n_int_r,
                    double hi_r, int n_planes, ants_lrf **out, int n_groups, const int *group, const int *op,
                    const double *centre)
{
    *out = nullptr;
    if (op && (type != ANTS_LRF_XY || !group || !centre))
        return fail(ANTS_E_ARG, "ants_lrf_create_symmetric: symmetry classes need an XY LRF, classes and a centre");
    if (op)
        for (int i = 0; det && i < det->n_s; ++i)
            if (op[i] < 0 || op[i] > 23) return fail(ANTS_E_ARG, "ants_lrf_create_symmetric: operation %d", op[i]);
    if (group) {
        if ((type != ANTS_LRF_RADIAL && !op) || shared || !det)
            return fail(ANTS_E_ARG, "groups need a RADIAL LRF that is not shared, or XY symmetry classes");
        if (n_groups < 1 || n_groups > det->n_s)
            return fail(ANTS_E_ARG, "ants_lrf_create_grouped: 1 <= n_groups <= n_sensors");
        for (int i = 0; i < det->n_s; ++i)
            if (group[i] < 0 || group[i] >= n_groups)
                return fail(ANTS_E_ARG, "ants_lrf_create_grouped: sensor %d in group %d of %d", i, group[i], n_groups);
    }
    if (!ctx || !det || !n_int || !lo || !hi || !coef_host)
        return fail(ANTS_E_ARG, "ants_lrf_create: NULL argument");
    if (type < ANTS_LRF_RADIAL || type > ANTS_LRF_SLICED)
        return fail(ANTS_E_ARG, "ants_lrf_create: unknown LRF type %d", type);
    if (shared && type != ANTS_LRF_RADIAL)
        return fail(ANTS_E_ARG, "ants_lrf_create: shared coefficients need a RADIAL LRF");
    if (gain_host && type != ANTS_LRF_RADIAL && !op)
        return fail(ANTS_E_ARG, "ants_lrf_create: gains apply to RADIAL LRFs and XY symmetry classes only");
    int dims = lrf_dims(type);
    if (type == ANTS_LRF_COMPOSITE && (n_int_r < 1 || n_int_r > 256 || !(hi_r > 0.0) || !std::isfinite(hi_r)))
        return fail(ANTS_E_ARG, "ants_lrf_create: a composite LRF needs 1 <= n_int_r <= 256 and hi_r > 0");
    if (type == ANTS_LRF_SLICED &&
        (n_planes < 2 || n_planes > 64 || !(lo[2] < hi[2]) || !std::isfinite(lo[2]) || !std::isfinite(hi[2])))
        return fail(ANTS_E_ARG, "ants_lrf_create: a sliced LRF needs 2..64 planes and a z range lo[2] < hi[2]");
    ants_lrf *L = new (std::nothrow) ants_lrf();
    if (!L) return fail(ANTS_E_OOM, "ants_lrf_create: out of host memory");
    L->ctx = ctx;
    L->device = ctx->device;
    L->type = type;
    L->n_s = det->n_s;
    L->shared = shared ? 1 : 0;
    L->n_coef = 1;
    for (int a = 0; a < dims; ++a) {
        if (n_int[a] < 1 || n_int[a] > 256 || !(lo[a] < hi[a]) || !std::isfinite(lo[a]) ||
            !std::isfinite(hi[a])) {
            delete L;
            return fail(ANTS_E_ARG, "ants_lrf_create: axis %d needs 1 <= n_int <= 256, lo < hi", a);
        }
        L->n_int[a] = n_int[a];
        L->lo[a] = lo[a];
        L->hi[a] = hi[a];
        L->n_coef *= n_int[a] + 3;
    }
    if ((type == ANTS_LRF_RADIAL || type == ANTS_LRF_AXIAL_Z) && lo[0] != 0.0) {
        delete L;
        return fail(ANTS_E_ARG, "ants_lrf_create: an axial LRF starts at r = 0");
    }
    if (type == ANTS_LRF_COMPOSITE) {
        L->n_int_r = n_int_r;
        L->hi_r = hi_r;
        L->n_coef += n_int_r + 3;
    }
    if (type == ANTS_LRF_SLICED) {
        L->n_planes = n_planes;
        L->lo[2] = lo[2];
        L->hi[2] = hi[2];
        L->n_coef *= n_planes;
    }
    L->n_sets = L->shared ? 1 : group ? n_groups : L->n_s;
    if (group) L->groups.assign(group, group + L->n_s);
    if (op) {
        L->ops.assign(op, op + L->n_s);
        L->sym_c[0] = centre[0];
        L->sym_c[1] = centre[1];
    }
    size_t nc = (size_t)L->n_sets * L->n_coef;
    L->coef.assign(coef_host, coef_host + nc);
    for (size_t k = 0; k < nc; ++k)
        if (!std::isfinite(L->coef[k])) {
            delete L;
            return fail(ANTS_E_ARG, "ants_lrf_create: coefficient %zu not finite", k);
        }
    L->gain.assign(L->n_s, 1.0);
    if (gain_host) L->gain.assign(gain_host, gain_host + L->n_s);
    L->sxy = det->xy;
    L->rel_gain = det->gain;
    int rc = upload_lrf(L);
    if (rc != ANTS_OK) {
        std::string keep = t_err;
        ants_lrf_free(L);
        t_err = keep;
        return rc;
    }
    *out = L;
    return ANTS_OK;
}

}  // namespace ants

extern "C" {

ANTS_API int ants_lrf_create(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                             const double *lo, const double *hi, int shared,
                             const double *coef_host, const double *gain_host, ants_lrf **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_create: out is NULL");
    *out = nullptr;
    if (type != ANTS_LRF_RADIAL && type != ANTS_LRF_XY && type != ANTS_LRF_XYZ)
        return fail(ANTS_E_ARG, "ants_lrf_create: type %d (the other schemes: ants_lrf_create_scheme)", type);
    return lrf_create_impl(ctx, det, type, n_int, lo, hi, shared, coef_host, gain_host, 0, 0.0, 0, out);
}

ANTS_API int ants_lrf_create_grouped(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo,
                                     const double *hi, int n_groups, const int *group_host, const double *coef_host,
                                     const double *gain_host, ants_lrf **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_create_grouped: out is NULL");
    *out = nullptr;
    if (!group_host) return fail(ANTS_E_ARG, "ants_lrf_create_grouped: group_host is NULL");
    return lrf_create_impl(ctx, det, ANTS_LRF_RADIAL, n_int, lo, hi, 0, coef_host, gain_host, 0, 0.0, 0, out, n_groups,
                           group_host);
}

ANTS_API int ants_lrf_create_symmetric(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo,
                                       const double *hi, int n_classes, const int *class_host, const int *op_host,
                                       const double *centre, const double *coef_host, const double *gain_host,
                                       ants_lrf **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_create_symmetric: out is NULL");
    *out = nullptr;
    if (!class_host || !op_host || !centre) return fail(ANTS_E_ARG, "ants_lrf_create_symmetric: NULL argument");
    return lrf_create_impl(ctx, det, ANTS_LRF_XY, n_int, lo, hi, 0, coef_host, gain_host, 0, 0.0, 0, out, n_classes,
                           class_host, op_host, centre);
}

ANTS_API int ants_sensor_symmetry(const ants_detector *det, double tol, int *class_host, int *op_host,
                                  double *centre_out, int *n_classes_out)
{
    begin_call();
    if (!det || !class_host || !op_host || !centre_out || !n_classes_out)
        return fail(ANTS_E_ARG, "ants_sensor_symmetry: NULL argument");
    if (!(tol >= 0.0)) return fail(ANTS_E_ARG, "ants_sensor_symmetry: tol must be >= 0");
    const int n = det->n_s;
    double cx = 0.0, cy = 0.0;
    for (int i = 0; i < n; ++i) {
        cx += det->xy[2 * i];
        cy += det->xy[2 * i + 1];
    }
    cx /= n;
    cy /= n;
    double M[24][4];
    for (int k = 0; k < 24; ++k) {
        const double t = (double)(k % 12) * (3.14159265358979323846 / 6.0);
        double c = std::cos(t), sn = std::sin(t);
        if (k % 3 == 0) {
            const int q = (k % 12) / 3;
            c = q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
            sn = q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
        }
        const double f = k >= 12 ? -1.0 : 1.0;
        M[k][0] = c;
        M[k][1] = -sn * f;
        M[k][2] = sn;
        M[k][3] = c * f;
    }
    auto image = [&](int k, int i, double &x, double &y) {
        const double dx = det->xy[2 * i] - cx, dy = det->xy[2 * i + 1] - cy;
        x = M[k][0] * dx + M[k][1] * dy + cx;
        y = M[k][2] * dx + M[k][3] * dy + cy;
    };
    std::vector<int> valid;
    for (int k = 0; k < 24; ++k) {
        bool ok = true;
        for (int i = 0; i < n && ok; ++i) {
            double x, y;
            image(k, i, x, y);
            bool hit = false;
            for (int j = 0; j < n && !hit; ++j) hit = std::hypot(det->xy[2 * j] - x, det->xy[2 * j + 1] - y) <= tol;
            ok = hit;
        }
        if (ok) valid.push_back(k);
    }
    for (int i = 0; i < n; ++i) class_host[i] = -1;
    int g = 0;
    for (int r = 0; r < n; ++r) {
        if (class_host[r] >= 0) continue;
        for (int k : valid) {
            double x, y;
            image(k, r, x, y);
            for (int j = 0; j < n; ++j)
                if (class_host[j] < 0 && std::hypot(det->xy[2 * j] - x, det->xy[2 * j + 1] - y) <= tol) {
                    class_host[j] = g;
                    op_host[j] = k;
                    break;
                }
        }
        ++g;
    }
    centre_out[0] = cx;
    centre_out[1] = cy;
    *n_classes_out = g;
    return ANTS_OK;
}

ANTS_API int ants_sensor_rings(const ants_detector *det, double tol, int *group_host, int *n_groups_out)
{
    begin_call();
    if (!det || !group_host || !n_groups_out) return fail(ANTS_E_ARG, "ants_sensor_rings: NULL argument");
    if (!(tol >= 0.0)) return fail(ANTS_E_ARG, "ants_sensor_rings: tol must be >= 0");
    const int n = det->n_s;
    double cx = 0.0, cy = 0.0;
    for (int i = 0; i < n; ++i) {
        cx += det->xy[2 * i];
        cy += det->xy[2 * i + 1];
    }
    cx /= n;
    cy /= n;
    std::vector<double> d(n);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) {
        d[i] = std::hypot(det->xy[2 * i] - cx, det->xy[2 * i + 1] - cy);
        order[i] = i;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
    int g = -1;
    double first = 0.0;
    for (int i : order) {
        if (g < 0 || d[i] - first > tol) {
            ++g;
            first = d[i];
        }
        group_host[i] = g;
    }
    *n_groups_out = g + 1;
    return ANTS_OK;
}

ANTS_API int ants_lrf_create_scheme(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                    const double *lo, const double *hi, int n_int_r, double hi_r, int n_planes,
                                    const double *coef_host, ants_lrf **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_create_scheme: out is NULL");
    *out = nullptr;
    if (type != ANTS_LRF_COMPOSITE && type != ANTS_LRF_AXIAL_Z && type != ANTS_LRF_SLICED)
        return fail(ANTS_E_ARG, "ants_lrf_create_scheme: type %d is not a composite, axial+z or sliced LRF", type);
    return lrf_create_impl(ctx, det, type, n_int, lo, hi, 0, coef_host, nullptr, n_int_r, hi_r, n_planes, out);
}

ANTS_API int ants_lrf_coefficients(const ants_lrf *lrf, double *coef_host, size_t count,
                                   int *n_sets_out, int *n_coef_out)
{
    begin_call();
    if (!lrf) return fail(ANTS_E_ARG, "ants_lrf_coefficients: lrf is NULL");
    if (n_sets_out) *n_sets_out = lrf->n_sets;
    if (n_coef_out) *n_coef_out = lrf->n_coef;
    if (!coef_host) return ANTS_OK;
    if (count < lrf->coef.size())
        return fail(ANTS_E_ARG, "ants_lrf_coefficients: capacity %zu < %zu", count, lrf->coef.size());
    std::memcpy(coef_host, lrf->coef.data(), lrf->coef.size() * sizeof(double));
    return ANTS_OK;
}

ANTS_API int ants_lrf_gains(const ants_lrf *lrf, double *gain_host, size_t count)
{
    begin_call();
    if (!lrf || !gain_host) return fail(ANTS_E_ARG, "ants_lrf_gains: NULL argument");
    if (count < (size_t)lrf->n_s) return fail(ANTS_E_ARG, "ants_lrf_gains: capacity %zu < %d", count, lrf->n_s);
    std::memcpy(gain_host, lrf->gain.data(), lrf->n_s * sizeof(double));
    return ANTS_OK;
}

// eta_i at arbitrary points: one thread per (point, sensor)
__global__ void lrf_eval_kernel(LrfDev L, const float *pts, long n_pts, int dim, float *out)
{
    long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = n_pts * L.n_s;
    for (; tid < total; tid += (long)gridDim.x * blockDim.x) {
        long p = tid / L.n_s;
        int i = (int)(tid - p * L.n_s);
        float x = pts[p * dim], y = pts[p * dim + 1], z = dim > 2 ? pts[p * dim + 2] : 0.0f;
        bool ok;
        float v = lrf_eta_point(L, i, x, y, z, ok);
        out[tid] = ok ? v : __int_as_float(0x7fc00000);
    }
}

ANTS_API int ants_lrf_eval(const ants_lrf *lrf, const float *pts_dev, long n_pts, int dim,
                           float *out_dev, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_lrf_eval");
    if (!lrf) return fail(ANTS_E_ARG, "ants_lrf_eval: lrf is NULL");
    if (n_pts < 0) return fail(ANTS_E_ARG, "ants_lrf_eval: n_pts < 0");
    int need = lrf_is_3d(lrf->type) ? 3 : 2;
    if (dim != need) return fail(ANTS_E_SHAPE, "ants_lrf_eval: dim %d, LRF needs %d", dim, need);
    if (n_pts == 0) return ANTS_OK;
    if (!pts_dev || !out_dev) return fail(ANTS_E_ARG, "ants_lrf_eval: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(lrf->ctx->device), "cudaSetDevice");
    long total = n_pts * lrf->n_s;
    long blocks = (total + 255) / 256;
    long cap = (long)lrf->ctx->n_sm * 16;
    if (blocks > cap) blocks = cap;
    lrf_eval_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(lrf->dev, pts_dev, n_pts, dim,
                                                                          out_dev);
    ANTS_CUDA_TRY(cudaGetLastError(), "lrf_eval_kernel launch");
    count_launch();
    return ANTS_OK;
}

// --- save / load ------------------------------------------------------------

static const char kMagic[8] = {'A', 'N', 'T', 'S', 'L', 'R', 'F', '1'};

ANTS_API int ants_lrf_save(const ants_lrf *lrf, const char *path)
{
    begin_call();
    if (!lrf || !path) return fail(ANTS_E_ARG, "ants_lrf_save: NULL argument");
    if (lrf->type > ANTS_LRF_XYZ || !lrf->groups.empty())
        return fail(ANTS_E_UNIMPLEMENTED, "ants_lrf_save: ungrouped RADIAL, XY and XYZ sets only");
    FILE *f = fopen(path, "wb");
    if (!f) return fail(ANTS_E_IO, "ants_lrf_save: cannot open %s", path);
    int32_t hdr[8] = {1, lrf->type, lrf->n_s, lrf->shared, lrf->n_int[0], lrf->n_int[1], lrf->n_int[2],
                      lrf->n_coef};
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int32_t), 8, f) == 8 &&
              fwrite(lrf->lo, sizeof(double), 3, f) == 3 && fwrite(lrf->hi, sizeof(double), 3, f) == 3 &&
              fwrite(lrf->gain.data(), sizeof(double), lrf->n_s, f) == (size_t)lrf->n_s &&
              fwrite(lrf->coef.data(), sizeof(double), lrf->coef.size(), f) == lrf->coef.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) return fail(ANTS_E_IO, "ants_lrf_save: write to %s failed", path);
    return ANTS_OK;
}

ANTS_API int ants_lrf_load(ants_ctx *ctx, const ants_detector *det, const char *path, ants_lrf **out)
{
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_load: out is NULL");
    *out = nullptr;
    if (!ctx || !det || !path) return fail(ANTS_E_ARG, "ants_lrf_load: NULL argument");
    FILE *f = fopen(path, "rb");
    if (!f) return fail(ANTS_E_IO, "ants_lrf_load: cannot open %s", path);
    char magic[8];
    int32_t hdr[8];
    double lo[3], hi[3];
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kMagic, 8) == 0 &&
              fread(hdr, sizeof(int32_t), 8, f) == 8 && hdr[0] == 1 &&
              fread(lo, sizeof(double), 3, f) == 3 && fread(hi, sizeof(double), 3, f) == 3;
    if (!ok) { fclose(f); return fail(ANTS_E_IO, "ants_lrf_load: %s is not an LRF file", path); }
    int type = hdr[1], n_s = hdr[2], shared = hdr[3];
    if (n_s != det->n_s) {
        fclose(f);
        return fail(ANTS_E_SHAPE, "ants_lrf_load: file has %d sensors, detector %d", n_s, det->n_s);
    }
    int n_int[3] = {hdr[4], hdr[5], hdr[6]};
    int dims = (type == ANTS_LRF_RADIAL) ? 1 : (type == ANTS_LRF_XY ? 2 : (type == ANTS_LRF_XYZ ? 3 : 0));
    long nc = 1;
    for (int a = 0; a < dims; ++a) nc *= (n_int[a] >= 1 && n_int[a] <= 256) ? n_int[a] + 3 : -1000000;
    if (dims == 0 || nc != hdr[7] || nc <= 0) {
        fclose(f);
        return fail(ANTS_E_IO, "ants_lrf_load: %s has an inconsistent header", path);
    }
    std::vector<double> gain(n_s), coef((size_t)(shared ? 1 : n_s) * nc);
    ok = fread(gain.data(), sizeof(double), n_s, f) == (size_t)n_s &&
         fread(coef.data(), sizeof(double), coef.size(), f) == coef.size();
    fclose(f);
    if (!ok) return fail(ANTS_E_IO, "ants_lrf_load: %s is truncated", path);
    return ants_lrf_create(ctx, det, type, n_int, lo, hi, shared, coef.data(),
                           type == ANTS_LRF_RADIAL ? gain.data() : nullptr, out);
}

// ---------------------------------------------------------------------------
// reconstruction entry points
// ---------------------------------------------------------------------------

static int check_common(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params,
                        int signal_dtype, long n_events, int n_sensors)
{
    if (!ctx || !lrf || !params) return fail(ANTS_E_ARG, "ants_reconstruct: NULL ctx, lrf or params");
    if (lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_reconstruct: lrf belongs to another context");
    if (n_events < 0) return fail(ANTS_E_ARG, "ants_reconstruct: n_events < 0");
    if (n_sensors != lrf->n_s)
        return fail(ANTS_E_SHAPE, "ants_reconstruct: n_sensors %d but the LRF has %d", n_sensors, lrf->n_s);
    if (signal_dtype != ANTS_F32 && signal_dtype != ANTS_F16)
        return fail(ANTS_E_ARG, "ants_reconstruct: signal dtype %d", signal_dtype);
    if (method == ANTS_MLP_SEEDED) return check_seeded_params(lrf, (const ants_mlp_seeded_params *)params);
    if (method == ANTS_GEMM_TOPK) return check_gemm_params(lrf, (const ants_gemm_params *)params);
    if (method == ANTS_CGS_VARIANT) return check_variant_params(lrf, (const ants_cgs_variant_params *)params);
    if (method == ANTS_MINIMIZE) return check_minimize_params(lrf, (const ants_minimize_params *)params);
    if (method != ANTS_CGS_PLAIN) return fail(ANTS_E_UNIMPLEMENTED, "ants_reconstruct: method %d", method);
    return check_cgs_params(lrf, (const ants_cgs_params *)params);
}

static int reconstruct_f32(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params, const float *sig,
                           long n_events, const float *start_xyz_dev, float *xyz_dev, float *E_dev, float *logL_dev,
                           int32_t *status_dev, int16_t *trace_dev, cudaStream_t stream)
{
    if (method == ANTS_GEMM_TOPK)
        return reconstruct_gemm_topk(ctx, lrf, *(const ants_gemm_params *)params, sig, n_events, xyz_dev, E_dev,
                                     logL_dev, status_dev, stream);
    if (method == ANTS_MLP_SEEDED)
        return reconstruct_mlp_seeded(ctx, lrf, *(const ants_mlp_seeded_params *)params, sig, n_events, xyz_dev,
                                      E_dev, logL_dev, status_dev, trace_dev, stream);
    if (method == ANTS_CGS_VARIANT)
        return reconstruct_variant(ctx, lrf, *(const ants_cgs_variant_params *)params, sig, n_events, nullptr,
                                   xyz_dev, E_dev, logL_dev, status_dev, trace_dev, stream);
    if (method == ANTS_MINIMIZE)
        return reconstruct_minimize(ctx, lrf, *(const ants_minimize_params *)params, sig, n_events, start_xyz_dev,
                                    xyz_dev, E_dev, logL_dev, status_dev, trace_dev, stream);
    return launch_cgs_plain(ctx, lrf, *(const ants_cgs_params *)params, sig, n_events, start_xyz_dev, xyz_dev, E_dev,
                            logL_dev, status_dev, trace_dev, stream);
}

static int reconstruct_device(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params,
                              const void *signals_dev, int signal_dtype, long n_events, int n_sensors,
                              const float *start_xyz_dev, float *xyz_dev, float *E_dev, float *logL_dev,
                              int32_t *status_dev, int16_t *trace_dev, void *stream)
{
    int rc = check_common(ctx, lrf, method, params, signal_dtype, n_events, n_sensors);
    if (rc != ANTS_OK) return rc;
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !xyz_dev || !E_dev || !logL_dev || !status_dev)
        return fail(ANTS_E_ARG, "ants_reconstruct: NULL signal or output buffer");
    if (method == ANTS_GEMM_TOPK && (start_xyz_dev || trace_dev))
        return fail(ANTS_E_ARG, "ants_reconstruct: the precision form takes no start or trace");
    if (method == ANTS_MLP_SEEDED && start_xyz_dev)
        return fail(ANTS_E_ARG, "ants_reconstruct: the learned form proposes its own start");
    if (method == ANTS_CGS_VARIANT && start_xyz_dev)
        return fail(ANTS_E_ARG, "ants_reconstruct: a search variant picks its own start");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (signal_dtype == ANTS_F32)
        return reconstruct_f32(ctx, lrf, method, params, (const float *)signals_dev, n_events, start_xyz_dev, xyz_dev,
                               E_dev, logL_dev, status_dev, trace_dev, s);
    // FP16 signals: widen chunk by chunk into scratch slot 7 (no other user)
    const int iters = method == ANTS_CGS_PLAIN     ? ((const ants_cgs_params *)params)->iters
                      : method == ANTS_MLP_SEEDED  ? ((const ants_mlp_seeded_params *)params)->refine.iters
                      : method == ANTS_CGS_VARIANT ? ((const ants_cgs_variant_params *)params)->grid.iters
                      : method == ANTS_MINIMIZE    ? 1
                                                   : 0;
    const long chunk = n_events < (1L << 20) ? n_events : (1L << 20);
    float *wide = (float *)ctx_scratch(ctx, 7, (size_t)chunk * n_sensors * sizeof(float));
    if (!wide) return ANTS_E_OOM;
    const __half *h = (const __half *)signals_dev;
    for (long off = 0; off < n_events; off += chunk) {
        const long n = n_events - off < chunk ? n_events - off : chunk;
        rc = widen_half(h + (size_t)off * n_sensors, (size_t)n * n_sensors, wide, s);
        if (rc != ANTS_OK) return rc;
        rc = reconstruct_f32(ctx, lrf, method, params, wide, n, start_xyz_dev ? start_xyz_dev + 3 * off : nullptr,
                             xyz_dev + 3 * off, E_dev + off, logL_dev + off, status_dev + off,
                             trace_dev ? trace_dev + (size_t)off * iters : nullptr, s);
        if (rc != ANTS_OK) return rc;
    }
    return ANTS_OK;
}

ANTS_API int ants_reconstruct(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params,
                              const void *signals_dev, int signal_dtype, long n_events, int n_sensors,
                              const float *start_xyz_dev, float *xyz_dev, float *E_dev, float *logL_dev,
                              int32_t *status_dev, int16_t *trace_dev, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_reconstruct");
    int rc = reconstruct_device(ctx, lrf, method, params, signals_dev, signal_dtype, n_events, n_sensors,
                                start_xyz_dev, xyz_dev, E_dev, logL_dev, status_dev, trace_dev, stream);
    if (rc == ANTS_OK && ctx && n_events > 0) rc = check_bounds(ctx, (cudaStream_t)stream);
    return rc;
}

ANTS_API int ants_reconstruct_host(ants_ctx *ctx, const ants_lrf *lrf, int method, const void *params,
                                   const void *signals_host, int signal_dtype, long n_events,
                                   int n_sensors, const float *start_xyz_host, float *xyz_host,
                                   float *E_host, float *logL_host, int32_t *status_host)
{
    begin_call();
    ANTS_NVTX("ants_reconstruct_host");
    int rc = check_common(ctx, lrf, method, params, signal_dtype, n_events, n_sensors);
    if (rc != ANTS_OK) return rc;
    if (n_events == 0) return ANTS_OK;
    if (!signals_host || !xyz_host || !E_host || !logL_host || !status_host)
        return fail(ANTS_E_ARG, "ants_reconstruct_host: NULL signal or output buffer");
    if (method != ANTS_CGS_PLAIN && method != ANTS_MINIMIZE && start_xyz_host)
        return fail(ANTS_E_ARG, "ants_reconstruct_host: only the plain search and the minimisation take a start");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    // the plain search overlaps chunks on two streams; the two forms use the
    // context's scratch buffers, so their chunks run one after the other
    const bool overlap = method == ANTS_CGS_PLAIN || method == ANTS_CGS_VARIANT || method == ANTS_MINIMIZE;
    // chunk large enough to fill the GPU, small enough to pipeline
    const long chunk = 1L << 17;
    if (ctx->host_cap_events < (size_t)chunk || ctx->host_cap_sensors < n_sensors) {
        free_host_buffers(ctx);
        for (int k = 0; k < 2; ++k) {
            // FP32 chunk, then room for the FP16 copy that is widened into it
            cudaError_t e = cudaMalloc(&ctx->d_sig[k], (size_t)chunk * n_sensors * (sizeof(float) + sizeof(__half)));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->d_start[k], (size_t)chunk * 3 * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->d_out[k], (size_t)chunk * 5 * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status[k], (size_t)chunk * sizeof(int32_t));
            if (e != cudaSuccess) {
                free_host_buffers(ctx);
                return fail(ANTS_E_OOM, "ants_reconstruct_host: device buffers: %s", cudaGetErrorString(e));
            }
        }
        ctx->host_cap_events = chunk;
        ctx->host_cap_sensors = n_sensors;
    }
    for (long off = 0, c = 0; off < n_events; off += chunk, ++c) {
        int k = overlap ? (int)(c & 1) : 0;
        cudaStream_t s = ctx->stream[k];
        long n = n_events - off < chunk ? n_events - off : chunk;
        if (signal_dtype == ANTS_F32) {
            const float *sig = (const float *)signals_host + off * n_sensors;
            ANTS_CUDA_TRY(cudaMemcpyAsync(ctx->d_sig[k], sig, (size_t)n * n_sensors * sizeof(float),
                                          cudaMemcpyHostToDevice, s), "H2D signals");
        } else {
            const __half *sig = (const __half *)signals_host + off * n_sensors;
            __half *stage = (__half *)((float *)ctx->d_sig[k] + (size_t)chunk * n_sensors);
            ANTS_CUDA_TRY(cudaMemcpyAsync(stage, sig, (size_t)n * n_sensors * sizeof(__half), cudaMemcpyHostToDevice,
                                          s), "H2D signals");
            rc = widen_half(stage, (size_t)n * n_sensors, (float *)ctx->d_sig[k], s);
            if (rc != ANTS_OK) return rc;
        }
        if (start_xyz_host)
            ANTS_CUDA_TRY(cudaMemcpyAsync(ctx->d_start[k], start_xyz_host + off * 3, (size_t)n * 3 * sizeof(float),
                                          cudaMemcpyHostToDevice, s), "H2D start");
        float *o = ctx->d_out[k];
        rc = reconstruct_f32(ctx, lrf, method, params, (const float *)ctx->d_sig[k], n,
                             start_xyz_host ? ctx->d_start[k] : nullptr, o, o + 3 * chunk, o + 4 * chunk,
                             ctx->d_status[k], nullptr, s);
        if (rc != ANTS_OK) return rc;
        ANTS_CUDA_TRY(cudaMemcpyAsync(xyz_host + off * 3, o, (size_t)n * 3 * sizeof(float),
                                      cudaMemcpyDeviceToHost, s), "D2H xyz");
        ANTS_CUDA_TRY(cudaMemcpyAsync(E_host + off, o + 3 * chunk, (size_t)n * sizeof(float),
                                      cudaMemcpyDeviceToHost, s), "D2H E");
        ANTS_CUDA_TRY(cudaMemcpyAsync(logL_host + off, o + 4 * chunk, (size_t)n * sizeof(float),
                                      cudaMemcpyDeviceToHost, s), "D2H logL");
        ANTS_CUDA_TRY(cudaMemcpyAsync(status_host + off, ctx->d_status[k], (size_t)n * sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s), "D2H status");
    }
    ANTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream[0]), "stream 0");
    ANTS_CUDA_TRY(cudaStreamSynchronize(ctx->stream[1]), "stream 1");
    return ANTS_OK;
}

}  // extern "C"
