// Learned-proposal reconstruction and the Poisson deviance.
//
//   1. the network proposes (x, y) from the sum-normalised signals;
//   2. a small contracting-grid search (Sec. 5.1.2.2) refines it;
//   3. events whose Poisson deviance D = 2 sum[s ln(s/mu) - (s - mu)] exceeds
//      a threshold, or whose final node lies on the border of the last refine
//      grid (the optimum may lie outside it), are flagged -- the chi-squared
//      style event filter of Sec. 5.2 used as a trigger;
//   4. the flagged events are gathered and re-run with the plain search, and
//      their results scattered back with status ANTS_EVT_FALLBACK.
#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;

// s ln s - s - lgamma(s+1), s > 0 (Stirling series for s >= 10, A&S 6.1.41)
__device__ __forceinline__ float saturated_term(float s)
{
    if (s >= 10.0f) {
        float r = 1.0f / s, r2 = r * r;
        float series = r * (-1.0f / 12.0f + r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
        return -0.5f * logf(6.283185307179586f * s) + series;
    }
    return s * logf(s) - s - lgammaf(s + 1.0f);
}

__device__ __forceinline__ float wsum(float v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// one warp per event: D = 2 (logL_saturated - logL); flag for the fallback
__global__ void flag_kernel(const float *__restrict__ sig, long n, int n_s, const float *__restrict__ logL,
                            const int32_t *__restrict__ status, const int16_t *__restrict__ trace, int iters,
                            int n_xy, float dev_max, int border, int *__restrict__ count, long *__restrict__ idx)
{
    const long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n) return;
    float c = 0.0f;
    for (int i = lane; i < n_s; i += 32) {
        const float s = sig[e * n_s + i];
        if (s > 0.0f) c += saturated_term(s);
    }
    c = wsum(c);
    if (lane != 0) return;
    const int st = status[e];
    if (st == ANTS_EVT_ZERO_SIGNAL || st == ANTS_EVT_BAD_SIGNAL) return;  // no search can help
    const float D = 2.0f * (c - logL[e]);
    // a start the refine could not use (outside the domain) also goes to the plain search
    bool f = st == ANTS_EVT_OUT_OF_DOMAIN || (dev_max > 0.0f && D > dev_max);
    if (border && trace && st == ANTS_EVT_OK) {
        const int k = trace[e * iters + iters - 1];
        const int ix = k % n_xy, iy = (k / n_xy) % n_xy;
        f = f || ix == 0 || ix == n_xy - 1 || iy == 0 || iy == n_xy - 1;
    }
    if (f) idx[atomicAdd(count, 1)] = e;
}

__global__ void gather_rows(const float *__restrict__ sig, const long *__restrict__ idx, long m, int n_s,
                            float *__restrict__ out)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * n_s) return;
    const long r = t / n_s;
    out[t] = sig[idx[r] * n_s + (t - r * n_s)];
}

__global__ void scatter_results(const long *__restrict__ idx, long m, const float *__restrict__ xyz_s,
                                const float *__restrict__ E_s, const float *__restrict__ logL_s,
                                const int32_t *__restrict__ st_s, float *__restrict__ xyz, float *__restrict__ E,
                                float *__restrict__ logL, int32_t *__restrict__ status)
{
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const long e = idx[r];
    xyz[3 * e] = xyz_s[3 * r];
    xyz[3 * e + 1] = xyz_s[3 * r + 1];
    xyz[3 * e + 2] = xyz_s[3 * r + 2];
    E[e] = E_s[r];
    logL[e] = logL_s[r];
    status[e] = st_s[r] == ANTS_EVT_OK ? ANTS_EVT_FALLBACK : st_s[r];
}

// one warp per event: Poisson deviance at a given position, E = S/H
__global__ void deviance_kernel(LrfDev L, const float *__restrict__ sig, long n, const float *__restrict__ xyz,
                                float *__restrict__ D)
{
    const long e = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= n) return;
    const float x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2];
    float S = 0.0f, H = 0.0f;
    bool inside = true;
    for (int i = lane; i < L.n_s; i += 32) {
        bool ok;
        const float v = lrf_eta_point(L, i, x, y, z, ok);
        inside = inside && ok;
        S += sig[e * L.n_s + i];
        H += fmaxf(v, kEtaFloor);
    }
    S = wsum(S);
    H = wsum(H);
    inside = __all_sync(kFull, inside);
    const float En = S / H;
    float d = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) {
        bool ok;
        const float mu = En * fmaxf(lrf_eta_point(L, i, x, y, z, ok), kEtaFloor);
        const float s = sig[e * L.n_s + i];
        d += s > 0.0f ? fmaf(s, logf(s / mu), mu - s) : mu;
    }
    d = wsum(d);
    if (lane == 0) D[e] = inside ? 2.0f * d : __int_as_float(0x7fc00000);
}

// keep network proposals inside the XY box of the LRF (as the centroid start is)
__global__ void clamp_seeds(float *__restrict__ xyz, long n, float lx, float hx, float ly, float hy)
{
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    xyz[3 * r] = fminf(fmaxf(xyz[3 * r], lx), hx);
    xyz[3 * r + 1] = fminf(fmaxf(xyz[3 * r + 1], ly), hy);
}

unsigned nblocks(long n, int per) { return (unsigned)((n + per - 1) / per); }

}  // namespace

int check_seeded_params(const ants_lrf *lrf, const ants_mlp_seeded_params *P)
{
    if (!P || !P->mlp) return fail(ANTS_E_ARG, "learned form: NULL params or network");
    if (mlp_n_in(P->mlp) != lrf->n_s)
        return fail(ANTS_E_SHAPE, "learned form: network takes %d inputs, the LRF has %d sensors",
                    mlp_n_in(P->mlp), lrf->n_s);
    if (lrf->type != ANTS_LRF_XY && lrf->type != ANTS_LRF_RADIAL)
        return fail(ANTS_E_UNIMPLEMENTED, "learned form: RADIAL and XY LRFs only");
    int rc = check_cgs_params(lrf, &P->refine);
    if (rc != ANTS_OK) return rc;
    return check_cgs_params(lrf, &P->fallback);
}

int reconstruct_mlp_seeded(ants_ctx *ctx, const ants_lrf *lrf, const ants_mlp_seeded_params &P, const float *sig,
                           long n, float *xyz, float *E, float *logL, int32_t *status, int16_t *trace,
                           cudaStream_t s)
{
    const int n_s = lrf->n_s;
    float *O = (float *)ctx_scratch(ctx, 1, (size_t)n * 3 * sizeof(float));
    float *seeds = (float *)ctx_scratch(ctx, 2, (size_t)n * 3 * sizeof(float));
    int16_t *tr = trace ? trace : (int16_t *)ctx_scratch(ctx, 3, (size_t)n * P.refine.iters * sizeof(int16_t));
    unsigned char *cl = (unsigned char *)ctx_scratch(ctx, 4, 256 + (size_t)n * sizeof(long));
    if (!O || !seeds || !tr || !cl) return ANTS_E_OOM;
    int *d_count = (int *)cl;
    long *d_idx = (long *)(cl + 256);
    int rc = mlp_forward(ctx, P.mlp, sig, n, P.bf16 != 0, O, s);
    if (rc != ANTS_OK) return rc;
    rc = mlp_decode(P.mlp, O, n, seeds, nullptr, s);
    if (rc != ANTS_OK) return rc;
    if (lrf->type == ANTS_LRF_XY) {
        clamp_seeds<<<nblocks(n, 256), 256, 0, s>>>(seeds, n, lrf->dev.lo[0], lrf->dev.hi[0], lrf->dev.lo[1],
                                                    lrf->dev.hi[1]);
        count_launch();
    }
    rc = launch_cgs_plain(ctx, lrf, P.refine, sig, n, seeds, xyz, E, logL, status, tr, s);
    if (rc != ANTS_OK) return rc;
    ANTS_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int), s), "fallback counter");
    flag_kernel<<<nblocks(n, 8), 256, 0, s>>>(sig, n, n_s, logL, status, tr, P.refine.iters, P.refine.n_xy,
                                              P.deviance_max, P.border_fallback, d_count, d_idx);
    count_launch();
    ANTS_CUDA_TRY(cudaGetLastError(), "flag launch");
    int h_count = 0;
    ANTS_CUDA_TRY(cudaMemcpyAsync(&h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s), "fallback count");
    ANTS_CUDA_TRY(cudaStreamSynchronize(s), "fallback count");
    if (h_count == 0) return ANTS_OK;
    const long m = h_count;
    float *sub = (float *)ctx_scratch(ctx, 5, (size_t)m * n_s * sizeof(float));
    unsigned char *so = (unsigned char *)ctx_scratch(ctx, 6, (size_t)m * 6 * sizeof(float) + 1024);
    if (!sub || !so) return ANTS_E_OOM;
    float *xyz_s = (float *)so;
    float *E_s = xyz_s + 3 * m;
    float *logL_s = E_s + m;
    int32_t *st_s = (int32_t *)(logL_s + m);
    gather_rows<<<nblocks(m * n_s, 256), 256, 0, s>>>(sig, d_idx, m, n_s, sub);
    count_launch();
    rc = launch_cgs_plain(ctx, lrf, P.fallback, sub, m, nullptr, xyz_s, E_s, logL_s, st_s, nullptr, s);
    if (rc != ANTS_OK) return rc;
    scatter_results<<<nblocks(m, 256), 256, 0, s>>>(d_idx, m, xyz_s, E_s, logL_s, st_s, xyz, E, logL, status);
    count_launch();
    ANTS_CUDA_TRY(cudaGetLastError(), "fallback launch");
    return ANTS_OK;
}

}  // namespace ants

extern "C" ANTS_API int ants_deviance(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                                      int n_sensors, const float *xyz_dev, float *D_dev, void *stream)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_deviance");
    if (!ctx || !lrf || lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_deviance: bad ctx or lrf");
    if (n_sensors != lrf->n_s) return fail(ANTS_E_SHAPE, "ants_deviance: n_sensors %d", n_sensors);
    if (n_events < 0) return fail(ANTS_E_ARG, "ants_deviance: n_events < 0");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !xyz_dev || !D_dev) return fail(ANTS_E_ARG, "ants_deviance: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    deviance_kernel<<<nblocks(n_events, 8), 256, 0, (cudaStream_t)stream>>>(lrf->dev, signals_dev, n_events, xyz_dev,
                                                                           D_dev);
    ANTS_CUDA_TRY(cudaGetLastError(), "deviance launch");
    count_launch();
    return ANTS_OK;
}
