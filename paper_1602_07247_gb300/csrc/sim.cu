// Synthetic events from an LRF set: sources uniform in a disk or square (z
// uniform for XYZ LRFs), energy uniform in e0 (1 +- e_spread), and Poisson
// photo-electron counts with mean E eta_i(source) (Sec. 4.2.5 signals; the
// optical transport of Sec. 4.2.3 is summarised by the LRFs), optionally with
// a normal single-photo-electron response.
//
// Random numbers: Philox4x32-10 (philox.cuh) keyed by the seed.  Event e
// draws its source from the block at counter (e_lo, e_hi, 0xFFFFFFFF, 0);
// sensor i of event e consumes the blocks at
// (e_lo, e_hi, i, 0), (e_lo, e_hi, i, 1), ...  Poisson counts: CDF inversion
// below rate 10, Hormann's transformed rejection with squeeze (PTRS, 1993)
// above.  One thread per (event, sensor); results are independent of the
// launch shape.
#include "bspline.cuh"
#include "internal.cuh"
#include "philox.cuh"

namespace ants {

namespace {

struct Philox {
    uint32_t k0, k1, c0, c1, c2, c3;
    uint32_t buf[4];
    int pos;
};

__device__ __forceinline__ float next_u(Philox &s)
{
    if (s.pos == 4) {
        uint32_t c[4] = {s.c0, s.c1, s.c2, s.c3};
        philox10(s.k0, s.k1, c);
        s.buf[0] = c[0];
        s.buf[1] = c[1];
        s.buf[2] = c[2];
        s.buf[3] = c[3];
        s.c3 += 1;
        s.pos = 0;
    }
    return u01(s.buf[s.pos++]);
}

__device__ float poisson(float lam, Philox &s)
{
    if (!(lam > 0.0f)) return 0.0f;
    if (lam < 10.0f) {
        const float u = next_u(s);
        float p = expf(-lam), F = p;
        int k = 0;
        while (u > F && k < 1000) {
            ++k;
            p *= lam / (float)k;
            F += p;
        }
        return (float)k;
    }
    const float slam = sqrtf(lam), loglam = logf(lam);
    const float b = 0.931f + 2.53f * slam, a = -0.059f + 0.02483f * b;
    const float inv_alpha = 1.1239f + 1.1328f / (b - 3.4f), vr = 0.9277f - 3.6224f / (b - 2.0f);
    for (int it = 0; it < 1000; ++it) {
        const float U = next_u(s) - 0.5f, V = next_u(s);
        const float us = 0.5f - fabsf(U);
        const float k = floorf((2.0f * a / us + b) * U + lam + 0.43f);
        if (us >= 0.07f && V <= vr) return k;
        if (k < 0.0f || (us < 0.013f && V > us)) continue;
        if (logf(V) + logf(inv_alpha) - logf(a / (us * us) + b) <= -lam + k * loglam - lgammaf(k + 1.0f)) return k;
    }
    return floorf(lam);
}

struct SimArgs {
    LrfDev L;
    ants_sim_params p;
    uint32_t k0, k1;
    long first, n;
    float *sig, *truth;
};

__global__ void simulate_kernel(SimArgs a)
{
    const long total = a.n * a.L.n_s;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const long r = t / a.L.n_s;
        const int i = (int)(t - r * a.L.n_s);
        const long e = a.first + r;
        const uint32_t elo = (uint32_t)e, ehi = (uint32_t)((unsigned long long)e >> 32);
        uint32_t c[4] = {elo, ehi, 0xFFFFFFFFu, 0u};
        philox10(a.k0, a.k1, c);
        const float u0 = u01(c[0]), u1 = u01(c[1]), u2 = u01(c[2]), u3 = u01(c[3]);
        float x, y;
        if (a.p.region == 0) {
            const float rad = a.p.extent * sqrtf(u0), th = 6.283185307179586f * u1;
            float sn, cs;
            sincosf(th, &sn, &cs);
            x = a.p.cx + rad * cs;
            y = a.p.cy + rad * sn;
        } else {
            x = a.p.cx + a.p.extent * (2.0f * u0 - 1.0f);
            y = a.p.cy + a.p.extent * (2.0f * u1 - 1.0f);
        }
        const float E = a.p.e0 * (1.0f + a.p.e_spread * (2.0f * u2 - 1.0f));
        const float z = lrf_is_3d(a.L.type) ? a.p.z_lo + (a.p.z_hi - a.p.z_lo) * u3 : 0.0f;
        if (i == 0 && a.truth) {
            a.truth[4 * r] = x;
            a.truth[4 * r + 1] = y;
            a.truth[4 * r + 2] = z;
            a.truth[4 * r + 3] = E;
        }
        bool ok;
        const float eta = lrf_eta_point(a.L, i, x, y, z, ok);
        const float lam = ok && eta > 0.0f ? E * eta : 0.0f;
        Philox st{a.k0, a.k1, elo, ehi, (uint32_t)i, 0u, {0, 0, 0, 0}, 4};
        float cnt = poisson(lam, st);
        if (a.p.spe_sigma > 0.0f && cnt > 0.0f) {
            const float ua = next_u(st), ub = next_u(st);
            const float zn = sqrtf(-2.0f * logf(ua)) * cosf(6.283185307179586f * ub);
            cnt = fmaxf(cnt + a.p.spe_sigma * sqrtf(cnt) * zn, 0.0f);
        }
        a.sig[t] = cnt;
    }
}

}  // namespace

}  // namespace ants

extern "C" ANTS_API int ants_simulate_events(ants_ctx *ctx, const ants_lrf *lrf, const ants_sim_params *params,
                                             uint64_t seed, long first_event, long n_events, float *signals_dev,
                                             float *truth_dev, void *stream)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_simulate_events");
    if (!ctx || !lrf || !params || lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_simulate_events: bad arguments");
    if (n_events < 0 || first_event < 0) return fail(ANTS_E_ARG, "ants_simulate_events: negative count");
    const ants_sim_params &p = *params;
    if ((p.region != 0 && p.region != 1) || !(p.extent >= 0.0f) || !(p.e0 > 0.0f) || !(p.e_spread >= 0.0f) ||
        !(p.e_spread < 1.0f) || !(p.spe_sigma >= 0.0f) || !(p.z_hi >= p.z_lo))
        return fail(ANTS_E_ARG, "ants_simulate_events: bad simulation parameters");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev) return fail(ANTS_E_ARG, "ants_simulate_events: NULL signals buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    SimArgs a;
    a.L = lrf->dev;
    a.p = p;
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.first = first_event;
    a.n = n_events;
    a.sig = signals_dev;
    a.truth = truth_dev;
    const long total = n_events * lrf->n_s;
    long blocks = (total + 255) / 256;
    const long cap = (long)ctx->n_sm * 32;
    if (blocks > cap) blocks = cap;
    simulate_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(a);
    ANTS_CUDA_TRY(cudaGetLastError(), "simulate launch");
    count_launch();
    return ANTS_OK;
}
