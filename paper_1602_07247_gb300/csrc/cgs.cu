// Contracting-grid maximum-likelihood search (Sec. 5.1.2, 5.1.2.2), FP32.
//
// One warp reconstructs one event at a time (grid-stride over events):
//   prologue   signals -> S = sum s, centroid (Sec. 5.1.1) -> start, checks
//   per grid   lanes take nodes; each node sums over all sensors
//              s_i log2(eta_i(node) / eta_i(centre)) and eta_i - eta_i(centre);
//              the profiled score is F = sum - S log2(1 + dH / H_centre)
//              (log-likelihood with E = S/H substituted, in log2 units,
//              relative to the grid centre: the ratios stay near 1, where the
//              hardware log2 is accurate, and the dH sum avoids subtracting
//              two large rounded sums); warp-shuffle argmax, ties to the
//              lowest node index.
//   epilogue   E = S/H and the full Poisson logL at the final node.
#include <cfloat>

#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;

struct CgsArgs {
    LrfDev L;
    int n_xy, n_z, iters;
    float shrink, step_xy, step_z, z0;
    const float *sig;
    long n_e;
    const float *start;
    float *xyz, *E, *logL;
    int32_t *status;
    int16_t *trace;
};

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// ln(s!) - (s ln s - s) complement: returns s ln s - s - lgamma(s+1) for s > 0.
// For s >= 10 the Stirling series (Abramowitz & Stegun 6.1.41) avoids the
// cancellation of three large terms; below it lgammaf is accurate enough.
__device__ __forceinline__ float poisson_const(float s)
{
    if (s >= 10.0f) {
        float r = 1.0f / s, r2 = r * r;
        float series = r * (-1.0f / 12.0f + r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
        return -0.5f * logf(6.283185307179586f * s) + series;
    }
    return s * logf(s) - s - lgammaf(s + 1.0f);
}

__device__ __forceinline__ bool node_in_domain_radial(const LrfDev &L, float x, float y)
{
    bool ok = true;
    for (int i = 0; i < L.n_s; ++i) {
        float dx = x - L.sxy[2 * i], dy = y - L.sxy[2 * i + 1];
        ok = ok && sqrtf(fmaf(dx, dx, dy * dy)) <= L.hi[0];
    }
    return ok;
}

template <int TYPE>
__device__ __forceinline__ float eta_floor(const LrfDev &L, int i, float x, float y, float z)
{
    bool ok;
    float v = lrf_eta_point(L, i, x, y, z, ok);
    return fmaxf(v, kEtaFloor);
}

// Score of one node relative to the centre c (log2 units):
// sum_i s_i log2(eta_i / eta_i(c)) - S log2(1 + sum_i (eta_i - eta_i(c)) / H(c)).
template <int TYPE>
__device__ __forceinline__ float node_score(const LrfDev &L, const float *s_sig, const float *s_ic,
                                            const float *s_ec, float S, float inv_hc, float x, float y,
                                            float z)
{
    const int n_s = L.n_s;
    float acc = 0.0f, dH = 0.0f;
    if (TYPE == ANTS_LRF_RADIAL) {
        bool ok = true;
        for (int i = 0; i < n_s; ++i) {
            float dx = x - L.sxy[2 * i], dy = y - L.sxy[2 * i + 1];
            float r = sqrtf(fmaf(dx, dx, dy * dy));
            ok = ok && r <= L.hi[0];
            float eta = fmaxf(radial_eta(L, i, fminf(r, L.hi[0])), kEtaFloor);
            acc = fmaf(s_sig[i], __log2f(eta * s_ic[i]), acc);
            dH += eta - s_ec[i];
        }
        if (!ok) return -INFINITY;
    } else {
        if (!in_box(L, x, y, z)) return -INFINITY;
        float tx, ty, tz = 0.0f, wx[4], wy[4], wz[4] = {1.0f, 0.0f, 0.0f, 0.0f};
        int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
        int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
        int jz = 0;
        bs_weights(tx, wx);
        bs_weights(ty, wy);
        if (TYPE == ANTS_LRF_XYZ) {
            jz = bs_span(z, L.lo[2], L.inv_h[2], L.n_int[2], tz);
            bs_weights(tz, wz);
        }
        const int nz = TYPE == ANTS_LRF_XYZ ? 4 : 1;
        const float *base = L.coef + jz * L.stride_z + jy * L.stride_y + jx;
        for (int i = 0; i < n_s; ++i) {
            const float *c = base + (size_t)i * L.n_coef;
            float f = 0.0f;
#pragma unroll
            for (int cz = 0; cz < nz; ++cz) {
                float fz = 0.0f;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const float *row = c + cz * L.stride_z + b * L.stride_y;
                    float fr = __ldg(row) * wx[0];
                    fr = fmaf(__ldg(row + 1), wx[1], fr);
                    fr = fmaf(__ldg(row + 2), wx[2], fr);
                    fr = fmaf(__ldg(row + 3), wx[3], fr);
                    fz = fmaf(fr, wy[b], fz);
                }
                f = fmaf(fz, wz[cz], f);
            }
            float eta = fmaxf(f, kEtaFloor);
            acc = fmaf(s_sig[i], __log2f(eta * s_ic[i]), acc);
            dH += eta - s_ec[i];
        }
    }
    return acc - S * (log1pf(dH * inv_hc) * 1.4426950408889634f);
}

template <int TYPE>
__global__ void __launch_bounds__(256) cgs_plain_kernel(CgsArgs a)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const LrfDev &L = a.L;
    const int n_s = L.n_s;
    float *s_sig = smem + (size_t)wib * 3 * n_s;
    float *s_ic = s_sig + n_s;  // 1 / eta_i(centre)
    float *s_ec = s_ic + n_s;   // eta_i(centre)
    const int nodes = a.n_xy * a.n_xy * a.n_z;
    const int c_xy = (a.n_xy - 1) / 2, c_z = (a.n_z - 1) / 2;
    const float qnan = __int_as_float(0x7fc00000);

    for (long e = (long)blockIdx.x * wpb + wib; e < a.n_e; e += (long)gridDim.x * wpb) {
        const float *sg = a.sig + e * n_s;
        float S = 0.0f, Sx = 0.0f, Sy = 0.0f, Sw = 0.0f;
        int bad = 0;
        for (int i = lane; i < n_s; i += 32) {
            float v = sg[i];
            bad |= !(v >= 0.0f) || isinf(v);
            s_sig[i] = v;
            float w = v * L.cog_w[i];
            S += v;
            Sx = fmaf(L.sxy[2 * i], w, Sx);
            Sy = fmaf(L.sxy[2 * i + 1], w, Sy);
            Sw += w;
        }
        bad = __any_sync(kFull, bad);
        S = warp_sum(S);
        Sx = warp_sum(Sx);
        Sy = warp_sum(Sy);
        Sw = warp_sum(Sw);
        __syncwarp();
        int st = ANTS_EVT_OK;
        float cx = 0.0f, cy = 0.0f, cz = 0.0f;
        if (bad) st = ANTS_EVT_BAD_SIGNAL;
        else if (!(S > 0.0f)) st = ANTS_EVT_ZERO_SIGNAL;
        if (st == ANTS_EVT_OK) {
            if (a.start) {
                cx = a.start[3 * e];
                cy = a.start[3 * e + 1];
                cz = a.start[3 * e + 2];
            } else {
                cx = Sx / Sw;
                cy = Sy / Sw;
                cz = TYPE == ANTS_LRF_XYZ ? a.z0 : 0.0f;
                if (TYPE != ANTS_LRF_RADIAL) {
                    cx = fminf(fmaxf(cx, L.lo[0]), L.hi[0]);
                    cy = fminf(fmaxf(cy, L.lo[1]), L.hi[1]);
                }
            }
            bool ok = TYPE == ANTS_LRF_RADIAL ? node_in_domain_radial(L, cx, cy) : in_box(L, cx, cy, cz);
            if (!ok) st = ANTS_EVT_OUT_OF_DOMAIN;
        }
        if (st != ANTS_EVT_OK) {
            if (lane == 0) {
                a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = qnan;
                a.E[e] = qnan;
                a.logL[e] = qnan;
                a.status[e] = st;
            }
            if (a.trace)
                for (int it = lane; it < a.iters; it += 32) a.trace[e * a.iters + it] = -1;
            continue;
        }

        float sxy = a.step_xy, sz = a.step_z;
        for (int it = 0; it < a.iters; ++it) {
            // eta_i and H at the grid centre
            float hc = 0.0f;
            for (int i = lane; i < n_s; i += 32) {
                float eta = eta_floor<TYPE>(L, i, cx, cy, cz);
                s_ec[i] = eta;
                s_ic[i] = __frcp_rn(eta);
                hc += eta;
            }
            hc = warp_sum(hc);
            const float inv_hc = __frcp_rn(hc);
            __syncwarp();
            float bestF = -INFINITY;
            int bestk = 0x7fffffff;
            for (int k = lane; k < nodes; k += 32) {
                int ix = k % a.n_xy, iy = (k / a.n_xy) % a.n_xy, iz = k / (a.n_xy * a.n_xy);
                float x = fmaf((float)(ix - c_xy), sxy, cx);
                float y = fmaf((float)(iy - c_xy), sxy, cy);
                float z = fmaf((float)(iz - c_z), sz, cz);
                float F = node_score<TYPE>(L, s_sig, s_ic, s_ec, S, inv_hc, x, y, z);
                if (F > bestF) {
                    bestF = F;
                    bestk = k;
                }
            }
            for (int o = 16; o; o >>= 1) {
                float F2 = __shfl_xor_sync(kFull, bestF, o);
                int k2 = __shfl_xor_sync(kFull, bestk, o);
                if (F2 > bestF || (F2 == bestF && k2 < bestk)) {
                    bestF = F2;
                    bestk = k2;
                }
            }
            int ix = bestk % a.n_xy, iy = (bestk / a.n_xy) % a.n_xy, iz = bestk / (a.n_xy * a.n_xy);
            cx = fmaf((float)(ix - c_xy), sxy, cx);
            cy = fmaf((float)(iy - c_xy), sxy, cy);
            cz = fmaf((float)(iz - c_z), sz, cz);
            if (a.trace && lane == 0) a.trace[e * a.iters + it] = (int16_t)bestk;
            sxy *= a.shrink;
            sz *= a.shrink;
            __syncwarp();
        }

        // energy and full Poisson log-likelihood at the result
        float H = 0.0f;
        for (int i = lane; i < n_s; i += 32) H += eta_floor<TYPE>(L, i, cx, cy, cz);
        H = warp_sum(H);
        const float E = S / H;
        float ll = 0.0f;
        for (int i = lane; i < n_s; i += 32) {
            float mu = E * eta_floor<TYPE>(L, i, cx, cy, cz);
            float s = s_sig[i];
            ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + poisson_const(s) : -mu;
        }
        ll = warp_sum(ll);
        if (lane == 0) {
            a.xyz[3 * e] = cx;
            a.xyz[3 * e + 1] = cy;
            a.xyz[3 * e + 2] = cz;
            a.E[e] = E;
            a.logL[e] = ll;
            a.status[e] = ANTS_EVT_OK;
        }
        __syncwarp();
    }
}

template <int TYPE>
int launch_typed(const ants_ctx *ctx, const CgsArgs &a, cudaStream_t stream)
{
    const int threads = 256, wpb = threads / 32;
    size_t smem = (size_t)wpb * 3 * a.L.n_s * sizeof(float);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(cgs_plain_kernel<TYPE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_plain)");
    }
    long blocks = (a.n_e + wpb - 1) / wpb;
    long cap = (long)ctx->n_sm * 8;
    if (blocks > cap) blocks = cap;
    cgs_plain_kernel<TYPE><<<(unsigned)blocks, threads, smem, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cgs_plain_kernel launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace

int check_cgs_params(const ants_lrf *lrf, const ants_cgs_params *p)
{
    if (!p) return fail(ANTS_E_ARG, "cgs params: NULL");
    if (p->n_xy < 3 || p->n_xy > 15 || !(p->n_xy & 1))
        return fail(ANTS_E_ARG, "cgs params: n_xy %d must be odd in [3, 15]", p->n_xy);
    if (p->n_z < 1 || p->n_z > 15 || !(p->n_z & 1))
        return fail(ANTS_E_ARG, "cgs params: n_z %d must be odd in [1, 15]", p->n_z);
    if (p->n_z > 1 && lrf->type != ANTS_LRF_XYZ)
        return fail(ANTS_E_ARG, "cgs params: n_z > 1 needs an XYZ LRF");
    if (p->iters < 1 || p->iters > 32) return fail(ANTS_E_ARG, "cgs params: iters %d not in [1, 32]", p->iters);
    if (!(p->shrink > 0.0f && p->shrink < 1.0f)) return fail(ANTS_E_ARG, "cgs params: shrink must be in (0, 1)");
    if (!(p->step_xy > 0.0f) || !isfinite(p->step_xy)) return fail(ANTS_E_ARG, "cgs params: step_xy must be > 0");
    if (lrf->type == ANTS_LRF_XYZ && p->n_z > 1 && !(p->step_z > 0.0f))
        return fail(ANTS_E_ARG, "cgs params: step_z must be > 0");
    return ANTS_OK;
}

int launch_cgs_plain(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig,
                     long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                     int16_t *trace, cudaStream_t stream)
{
    if (cgs_xy_supported(lrf, p))
        return launch_cgs_xy(ctx, lrf, p, sig, n_e, start, xyz, E, logL, status, trace, stream);
    CgsArgs a;
    a.L = lrf->dev;
    a.n_xy = p.n_xy;
    a.n_z = p.n_z;
    a.iters = p.iters;
    a.shrink = p.shrink;
    a.step_xy = p.step_xy;
    a.step_z = p.step_z;
    a.z0 = p.z0;
    a.sig = sig;
    a.n_e = n_e;
    a.start = start;
    a.xyz = xyz;
    a.E = E;
    a.logL = logL;
    a.status = status;
    a.trace = trace;
    switch (lrf->type) {
    case ANTS_LRF_RADIAL: return launch_typed<ANTS_LRF_RADIAL>(ctx, a, stream);
    case ANTS_LRF_XY: return launch_typed<ANTS_LRF_XY>(ctx, a, stream);
    default: return launch_typed<ANTS_LRF_XYZ>(ctx, a, stream);
    }
}

}  // namespace ants
