// Search variants of the contracting-grid reconstruction.
//   Sec. 5.1.2: the match between measured and LRF signals is evaluated by
//   maximum likelihood or by least squares, and sensors whose signal is
//   below a threshold, or that lie farther than a given distance from the
//   start position, can be left out;
//   Sec. 5.1.2.1 / 5.1.2.2: the start is the centroid or the position of the
//   sensor with the strongest signal;
//   Sec. 5.3: passive sensors are ignored.
// One warp per event, every node evaluated on its own (any LRF type); the
// sensors in the match are a per-event mask in shared memory.
//   maximum likelihood: F = sum_A s log2(eta / eta_c) - S log2(1 + sum_A
//     (eta - eta_c) / H_c), relative to the grid centre c as in the plain
//     search (A: the sensors in the match, S = sum_A s);
//   least squares (Pearson's statistic with the node's energy ratio E = S/H):
//     F = -sum_A (s - E eta)^2 / (E eta), H = sum_A eta, in two passes.
// Ties go to the lowest node index; nodes where an LRF in the match is not
// defined score -inf.
#include <cmath>

#include "bspline.cuh"
#include "internal.cuh"
#include "match.cuh"

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;
constexpr int kMaxVariantSensors = kMaxMatchSensors;
constexpr int kVarWarps = 8;

struct VarArgs {
    LrfDev L;
    int n_xy, n_z, iters;
    float shrink, step_xy, step_z;
    int criterion;
    const float *sig;
    long n_e;
    const float *start_xyz;  // given starts [n_e][3] (nullable)
    float *xyz, *E, *logL;
    int32_t *status;
    int16_t *trace;
    MatchArgs m;
};

__device__ __forceinline__ float vwarp_sum(float v) { return match_warp_sum(v); }

// s ln s - s - lgamma(s + 1) for s > 0 (Stirling series from s = 10)
__device__ __forceinline__ float vpoisson_const(float s)
{
    if (s >= 10.0f) {
        float r = 1.0f / s, r2 = r * r;
        float series = r * (-1.0f / 12.0f + r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
        return -0.5f * logf(6.283185307179586f * s) + series;
    }
    return s * logf(s) - s - lgammaf(s + 1.0f);
}

template <int TYPE>
__device__ __forceinline__ float eta_at(const LrfDev &L, int i, float x, float y, float z)
{
    bool ok;
    return fmaxf(lrf_eta_t<TYPE>(L, i, x, y, z, ok), kEtaFloor);
}

// every LRF in the match defined at the node
template <int TYPE>
__device__ __forceinline__ bool node_ok(const LrfDev &L, const float *s_act, float x, float y, float z)
{
    return lrf_defined(L, s_act, x, y, z);
}

__device__ __forceinline__ void set_failed(const VarArgs &a, long e, int st, int lane)
{
    if (lane == 0) {
        const float nan = __int_as_float(0x7fc00000);
        a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = nan;
        a.E[e] = a.logL[e] = nan;
        a.status[e] = st;
        if (a.trace)
            for (int it = 0; it < a.iters; ++it) a.trace[e * a.iters + it] = -1;
    }
    __syncwarp();
}

template <int TYPE>
__global__ void __launch_bounds__(32 * kVarWarps, 2) cgs_variant_kernel(const __grid_constant__ VarArgs a)
{
    extern __shared__ float smem[];
    const LrfDev &L = a.L;
    const int n_s = L.n_s;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *s_sig = smem + (size_t)wib * 4 * n_s;  // signals (0 for passive sensors)
    float *s_act = s_sig + n_s;                   // 1 in the match, 0 out
    float *s_ic = s_act + n_s;                    // 1 / eta at the grid centre
    float *s_ec = s_ic + n_s;                     // eta at the grid centre
    const int nodes = a.n_xy * a.n_xy * a.n_z;
    const int c_xy = (a.n_xy - 1) / 2, c_z = (a.n_z - 1) / 2;
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long e = (long)blockIdx.x * (blockDim.x >> 5) + wib; e < a.n_e; e += warps) {
        // ---- signals, status, start, the sensors in the match ---------------
        float S, cx, cy, cz;
        const int st = match_prologue<TYPE>(L, a.m, a.sig, e, a.start_xyz, s_sig, s_act, lane, S, cx, cy, cz);
        if (st != ANTS_EVT_OK) {
            set_failed(a, e, st, lane);
            continue;
        }
        // ---- contracting grids ------------------------------------------------
        float sxy = a.step_xy, sz = a.step_z;
        for (int it = 0; it < a.iters; ++it) {
            float inv_hc = 0.0f;
            if (a.criterion == 0) {
                float hc = 0.0f;
                for (int i = lane; i < n_s; i += 32) {
                    const float eta = eta_at<TYPE>(L, i, cx, cy, cz);
                    s_ec[i] = eta;
                    s_ic[i] = __frcp_rn(eta);
                    if (s_act[i] != 0.0f) hc += eta;
                }
                inv_hc = __frcp_rn(vwarp_sum(hc));
                __syncwarp();
            }
            float bestF = -INFINITY;
            int bestk = 0x7fffffff;
            for (int k = lane; k < nodes; k += 32) {
                const int ix = k % a.n_xy, iy = (k / a.n_xy) % a.n_xy, iz = k / (a.n_xy * a.n_xy);
                const float x = fmaf((float)(ix - c_xy), sxy, cx);
                const float y = fmaf((float)(iy - c_xy), sxy, cy);
                const float z = fmaf((float)(iz - c_z), sz, cz);
                float F = -INFINITY;
                if (node_ok<TYPE>(L, s_act, x, y, z)) {
                    if (a.criterion == 0) {
                        float acc = 0.0f, dh = 0.0f;
                        for (int i = 0; i < n_s; ++i) {
                            if (s_act[i] == 0.0f) continue;  // the same sensor on every lane
                            const float eta = eta_at<TYPE>(L, i, x, y, z);
                            acc = fmaf(s_sig[i], __log2f(eta * s_ic[i]), acc);
                            dh += eta - s_ec[i];
                        }
                        F = acc - S * (log1pf(dh * inv_hc) * 1.4426950408889634f);
                    } else {
                        float H = 0.0f;
                        for (int i = 0; i < n_s; ++i)
                            if (s_act[i] != 0.0f) H += eta_at<TYPE>(L, i, x, y, z);
                        const float En = S / H;
                        float chi = 0.0f;
                        for (int i = 0; i < n_s; ++i) {
                            if (s_act[i] == 0.0f) continue;
                            const float mu = En * eta_at<TYPE>(L, i, x, y, z), d = s_sig[i] - mu;
                            chi = fmaf(d, d / mu, chi);
                        }
                        F = -chi;
                    }
                }
                if (F > bestF) {
                    bestF = F;
                    bestk = k;
                }
            }
            for (int o = 16; o; o >>= 1) {
                const float F2 = __shfl_xor_sync(kFull, bestF, o);
                const int k2 = __shfl_xor_sync(kFull, bestk, o);
                if (F2 > bestF || (F2 == bestF && k2 < bestk)) {
                    bestF = F2;
                    bestk = k2;
                }
            }
            if (bestk >= nodes) bestk = c_z * a.n_xy * a.n_xy + c_xy * a.n_xy + c_xy;  // no valid node: stay
            const int ix = bestk % a.n_xy, iy = (bestk / a.n_xy) % a.n_xy, iz = bestk / (a.n_xy * a.n_xy);
            cx = fmaf((float)(ix - c_xy), sxy, cx);
            cy = fmaf((float)(iy - c_xy), sxy, cy);
            cz = fmaf((float)(iz - c_z), sz, cz);
            if (a.trace && lane == 0) a.trace[e * a.iters + it] = (int16_t)bestk;
            sxy *= a.shrink;
            sz *= a.shrink;
            __syncwarp();
        }
        // ---- energy and full Poisson log-likelihood over the match ----------
        float H = 0.0f;
        for (int i = lane; i < n_s; i += 32)
            if (s_act[i] != 0.0f) H += eta_at<TYPE>(L, i, cx, cy, cz);
        H = vwarp_sum(H);
        const float En = S / H;
        float ll = 0.0f;
        for (int i = lane; i < n_s; i += 32) {
            if (s_act[i] == 0.0f) continue;
            const float mu = En * eta_at<TYPE>(L, i, cx, cy, cz), s = s_sig[i];
            ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + vpoisson_const(s) : -mu;
        }
        ll = vwarp_sum(ll);
        if (lane == 0) {
            a.xyz[3 * e] = cx;
            a.xyz[3 * e + 1] = cy;
            a.xyz[3 * e + 2] = cz;
            a.E[e] = En;
            a.logL[e] = ll;
            a.status[e] = ANTS_EVT_OK;
        }
        __syncwarp();
    }
}

}  // namespace

int check_variant_params(const ants_lrf *lrf, const ants_cgs_variant_params *P)
{
    if (!P) return fail(ANTS_E_ARG, "variant parameters are NULL");
    int rc = check_cgs_params(lrf, &P->grid);
    if (rc != ANTS_OK) return rc;
    if (P->criterion != ANTS_CRIT_ML && P->criterion != ANTS_CRIT_LS)
        return fail(ANTS_E_ARG, "variant: unknown criterion %d", P->criterion);
    if (P->start != ANTS_START_COG && P->start != ANTS_START_MAX_SENSOR)
        return fail(ANTS_E_ARG, "variant: unknown start %d", P->start);
    if (!(P->min_signal >= 0.0f) || !(P->max_distance >= 0.0f))
        return fail(ANTS_E_ARG, "variant: min_signal and max_distance must be >= 0");
    if (lrf->n_s > kMaxVariantSensors)
        return fail(ANTS_E_UNIMPLEMENTED, "variant: at most %d sensors", kMaxVariantSensors);
    return ANTS_OK;
}

int reconstruct_variant(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_variant_params &P, const float *sig,
                        long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                        int16_t *trace, cudaStream_t s)
{
    VarArgs a;
    a.L = lrf->dev;
    a.n_xy = P.grid.n_xy;
    a.n_z = P.grid.n_z;
    a.iters = P.grid.iters;
    a.shrink = P.grid.shrink;
    a.step_xy = P.grid.step_xy;
    a.step_z = P.grid.step_z;
    a.m.z0 = P.grid.z0;
    a.criterion = P.criterion;
    a.m.start = P.start;
    a.m.min_signal = P.min_signal;
    a.m.max_distance = P.max_distance;
    a.sig = sig;
    a.n_e = n_e;
    a.start_xyz = start;
    a.xyz = xyz;
    a.E = E;
    a.logL = logL;
    a.status = status;
    a.trace = trace;
    const int n_s = lrf->n_s;
    for (int i = 0; i < kMaxVariantSensors; ++i) {
        a.m.gain[i] = i < n_s ? lrf->rel_gain[i] : 1.0;
        a.m.inv_gain[i] = (float)(1.0 / a.m.gain[i]);
        a.m.passive[i] = i < n_s && P.passive_host && P.passive_host[i] ? 1 : 0;
    }
    // as many warps per block as fit 4 n_s floats each in 48 KB
    int wpb = (int)(48 * 1024 / (16 * (size_t)n_s));
    wpb = wpb < 1 ? 1 : (wpb > kVarWarps ? kVarWarps : wpb);
    const size_t smem = (size_t)wpb * 16 * n_s;
    long blocks = (n_e + wpb - 1) / wpb;
    const long cap = (long)ctx->n_sm * 16;
    if (blocks > cap) blocks = cap;
    switch (lrf->type) {
    case ANTS_LRF_RADIAL: cgs_variant_kernel<ANTS_LRF_RADIAL><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a); break;
    case ANTS_LRF_XY:
        if (lrf->dev.set_of) cgs_variant_kernel<kLrfXYSym><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
        else cgs_variant_kernel<ANTS_LRF_XY><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
        break;
    case ANTS_LRF_XYZ: cgs_variant_kernel<ANTS_LRF_XYZ><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a); break;
    case ANTS_LRF_COMPOSITE:
        cgs_variant_kernel<ANTS_LRF_COMPOSITE><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a);
        break;
    case ANTS_LRF_AXIAL_Z: cgs_variant_kernel<ANTS_LRF_AXIAL_Z><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a); break;
    default: cgs_variant_kernel<ANTS_LRF_SLICED><<<(unsigned)blocks, 32 * wpb, smem, s>>>(a); break;
    }
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "cgs_variant_kernel launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace ants
