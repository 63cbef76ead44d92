// Contracting-grid ML search for XY LRFs (Sec. 5.1.2.2 with Sec. 6.1.1 XY
// LRFs), separable form.  FP32.
//
// Work decomposition (one warp per event, grid-stride over events):
//   lane = (column j of the N x N grid, sensor slot q), Q = 32 / N slots;
//   slot q owns sensor pairs q, q+Q, ...  (pairs are interleaved as float2
//   in the coefficient table, so one 64-bit load serves two sensors).
// A lane sweeps the N nodes of its column.  Because every node of a column
// shares x, the tensor-product B-spline eta(x_j, y_k) = sum_a wy_k[a] T[iy_k+a]
// with T[r] = sum_b wx_j[b] C[r][ix_j+b] reuses the x-contracted rows T of the
// column: a 4-row window slides along y and only rows entering the window are
// loaded (4 float2 loads + 4 packed FMAs per new row).
// Per node and sensor: r = eta / eta(centre) (packed), log2 r on the MUFU
// pipe, acc += s log2 r, dH += eta - eta(centre); the slots of a column are
// summed with shuffles, and F = acc - S log2(1 + dH / H(centre)) decides the
// argmax (ties to the lowest flat node index), as in the generic kernel.
#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;
constexpr float kInvLn2 = 1.4426950408889634f;
constexpr int kXyThreads = 384;  // 12 warps: up to 168 registers per thread, one block per SM

struct XyArgs {
    LrfDev L;
    int iters;
    float shrink, step_xy;
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

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c)
{
    float2 d;
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rc = *reinterpret_cast<unsigned long long *>(&c);
    unsigned long long rd;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(rd) : "l"(ra), "l"(rb), "l"(rc));
    d = *reinterpret_cast<float2 *>(&rd);
    return d;
}

__device__ __forceinline__ float2 fmul2(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rd;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}

__device__ __forceinline__ float2 fsub2(float2 a, float2 b)
{
    unsigned long long ra = *reinterpret_cast<unsigned long long *>(&a);
    unsigned long long rb = *reinterpret_cast<unsigned long long *>(&b);
    unsigned long long rd;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    return *reinterpret_cast<float2 *>(&rd);
}

// s ln s - s - lgamma(s+1), s > 0 (Stirling series for s >= 10, A&S 6.1.41)
__device__ __forceinline__ float poisson_const(float s)
{
    if (s >= 10.0f) {
        float r = 1.0f / s, r2 = r * r;
        float series = r * (-1.0f / 12.0f + r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
        return -0.5f * logf(6.283185307179586f * s) + series;
    }
    return s * logf(s) - s - lgammaf(s + 1.0f);
}

// eta of both sensors of pair p at one point (inside the box), from the
// interleaved table
__device__ __forceinline__ float2 pair_eta(const LrfDev &L, const float2 *coef2, int p, float x, float y)
{
    float tx, ty, wx[4], wy[4];
    int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
    int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
    bs_weights(tx, wx);
    bs_weights(ty, wy);
    const float2 *c = coef2 + (size_t)p * L.pair_stride + jy * L.stride_y + jx;
    float2 f = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float2 *row = c + b * L.stride_y;
        float2 fr = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < 4; ++a) fr = ffma2(make_float2(wx[a], wx[a]), row[a], fr);
        f = ffma2(make_float2(wy[b], wy[b]), fr, f);
    }
    return f;
}

// x-contracted row r of the lane's column: sum_b wx[b] C[r][ix+b] (both sensors)
__device__ __forceinline__ float2 trow(const float2 *colbase, int stride_y, int r, const float2 wx2[4])
{
    const float2 *row = colbase + r * stride_y;
    float2 v = fmul2(wx2[0], row[0]);
    v = ffma2(wx2[1], row[1], v);
    v = ffma2(wx2[2], row[2], v);
    v = ffma2(wx2[3], row[3], v);
    return v;
}

template <int N, bool SMEM, bool FLOOR>
__global__ void __launch_bounds__(kXyThreads, 1) cgs_xy_kernel(XyArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LrfDev &L = a.L;
    const int n_s = L.n_s, n_pairs = L.n_pairs, n_pad = 2 * n_pairs;
    const size_t table = SMEM ? (size_t)n_pairs * L.pair_stride : 0;
    float2 *cs = reinterpret_cast<float2 *>(smem_raw);
    const float2 *coef2 = L.coef2;
    if (SMEM) {
        const float4 *src = reinterpret_cast<const float4 *>(L.coef2);
        float4 *dst = reinterpret_cast<float4 *>(cs);
        for (size_t k = threadIdx.x; k < table / 2; k += blockDim.x) dst[k] = src[k];
        if ((table & 1) && threadIdx.x == 0) cs[table - 1] = L.coef2[table - 1];
        __syncthreads();
        coef2 = cs;
    }
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float *wbase = reinterpret_cast<float *>(cs + table) + (size_t)wib * 3 * n_pad;
    float *s_sig = wbase, *s_ic = wbase + n_pad, *s_ec = wbase + 2 * n_pad;
    const float2 *s_sig2 = reinterpret_cast<const float2 *>(s_sig);
    const float2 *s_ic2 = reinterpret_cast<const float2 *>(s_ic);
    const float2 *s_ec2 = reinterpret_cast<const float2 *>(s_ec);

    constexpr int Q = 32 / N;
    constexpr int C = (N - 1) / 2;
    const int q = lane / N, j = lane - q * N;
    const bool active = q < Q;
    const float qnan = __int_as_float(0x7fc00000);

    for (long e = (long)blockIdx.x * wpb + wib; e < a.n_e; e += (long)gridDim.x * wpb) {
        // ---- prologue: signals, S, centroid, status --------------------------
        const float *sg = a.sig + e * n_s;
        float S = 0.0f, Sx = 0.0f, Sy = 0.0f, Sw = 0.0f;
        int bad = 0;
        for (int i = lane; i < n_pad; i += 32) {
            float v = i < n_s ? sg[i] : 0.0f;
            bad |= !(v >= 0.0f) || isinf(v);
            s_sig[i] = v;
            if (i < n_s) {
                float w = v * L.cog_w[i];
                S += v;
                Sx = fmaf(L.sxy[2 * i], w, Sx);
                Sy = fmaf(L.sxy[2 * i + 1], w, Sy);
                Sw += w;
            }
        }
        bad = __any_sync(kFull, bad);
        S = warp_sum(S);
        Sx = warp_sum(Sx);
        Sy = warp_sum(Sy);
        Sw = warp_sum(Sw);
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
                cx = fminf(fmaxf(Sx / Sw, L.lo[0]), L.hi[0]);
                cy = fminf(fmaxf(Sy / Sw, L.lo[1]), L.hi[1]);
            }
            if (!in_box(L, cx, cy, cz)) st = ANTS_EVT_OUT_OF_DOMAIN;
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
            __syncwarp();
            continue;
        }

        float sxy = a.step_xy;
        for (int it = 0; it < a.iters; ++it) {
            // ---- centre: eta_i, 1/eta_i, H -------------------------------------
            float hc = 0.0f;
            for (int p = lane; p < n_pairs; p += 32) {
                float2 ec = pair_eta(L, coef2, p, cx, cy);
                if (FLOOR) {
                    ec.x = fmaxf(ec.x, kEtaFloor);
                    ec.y = fmaxf(ec.y, kEtaFloor);
                }
                s_ec[2 * p] = ec.x;
                s_ec[2 * p + 1] = ec.y;
                s_ic[2 * p] = __frcp_rn(ec.x);
                s_ic[2 * p + 1] = __frcp_rn(ec.y);
                hc += ec.x + (2 * p + 1 < n_s ? ec.y : 0.0f);
            }
            hc = warp_sum(hc);
            const float inv_hc = __frcp_rn(hc);

            // ---- row bases (lane k computes row k, then broadcast) ----------
            float my_w[4], ty_;
            int my_iy = 0;
            bool my_yok = false;
            {
                int k = lane < N ? lane : 0;
                float y = fmaf((float)(k - C), sxy, cy);
                my_yok = y >= L.lo[1] && y <= L.hi[1];
                my_iy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty_);
                bs_weights(ty_, my_w);
            }
            float wy[N][4];
            int iy[N];
            unsigned yok_mask = __ballot_sync(kFull, my_yok && lane < N);
#pragma unroll
            for (int k = 0; k < N; ++k) {
                iy[k] = __shfl_sync(kFull, my_iy, k);
#pragma unroll
                for (int t = 0; t < 4; ++t) wy[k][t] = __shfl_sync(kFull, my_w[t], k);
            }
            // ---- the lane's column basis ------------------------------------
            const float x = fmaf((float)(j - C), sxy, cx);
            const bool xok = x >= L.lo[0] && x <= L.hi[0];
            float tx, wxs[4];
            const int ix = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
            bs_weights(tx, wxs);
            float2 wx2[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) wx2[t] = make_float2(wxs[t], wxs[t]);
            __syncwarp();

            float acc[N], dh[N];
#pragma unroll
            for (int k = 0; k < N; ++k) acc[k] = dh[k] = 0.0f;
            if (active) {
                for (int p = q; p < n_pairs; p += Q) {
                    const float2 sp = s_sig2[p], ic = s_ic2[p], ec = s_ec2[p];
                    const float2 *colbase = coef2 + (size_t)p * L.pair_stride + ix;
                    float2 W0 = trow(colbase, L.stride_y, iy[0], wx2);
                    float2 W1 = trow(colbase, L.stride_y, iy[0] + 1, wx2);
                    float2 W2 = trow(colbase, L.stride_y, iy[0] + 2, wx2);
                    float2 W3 = trow(colbase, L.stride_y, iy[0] + 3, wx2);
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        if (k > 0) {
                            int adv = iy[k] - iy[k - 1];
                            if (adv >= 4) {
                                W0 = trow(colbase, L.stride_y, iy[k], wx2);
                                W1 = trow(colbase, L.stride_y, iy[k] + 1, wx2);
                                W2 = trow(colbase, L.stride_y, iy[k] + 2, wx2);
                                W3 = trow(colbase, L.stride_y, iy[k] + 3, wx2);
                            } else {
                                for (int t = 0; t < adv; ++t) {
                                    W0 = W1;
                                    W1 = W2;
                                    W2 = W3;
                                    W3 = trow(colbase, L.stride_y, iy[k] + 4 - adv + t, wx2);
                                }
                            }
                        }
                        float2 eta;
                        eta.x = wy[k][0] * W0.x;
                        eta.y = wy[k][0] * W0.y;
                        eta.x = fmaf(wy[k][1], W1.x, eta.x);
                        eta.y = fmaf(wy[k][1], W1.y, eta.y);
                        eta.x = fmaf(wy[k][2], W2.x, eta.x);
                        eta.y = fmaf(wy[k][2], W2.y, eta.y);
                        eta.x = fmaf(wy[k][3], W3.x, eta.x);
                        eta.y = fmaf(wy[k][3], W3.y, eta.y);
                        if (FLOOR) {
                            eta.x = fmaxf(eta.x, kEtaFloor);
                            eta.y = fmaxf(eta.y, kEtaFloor);
                        }
                        const float2 r = fmul2(eta, ic);
                        acc[k] = fmaf(sp.x, __log2f(r.x), acc[k]);
                        acc[k] = fmaf(sp.y, __log2f(r.y), acc[k]);
                        const float2 d = fsub2(eta, ec);
                        dh[k] += d.x;
                        dh[k] += d.y;
                    }
                }
            }
            // ---- sum the slots of each column into slot 0 -------------------
#pragma unroll
            for (int t = 1; t < Q; ++t) {
                int src = lane + t * N;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    float va = __shfl_sync(kFull, acc[k], src < 32 ? src : lane);
                    float vd = __shfl_sync(kFull, dh[k], src < 32 ? src : lane);
                    if (q == 0 && src < 32) {
                        acc[k] += va;
                        dh[k] += vd;
                    }
                }
            }
            // ---- node scores, argmax (ties to the lowest flat index k*N+j) --
            float bestF = -INFINITY;
            int bestk = 0x7fffffff;
            if (q == 0) {
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    bool ok = xok && ((yok_mask >> k) & 1u);
                    float F = ok ? acc[k] - S * (log1pf(dh[k] * inv_hc) * kInvLn2) : -INFINITY;
                    if (F > bestF) {
                        bestF = F;
                        bestk = k * N + j;
                    }
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
            const int bj = bestk % N, bk = bestk / N;
            cx = fmaf((float)(bj - C), sxy, cx);
            cy = fmaf((float)(bk - C), sxy, cy);
            if (a.trace && lane == 0) a.trace[e * a.iters + it] = (int16_t)bestk;
            sxy *= a.shrink;
            __syncwarp();
        }

        // ---- energy and full Poisson log-likelihood at the result -----------
        float H = 0.0f, ll = 0.0f;
        float2 etas[2];
        int np = 0;
        for (int p = lane; p < n_pairs; p += 32, ++np) {
            float2 v = pair_eta(L, coef2, p, cx, cy);
            v.x = fmaxf(v.x, kEtaFloor);
            v.y = fmaxf(v.y, kEtaFloor);
            if (np < 2) etas[np] = v;
            H += v.x + (2 * p + 1 < n_s ? v.y : 0.0f);
        }
        H = warp_sum(H);
        const float E = S / H;
        np = 0;
        for (int p = lane; p < n_pairs; p += 32, ++np) {
            float2 v = np < 2 ? etas[np] : pair_eta(L, coef2, p, cx, cy);
            v.x = fmaxf(v.x, kEtaFloor);
            v.y = fmaxf(v.y, kEtaFloor);
            float vv[2] = {v.x, v.y};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                int i = 2 * p + h;
                if (i >= n_s) continue;
                float mu = E * vv[h];
                float s = s_sig[i];
                ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + poisson_const(s) : -mu;
            }
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

template <int N>
int launch_n(const ants_ctx *ctx, const XyArgs &a, bool floor_needed, cudaStream_t stream)
{
    const int threads = kXyThreads, wpb = threads / 32;
    const size_t table = (size_t)a.L.n_pairs * a.L.pair_stride * sizeof(float2);
    const size_t per_warp = (size_t)wpb * 3 * 2 * a.L.n_pairs * sizeof(float);
    bool smem_table = table + per_warp <= ctx->smem_optin;
    size_t smem = per_warp + (smem_table ? table : 0);
    cudaError_t e = cudaSuccess;
    long blocks = (a.n_e + wpb - 1) / wpb;
    long cap = (long)ctx->n_sm;
    if (blocks > cap) blocks = cap;
#define ANTS_XY_LAUNCH(SM, FL)                                                                               \
    do {                                                                                                     \
        e = cudaFuncSetAttribute(cgs_xy_kernel<N, SM, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                 (int)smem);                                                                 \
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_xy)");                            \
        cgs_xy_kernel<N, SM, FL><<<(unsigned)blocks, threads, smem, stream>>>(a);                             \
    } while (0)
    if (smem_table) {
        if (floor_needed) ANTS_XY_LAUNCH(true, true);
        else ANTS_XY_LAUNCH(true, false);
    } else {
        if (floor_needed) ANTS_XY_LAUNCH(false, true);
        else ANTS_XY_LAUNCH(false, false);
    }
#undef ANTS_XY_LAUNCH
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cgs_xy_kernel launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace

bool cgs_xy_supported(const ants_lrf *lrf, const ants_cgs_params &p)
{
    if (lrf->type != ANTS_LRF_XY || p.n_z != 1 || !lrf->dev.coef2) return false;
    return p.n_xy == 5 || p.n_xy == 7 || p.n_xy == 9 || p.n_xy == 11 || p.n_xy == 13 || p.n_xy == 15;
}

int launch_cgs_xy(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig, long n_e,
                  const float *start, float *xyz, float *E, float *logL, int32_t *status, int16_t *trace,
                  cudaStream_t stream)
{
    XyArgs a;
    a.L = lrf->dev;
    a.iters = p.iters;
    a.shrink = p.shrink;
    a.step_xy = p.step_xy;
    a.sig = sig;
    a.n_e = n_e;
    a.start = start;
    a.xyz = xyz;
    a.E = E;
    a.logL = logL;
    a.status = status;
    a.trace = trace;
    // the floor is needed when an LRF value can be <= 0, or to neutralise the
    // padding sensor of an odd sensor count (zero coefficients)
    bool floor_needed = !lrf->dev.positive || (lrf->n_s & 1);
    switch (p.n_xy) {
    case 5: return launch_n<5>(ctx, a, floor_needed, stream);
    case 7: return launch_n<7>(ctx, a, floor_needed, stream);
    case 9: return launch_n<9>(ctx, a, floor_needed, stream);
    case 11: return launch_n<11>(ctx, a, floor_needed, stream);
    case 13: return launch_n<13>(ctx, a, floor_needed, stream);
    default: return launch_n<15>(ctx, a, floor_needed, stream);
    }
}

}  // namespace ants
