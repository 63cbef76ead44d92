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
#include <algorithm>
#include <cfloat>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

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
    int row_div;  // event e reads signal row e / row_div (several searches per event)
    const float *start;
    float *xyz, *E, *logL;
    int32_t *status;
    int16_t *trace;
    // XYZ only: separable node evaluation (sep != 0) with per-warp tables
    // sized for at most ry_cap coefficient rows and rz_cap planes
    int sep, ry_cap, rz_cap;
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
        ok = ok && plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]) <= L.hi[0];
    }
    return ok;
}

template <int TYPE>
__device__ __forceinline__ float eta_floor(const LrfDev &L, int i, float x, float y, float z)
{
    bool ok;
    float v = lrf_eta_t<TYPE>(L, i, x, y, z, ok);
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
            const float r = plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]);
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

// Event prologue (one warp): signals into s_sig, S, the start (centroid of
// Sec. 5.1.1 or a given start) and its checks.  Returns false, with the
// outputs written, for an event that is not searched.
template <int TYPE>
__device__ __forceinline__ bool event_prologue(const CgsArgs &a, long e, float *s_sig, int lane, float &S, float &cx,
                                               float &cy, float &cz)
{
    const LrfDev &L = a.L;
    const int n_s = L.n_s;
    const float qnan = __int_as_float(0x7fc00000);
    const float *sg = a.sig + (e / a.row_div) * n_s;
    float Sx = 0.0f, Sy = 0.0f, Sw = 0.0f;
    S = 0.0f;
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
    cx = cy = cz = 0.0f;
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
    if (st == ANTS_EVT_OK) return true;
    if (lane == 0) {
        a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = qnan;
        a.E[e] = qnan;
        a.logL[e] = qnan;
        a.status[e] = st;
    }
    if (a.trace)
        for (int it = lane; it < a.iters; it += 32) a.trace[e * a.iters + it] = -1;
    return false;
}

// eta_i and 1/eta_i at the grid centre into s_ec, s_ic; returns 1 / H(centre)
template <int TYPE>
__device__ __forceinline__ float centre_values(const LrfDev &L, float *s_ic, float *s_ec, float cx, float cy,
                                               float cz, int lane)
{
    float hc = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) {
        float eta = eta_floor<TYPE>(L, i, cx, cy, cz);
        s_ec[i] = eta;
        s_ic[i] = __frcp_rn(eta);
        hc += eta;
    }
    hc = warp_sum(hc);
    __syncwarp();
    return __frcp_rn(hc);
}

// warp argmax (ties to the lowest node index), then the centre moves to the
// best node and the spacings shrink
__device__ __forceinline__ void pick_and_move(const CgsArgs &a, long e, int it, float bestF, int bestk, float &cx,
                                              float &cy, float &cz, float &sxy, float &sz, int lane)
{
    const int c_xy = (a.n_xy - 1) / 2, c_z = (a.n_z - 1) / 2;
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
template <int TYPE>
__device__ __forceinline__ void event_epilogue(const CgsArgs &a, long e, const float *s_sig, float S, float cx,
                                               float cy, float cz, int lane)
{
    const LrfDev &L = a.L;
    float H = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) H += eta_floor<TYPE>(L, i, cx, cy, cz);
    H = warp_sum(H);
    const float E = S / H;
    float ll = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) {
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

// one power-basis cubic of a radial table held in shared memory (32-bit
// shared address) or read through the read-only path
template <bool SPOLY>
__device__ __forceinline__ float4 poly_at(const float4 *poly, unsigned saddr, int j)
{
    if (SPOLY) {
        float4 v;
        asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
            : "r"(saddr + 16u * (unsigned)j));
        return v;
    }
    return __ldg(poly + j);
}

// Scores of a radial-LRF grid, NPL nodes per lane at a time sharing each
// sensor's data.  Sensors are taken in pairs with packed FP32x2 arithmetic
// (each element as node_score computes it; the two halves of a node's sums
// are added at the end), an odd last sensor on its own.  Updates the lane's
// best (score, node).  With SPOLY the cubics are read from the block's shared
// copy `polys`.
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

template <int NPL, bool SPOLY>
__device__ __forceinline__ void radial_nodes(const CgsArgs &a, const LrfDev &L, const float *s_sig, const float *s_ic,
                                             const float *s_ec, float S, float inv_hc, float cx, float cy, float sxy,
                                             int nodes, int lane, float &bestF, int &bestk, const float4 *polys)
{
    const int c_xy = (a.n_xy - 1) / 2;
    const float hi = L.hi[0];
    const float inv_h = L.inv_h[0];
    const int n_int = L.n_int[0];
    auto poly_of = [&](int i) { return polys + (L.shared ? 0 : (L.set_of ? __ldg(L.set_of + i) : i)) * n_int; };
    for (int k0 = 0; k0 < nodes; k0 += 32 * NPL) {
        float xs[NPL], ys[NPL], rmax[NPL];
        float2 acc[NPL], dh[NPL];
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
            const int k = k0 + lane + 32 * m;
            const int ix = k % a.n_xy, iy = (k / a.n_xy) % a.n_xy;
            xs[m] = fmaf((float)(ix - c_xy), sxy, cx);
            ys[m] = fmaf((float)(iy - c_xy), sxy, cy);
            acc[m] = dh[m] = make_float2(0.0f, 0.0f);
            rmax[m] = 0.0f;
        }
        const float2 inv_h2 = make_float2(inv_h, inv_h);
        const int n_pair = L.n_s >> 1;
        for (int pr = 0; pr < n_pair; ++pr) {
            const int i = 2 * pr;
            const float4 q = __ldg(reinterpret_cast<const float4 *>(L.sxy) + pr);  // x_i y_i x_i+1 y_i+1
            const float2 nsx = make_float2(-q.x, -q.z), nsy = make_float2(-q.y, -q.w);
            const float2 si = make_float2(s_sig[i], s_sig[i + 1]), ici = make_float2(s_ic[i], s_ic[i + 1]);
            const float2 neci = make_float2(-s_ec[i], -s_ec[i + 1]);
            const float2 gi = __ldg(reinterpret_cast<const float2 *>(L.gain) + pr);
            const float4 *p0 = poly_of(i), *p1 = poly_of(i + 1);
            const unsigned sp0 = SPOLY ? (unsigned)__cvta_generic_to_shared(p0) : 0u;
            const unsigned sp1 = SPOLY ? (unsigned)__cvta_generic_to_shared(p1) : 0u;
#pragma unroll
            for (int m = 0; m < NPL; ++m) {
                const float2 dx = fadd2(make_float2(xs[m], xs[m]), nsx);
                const float2 dy = fadd2(make_float2(ys[m], ys[m]), nsy);
                const float2 r2 = ffma2(dx, dx, fmul2(dy, dy));
                const float2 r = fmul2(r2, make_float2(rsqrtf(fmaxf(r2.x, 1e-30f)), rsqrtf(fmaxf(r2.y, 1e-30f))));
                rmax[m] = fmaxf(rmax[m], fmaxf(r.x, r.y));
                // the span and local parameter of radial_profile
                const float2 u = fmul2(make_float2(fminf(r.x, hi), fminf(r.y, hi)), inv_h2);
                const int j0 = min((int)u.x, n_int - 1), j1 = min((int)u.y, n_int - 1);
                const float2 t = fadd2(u, make_float2(-(float)j0, -(float)j1));
                const float4 c0 = poly_at<SPOLY>(p0, sp0, j0), c1 = poly_at<SPOLY>(p1, sp1, j1);
                float2 f = ffma2(t, make_float2(c0.w, c1.w), make_float2(c0.z, c1.z));
                f = ffma2(t, f, make_float2(c0.y, c1.y));
                f = ffma2(t, f, make_float2(c0.x, c1.x));
                float2 eta = fmul2(gi, f);
                eta = make_float2(fmaxf(eta.x, kEtaFloor), fmaxf(eta.y, kEtaFloor));
                const float2 rr = fmul2(eta, ici);
                acc[m] = ffma2(si, make_float2(__log2f(rr.x), __log2f(rr.y)), acc[m]);
                dh[m] = fadd2(dh[m], fadd2(eta, neci));
            }
        }
        if (L.n_s & 1) {
            const int i = L.n_s - 1;
            const float sx = __ldg(L.sxy + 2 * i), sy = __ldg(L.sxy + 2 * i + 1);
            const float si = s_sig[i], ici = s_ic[i], eci = s_ec[i];
            const float gi = __ldg(L.gain + i);
            const float4 *poly = poly_of(i);
            const unsigned sp = SPOLY ? (unsigned)__cvta_generic_to_shared(poly) : 0u;
#pragma unroll
            for (int m = 0; m < NPL; ++m) {
                const float r = plane_dist(xs[m] - sx, ys[m] - sy);
                rmax[m] = fmaxf(rmax[m], r);
                const float u = fminf(r, hi) * inv_h;
                const int j = min((int)u, n_int - 1);
                const float t = u - (float)j;
                const float4 pc = poly_at<SPOLY>(poly, sp, j);
                const float f = fmaf(t, fmaf(t, fmaf(t, pc.w, pc.z), pc.y), pc.x);
                const float eta = fmaxf(gi * f, kEtaFloor);
                acc[m].x = fmaf(si, __log2f(eta * ici), acc[m].x);
                dh[m].x += eta - eci;
            }
        }
#pragma unroll
        for (int m = 0; m < NPL; ++m) {
            const int k = k0 + lane + 32 * m;
            if (k < nodes) {
                const float A = acc[m].x + acc[m].y, D = dh[m].x + dh[m].y;
                const float F = rmax[m] <= hi ? A - S * (log1pf(D * inv_hc) * 1.4426950408889634f) : -INFINITY;
                if (F > bestF) {
                    bestF = F;
                    bestk = k;
                }
            }
        }
    }
}

// Reconstruct event e of a (one warp; s_sig, s_ic, s_ec: 3 n_s floats of
// this warp's shared memory), every node evaluated on its own.  Shared by the
// plain and the batched kernels.
template <int TYPE, bool SPOLY = false>
__device__ __forceinline__ void cgs_event(const CgsArgs &a, long e, float *s_sig, float *s_ic, float *s_ec,
                                          int lane, const float4 *s_poly = nullptr)
{
    const LrfDev &L = a.L;
    const int nodes = a.n_xy * a.n_xy * a.n_z;
    const int c_xy = (a.n_xy - 1) / 2, c_z = (a.n_z - 1) / 2;
    float S, cx, cy, cz;
    if (!event_prologue<TYPE>(a, e, s_sig, lane, S, cx, cy, cz)) return;
    float sxy = a.step_xy, sz = a.step_z;
    for (int it = 0; it < a.iters; ++it) {
        const float inv_hc = centre_values<TYPE>(L, s_ic, s_ec, cx, cy, cz, lane);
        float bestF = -INFINITY;
        int bestk = 0x7fffffff;
        if (TYPE == ANTS_LRF_RADIAL) {
            // a lane's nodes share each sensor's data (3 per lane covers a
            // 9 x 9 grid in one pass, 4 per lane larger grids)
            if (nodes <= 96)
                radial_nodes<3, SPOLY>(a, L, s_sig, s_ic, s_ec, S, inv_hc, cx, cy, sxy, nodes, lane, bestF, bestk,
                                       SPOLY ? s_poly : L.rpoly);
            else
                radial_nodes<4, SPOLY>(a, L, s_sig, s_ic, s_ec, S, inv_hc, cx, cy, sxy, nodes, lane, bestF, bestk,
                                       SPOLY ? s_poly : L.rpoly);
        } else {
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
        }
        pick_and_move(a, e, it, bestF, bestk, cx, cy, cz, sxy, sz, lane);
    }
    event_epilogue<TYPE>(a, e, s_sig, S, cx, cy, cz, lane);
}

// ---------------------------------------------------------------------------
// Separable evaluation of an XYZ grid.  For sensor i the node values
//   eta(x_j, y_k, z_l) = sum_{a,b,c} C[jz_l+c][jy_k+b][jx_j+a] wx_j,a wy_k,b wz_l,c
// are contracted one axis at a time through per-warp shared memory:
//   T1[zz][yy][j] = sum_a C[jz0+zz][jy0+yy][jx_j+a] wx_j,a     (x first)
//   T2[zz][k][j]  = sum_b T1[zz][jy_k-jy0+b][j] wy_k,b          (then y)
//   eta[l][k][j]  = sum_c T2[jz_l-jz0+c][k][j] wz_l,c           (then z)
// over the coefficient rows jy0.. and planes jz0.. that the grid touches.
// Once the spacing is below the knot spacing the grids touch a few rows and
// planes, and a node costs about 12 multiply-adds instead of 64 loads and
// multiply-adds.  Lanes own (row, x node) pairs in the first contraction and
// (y node, x node) columns in the other two, with the z loop inside, so the
// index arithmetic is done once per grid.  Limits: n_xy <= 7, n_z <= 8,
// n_xy x (rows touched) <= 32 kSepQ1.
// ---------------------------------------------------------------------------
constexpr int kSepAxis = 15, kSepQ1 = 5, kSepQ2 = 2, kSepZ = 8;

// per-warp shared memory of the separable path, after the 3 n_s floats
struct SepSmem {
    int t1, t2, tab;  // float offsets of T1, T2 and the axis tables
    int total;        // floats
    __host__ __device__ static SepSmem make(int n_xy, int n_z, int ry_cap, int rz_cap)
    {
        SepSmem m;
        m.t1 = 0;
        m.t2 = m.t1 + n_xy * ry_cap * rz_cap;
        m.tab = m.t2 + n_xy * n_xy * rz_cap;
        // per axis and node: 4 weights, span index, inside flag
        m.total = m.tab + 3 * kSepAxis * 6;
        m.total = (m.total + 3) & ~3;
        return m;
    }
};

// coefficient rows (or planes) a grid of n nodes, spacing s, can touch
__host__ __device__ inline int sep_rows(int n, float s, float inv_h, int n_int)
{
    const int span = (int)floorf((float)(n - 1) * s * inv_h) + 2;  // distinct spans, with rounding slack
    const int r = span + 3;
    return r < n_int + 3 ? r : n_int + 3;
}

__device__ __forceinline__ void cgs_event_xyz_sep(const CgsArgs &a, long e, float *s_sig, float *s_ic, float *s_ec,
                                                  float *sep, int lane)
{
    const LrfDev &L = a.L;
    const int NX = a.n_xy, NZ = a.n_z, NXX = NX * NX;
    const int nodes = NXX * NZ;
    const int c_xy = (NX - 1) / 2, c_z = (NZ - 1) / 2;
    const SepSmem sm = SepSmem::make(NX, NZ, a.ry_cap, a.rz_cap);
    float *T1 = sep + sm.t1, *T2 = sep + sm.t2;
    float *W = sep + sm.tab;                                  // [3][kSepAxis][4] weights
    int *J = reinterpret_cast<int *>(W + 3 * kSepAxis * 4);   // [3][kSepAxis] span index
    int *OK = J + 3 * kSepAxis;                               // [3][kSepAxis] node inside the box
    float S, cx, cy, cz;
    if (!event_prologue<ANTS_LRF_XYZ>(a, e, s_sig, lane, S, cx, cy, cz)) return;
    float sxy = a.step_xy, sz = a.step_z;
    for (int it = 0; it < a.iters; ++it) {
        const float inv_hc = centre_values<ANTS_LRF_XYZ>(L, s_ic, s_ec, cx, cy, cz, lane);
        // node coordinates along each axis: span, weights, inside flag
        for (int t = lane; t < 2 * NX + NZ; t += 32) {
            const int ax = t < NX ? 0 : (t < 2 * NX ? 1 : 2);
            const int q = ax == 0 ? t : (ax == 1 ? t - NX : t - 2 * NX);
            const float c0 = ax == 0 ? cx : (ax == 1 ? cy : cz);
            const float v = ax < 2 ? fmaf((float)(q - c_xy), sxy, c0) : fmaf((float)(q - c_z), sz, c0);
            float tt, w[4];
            const int j = bs_span(v, L.lo[ax], L.inv_h[ax], L.n_int[ax], tt);
            bs_weights(tt, w);
            float *wq = W + (ax * kSepAxis + q) * 4;
            wq[0] = w[0];
            wq[1] = w[1];
            wq[2] = w[2];
            wq[3] = w[3];
            J[ax * kSepAxis + q] = j;
            OK[ax * kSepAxis + q] = v >= L.lo[ax] && v <= L.hi[ax];
        }
        __syncwarp();
        const int jy0 = J[kSepAxis], jz0 = J[2 * kSepAxis];
        const int Ry = J[kSepAxis + NX - 1] - jy0 + 4, Rz = J[2 * kSepAxis + NZ - 1] - jz0 + 4;
        float bestF = -INFINITY;
        int bestk = 0x7fffffff;
        if (Ry > a.ry_cap || Rz > a.rz_cap || NX * Ry > 32 * kSepQ1) {
            // the grid touches more rows than the tables hold (not expected for
            // the caps the launcher derives): evaluate every node on its own
            for (int k = lane; k < nodes; k += 32) {
                int ix = k % NX, iy = (k / NX) % NX, iz = k / NXX;
                float x = fmaf((float)(ix - c_xy), sxy, cx);
                float y = fmaf((float)(iy - c_xy), sxy, cy);
                float z = fmaf((float)(iz - c_z), sz, cz);
                float F = node_score<ANTS_LRF_XYZ>(L, s_sig, s_ic, s_ec, S, inv_hc, x, y, z);
                if (F > bestF) {
                    bestF = F;
                    bestk = k;
                }
            }
        } else {
            // this lane's (row, x node) pairs of the first contraction
            int co[kSepQ1], to[kSepQ1];
            float wx[kSepQ1][4];
#pragma unroll
            for (int q = 0; q < kSepQ1; ++q) {
                const int p = lane + 32 * q;
                const int j = p % NX, yy = p / NX;
                co[q] = p < NX * Ry ? yy * L.stride_y + J[j] : -1;
                to[q] = yy * NX + j;
#pragma unroll
                for (int c = 0; c < 4; ++c) wx[q][c] = W[j * 4 + c];
            }
            // this lane's (y node, x node) columns of the other two
            int r2[kSepQ2];
            float wy[kSepQ2][4];
#pragma unroll
            for (int q = 0; q < kSepQ2; ++q) {
                const int p = lane + 32 * q;
                const int j = p % NX, k = p / NX;
                r2[q] = p < NXX ? (J[kSepAxis + k] - jy0) * NX + j : -1;
#pragma unroll
                for (int c = 0; c < 4; ++c) wy[q][c] = W[(kSepAxis + (k < NX ? k : 0)) * 4 + c];
            }
            float acc[kSepQ2 * kSepZ], dH[kSepQ2 * kSepZ];
#pragma unroll
            for (int m = 0; m < kSepQ2 * kSepZ; ++m) acc[m] = dH[m] = 0.0f;
            const int t1_plane = Ry * NX;
            for (int i = 0; i < L.n_s; ++i) {
                const float *C = L.coef + (size_t)i * L.n_coef + (size_t)jz0 * L.stride_z + (size_t)jy0 * L.stride_y;
#pragma unroll
                for (int q = 0; q < kSepQ1; ++q)
                    if (co[q] >= 0)
                        for (int zz = 0; zz < Rz; ++zz) {
                            const float *c = C + zz * L.stride_z + co[q];
                            float f = __ldg(c) * wx[q][0];
                            f = fmaf(__ldg(c + 1), wx[q][1], f);
                            f = fmaf(__ldg(c + 2), wx[q][2], f);
                            f = fmaf(__ldg(c + 3), wx[q][3], f);
                            T1[zz * t1_plane + to[q]] = f;
                        }
                __syncwarp();
#pragma unroll
                for (int q = 0; q < kSepQ2; ++q)
                    if (r2[q] >= 0)
                        for (int zz = 0; zz < Rz; ++zz) {
                            const float *c = T1 + zz * t1_plane + r2[q];
                            float f = c[0] * wy[q][0];
                            f = fmaf(c[NX], wy[q][1], f);
                            f = fmaf(c[2 * NX], wy[q][2], f);
                            f = fmaf(c[3 * NX], wy[q][3], f);
                            T2[zz * NXX + lane + 32 * q] = f;
                        }
                __syncwarp();
                const float si = s_sig[i], ici = s_ic[i], eci = s_ec[i];
#pragma unroll
                for (int iz = 0; iz < kSepZ; ++iz) {
                    if (iz < NZ) {
                        const float *wz = W + (2 * kSepAxis + iz) * 4;
                        const float *c = T2 + (J[2 * kSepAxis + iz] - jz0) * NXX;
#pragma unroll
                        for (int q = 0; q < kSepQ2; ++q)
                            if (r2[q] >= 0) {
                                const float *cq = c + lane + 32 * q;
                                float f = cq[0] * wz[0];
                                f = fmaf(cq[NXX], wz[1], f);
                                f = fmaf(cq[2 * NXX], wz[2], f);
                                f = fmaf(cq[3 * NXX], wz[3], f);
                                const float eta = fmaxf(f, kEtaFloor);
                                acc[q * kSepZ + iz] = fmaf(si, __log2f(eta * ici), acc[q * kSepZ + iz]);
                                dH[q * kSepZ + iz] += eta - eci;
                            }
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int iz = 0; iz < kSepZ; ++iz)
#pragma unroll
                for (int q = 0; q < kSepQ2; ++q) {
                    const int p = lane + 32 * q;
                    if (iz < NZ && p < NXX) {
                        const int k = iz * NXX + p, ix = p % NX, iy = p / NX;
                        const bool inside = OK[ix] && OK[kSepAxis + iy] && OK[2 * kSepAxis + iz];
                        const float F = inside ? acc[q * kSepZ + iz] -
                                                     S * (log1pf(dH[q * kSepZ + iz] * inv_hc) * 1.4426950408889634f)
                                               : -INFINITY;
                        if (F > bestF || (F == bestF && k < bestk)) {
                            bestF = F;
                            bestk = k;
                        }
                    }
                }
        }
        pick_and_move(a, e, it, bestF, bestk, cx, cy, cz, sxy, sz, lane);
    }
    event_epilogue<ANTS_LRF_XYZ>(a, e, s_sig, S, cx, cy, cz, lane);
}

// floats of shared memory one warp needs for an item
__host__ inline int warp_smem_floats(const CgsArgs &a)
{
    int f = 3 * a.L.n_s;
    f = (f + 3) & ~3;
    if (a.sep) f += SepSmem::make(a.n_xy, a.n_z, a.ry_cap, a.rz_cap).total;
    return f;
}

// enable the separable XYZ path when the grid fits it
__host__ inline void setup_sep(CgsArgs &a)
{
    a.sep = 0;
    a.ry_cap = a.rz_cap = 0;
    if (a.L.type != ANTS_LRF_XYZ || a.n_xy * a.n_xy > 32 * kSepQ2 || a.n_z > kSepZ) return;
    const int ry = sep_rows(a.n_xy, a.step_xy, a.L.inv_h[1], a.L.n_int[1]);
    if (a.n_xy * ry > 32 * kSepQ1) return;
    a.sep = 1;
    a.ry_cap = ry;
    a.rz_cap = sep_rows(a.n_z, a.step_z, a.L.inv_h[2], a.L.n_int[2]);
}

template <int TYPE, bool SPOLY>
__global__ void __launch_bounds__(256, TYPE == ANTS_LRF_XYZ ? 2 : 3) cgs_plain_kernel(CgsArgs a, int warp_floats,
                                                                                     int n_poly)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int n_s = a.L.n_s;
    float *s_sig = smem + (size_t)wib * warp_floats;
    float *s_ic = s_sig + n_s;  // 1 / eta_i(centre)
    float *s_ec = s_ic + n_s;   // eta_i(centre)
    float *sep = s_sig + ((3 * n_s + 3) & ~3);
    // SPOLY (radial): the power-basis cubics copied once per block
    float4 *s_poly = nullptr;
    if (SPOLY) {
        s_poly = (float4 *)(smem + (((size_t)wpb * warp_floats + 3) & ~(size_t)3));
        for (int k = threadIdx.x; k < n_poly; k += blockDim.x) s_poly[k] = a.L.rpoly[k];
        __syncthreads();
    }
    for (long e = (long)blockIdx.x * wpb + wib; e < a.n_e; e += (long)gridDim.x * wpb) {
        if (TYPE == ANTS_LRF_XYZ && a.sep)
            cgs_event_xyz_sep(a, e, s_sig, s_ic, s_ec, sep, lane);
        else
            cgs_event<TYPE, SPOLY>(a, e, s_sig, s_ic, s_ec, lane, s_poly);
    }
}

template <int TYPE>
int launch_typed(const ants_ctx *ctx, CgsArgs a, cudaStream_t stream, bool allow_sep = true)
{
    if (allow_sep) setup_sep(a);
    else a.sep = 0;
    const int warp_floats = warp_smem_floats(a);
    int wpb = 8;
    while (wpb > 1 && (size_t)wpb * warp_floats * sizeof(float) > ctx->smem_optin) wpb /= 2;
    if ((size_t)wpb * warp_floats * sizeof(float) > ctx->smem_optin && a.sep) {
        return launch_typed<TYPE>(ctx, a, stream, false);  // tables too large: per-node evaluation
    }
    const int threads = 32 * wpb;
    size_t smem = (size_t)wpb * warp_floats * sizeof(float);
    // radial cubics in shared memory when they take at most 32 KB
    int n_poly = 0;
    if (TYPE == ANTS_LRF_RADIAL) {
        const long np = (long)a.L.n_sets * a.L.n_int[0];
        if (np * 16 <= 32 * 1024) {
            n_poly = (int)np;
            smem = ((smem + 15) & ~(size_t)15) + (size_t)np * 16;
        }
    }
    if (smem > ctx->smem_optin) return fail(ANTS_E_SHAPE, "cgs: %d sensors need too much shared memory", a.L.n_s);
    long blocks = (a.n_e + wpb - 1) / wpb;
    long cap = (long)ctx->n_sm * (64 / wpb);
    if (blocks > cap) blocks = cap;
    if (TYPE == ANTS_LRF_RADIAL && n_poly > 0) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(cgs_plain_kernel<ANTS_LRF_RADIAL, true>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_plain)");
        }
        cgs_plain_kernel<ANTS_LRF_RADIAL, true><<<(unsigned)blocks, threads, smem, stream>>>(a, warp_floats, n_poly);
    } else {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(cgs_plain_kernel<TYPE, false>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_plain)");
        }
        cgs_plain_kernel<TYPE, false><<<(unsigned)blocks, threads, smem, stream>>>(a, warp_floats, 0);
    }
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
    if (p->n_z > 1 && !lrf_is_3d(lrf->type))
        return fail(ANTS_E_ARG, "cgs params: n_z > 1 needs an LRF with a z coordinate");
    if (p->iters < 1 || p->iters > 32) return fail(ANTS_E_ARG, "cgs params: iters %d not in [1, 32]", p->iters);
    if (!(p->shrink > 0.0f && p->shrink < 1.0f)) return fail(ANTS_E_ARG, "cgs params: shrink must be in (0, 1)");
    if (!(p->step_xy > 0.0f) || !isfinite(p->step_xy)) return fail(ANTS_E_ARG, "cgs params: step_xy must be > 0");
    if (lrf_is_3d(lrf->type) && p->n_z > 1 && !(p->step_z > 0.0f))
        return fail(ANTS_E_ARG, "cgs params: step_z must be > 0");
    return ANTS_OK;
}

int launch_cgs_plain(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig,
                     long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                     int16_t *trace, cudaStream_t stream)
{
    return launch_cgs_rows(ctx, lrf, p, sig, 1, n_e, start, xyz, E, logL, status, trace, stream);
}

int launch_cgs_rows(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig,
                    int row_div, long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                    int16_t *trace, cudaStream_t stream)
{
    if (cgs_xy_supported(lrf, p))
        return launch_cgs_xy(ctx, lrf, p, sig, row_div, nullptr, n_e, start, xyz, E, logL, status, trace, stream);
    if (lrf->type > ANTS_LRF_XYZ || !lrf->ops.empty()) {
        // composite, axial+z, sliced and XY symmetry-class sets: the per-node
        // kernel of the variants with no option set is this search
        if (row_div != 1) return fail(ANTS_E_UNIMPLEMENTED, "cgs: shared signal rows need an XY LRF");
        ants_cgs_variant_params v{};
        v.grid = p;
        return reconstruct_variant(ctx, lrf, v, sig, n_e, start, xyz, E, logL, status, trace, stream);
    }
    CgsArgs a;
    a.row_div = row_div;
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

// ---------------------------------------------------------------------------
// Batched persistent launch over several detectors (one work queue)
// ---------------------------------------------------------------------------

namespace ants {
namespace {

struct BatchUnit {
    int item;    // index into the items
    int count;   // events in this unit
    long first;  // first event of the unit
};

// Persistent warps take units from a global counter (largest work first) and
// reconstruct their events with the per-event search of the unit's detector.
__global__ void __launch_bounds__(256) cgs_batched_kernel(const CgsArgs *__restrict__ items,
                                                          const BatchUnit *__restrict__ units, int n_units,
                                                          int *__restrict__ counter, int warp_floats)
{
    extern __shared__ float smem[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float *base = smem + (size_t)wib * warp_floats;
    for (;;) {
        int u = 0;
        if (lane == 0) u = atomicAdd(counter, 1);
        u = __shfl_sync(kFull, u, 0);
        if (u >= n_units) break;
        const BatchUnit U = units[u];
        const CgsArgs a = items[U.item];
        const long end = U.first + U.count;
        const int n_s = a.L.n_s;
        float *s_sig = base, *s_ic = base + n_s, *s_ec = base + 2 * n_s;
        float *sep = base + ((3 * n_s + 3) & ~3);
        switch (a.L.type) {
        case ANTS_LRF_RADIAL:
            for (long e = U.first; e < end; ++e) cgs_event<ANTS_LRF_RADIAL>(a, e, s_sig, s_ic, s_ec, lane);
            break;
        case ANTS_LRF_XY:
            for (long e = U.first; e < end; ++e) cgs_event<ANTS_LRF_XY>(a, e, s_sig, s_ic, s_ec, lane);
            break;
        default:
            if (a.sep)
                for (long e = U.first; e < end; ++e) cgs_event_xyz_sep(a, e, s_sig, s_ic, s_ec, sep, lane);
            else
                for (long e = U.first; e < end; ++e) cgs_event<ANTS_LRF_XYZ>(a, e, s_sig, s_ic, s_ec, lane);
            break;
        }
    }
}

}  // namespace
}  // namespace ants

struct ants_batch_plan {
    ants_ctx *ctx = nullptr;
    int device = 0;
    std::vector<ants_batch_item> items;
    ants_batch_config cfg{};
    ants::CgsArgs *d_items = nullptr;
    ants::BatchUnit *d_units = nullptr;
    int *d_counter = nullptr;
    int n_units = 0, warp_floats = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace ants {
namespace {

void release_plan_device(ants_batch_plan *P)
{
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    cudaFree(P->d_items);
    cudaFree(P->d_units);
    cudaFree(P->d_counter);
    P->exec = nullptr;
    P->graph = nullptr;
    P->d_items = nullptr;
    P->d_units = nullptr;
    P->d_counter = nullptr;
}

// (Re)build the work list and the captured graph for the plan's config;
// event_cap > 0 limits every detector to its first event_cap events.
int build_plan(ants_batch_plan *P, long event_cap)
{
    release_plan_device(P);
    const ants_ctx *ctx = P->ctx;
    const int n_items = (int)P->items.size();
    std::vector<CgsArgs> args(n_items);
    std::vector<BatchUnit> units;
    std::vector<double> cost;
    P->warp_floats = 4;
    for (int k = 0; k < n_items; ++k) {
        const ants_batch_item &it = P->items[k];
        CgsArgs &a = args[k];
        a.L = it.lrf->dev;
        a.n_xy = it.params.n_xy;
        a.n_z = it.params.n_z;
        a.iters = it.params.iters;
        a.shrink = it.params.shrink;
        a.step_xy = it.params.step_xy;
        a.step_z = it.params.step_z;
        a.z0 = it.params.z0;
        a.sig = it.signals_dev;
        a.n_e = it.n_events;
        a.row_div = 1;
        a.start = it.start_xyz_dev;
        a.xyz = it.xyz_dev;
        a.E = it.E_dev;
        a.logL = it.logL_dev;
        a.status = it.status_dev;
        a.trace = it.trace_dev;
        setup_sep(a);
        P->warp_floats = std::max(P->warp_floats, warp_smem_floats(a));
        const long n = event_cap > 0 ? std::min(event_cap, it.n_events) : it.n_events;
        const double per_event = (double)a.n_xy * a.n_xy * a.n_z * a.iters * it.lrf->n_s;
        for (long f = 0; f < n; f += P->cfg.unit_events) {
            BatchUnit u{k, (int)std::min<long>(P->cfg.unit_events, n - f), f};
            units.push_back(u);
            cost.push_back(per_event * u.count);
        }
    }
    // largest units first; ties in (item, first) order
    std::vector<int> order(units.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<BatchUnit> sorted(units.size());
    for (size_t i = 0; i < order.size(); ++i) sorted[i] = units[order[i]];
    P->n_units = (int)sorted.size();
    ANTS_CUDA_TRY(cudaMalloc(&P->d_items, sizeof(CgsArgs) * std::max(1, n_items)), "plan items");
    ANTS_CUDA_TRY(cudaMalloc(&P->d_units, sizeof(BatchUnit) * std::max<size_t>(1, sorted.size())), "plan units");
    ANTS_CUDA_TRY(cudaMalloc(&P->d_counter, 256), "plan counter");
    ANTS_CUDA_TRY(cudaMemcpy(P->d_items, args.data(), sizeof(CgsArgs) * n_items, cudaMemcpyHostToDevice), "upload");
    if (!sorted.empty())
        ANTS_CUDA_TRY(cudaMemcpy(P->d_units, sorted.data(), sizeof(BatchUnit) * sorted.size(), cudaMemcpyHostToDevice),
                      "upload");
    const int threads = 32 * P->cfg.warps_per_block;
    const size_t smem = (size_t)P->cfg.warps_per_block * P->warp_floats * sizeof(float);
    if (smem > ctx->smem_optin)
        return fail(ANTS_E_SHAPE, "batch: %d warps of %d floats exceed the shared memory of a block",
                    P->cfg.warps_per_block, P->warp_floats);
    ANTS_CUDA_TRY(cudaFuncSetAttribute(cgs_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "cudaFuncSetAttribute(batched)");
    const unsigned blocks = (unsigned)(ctx->n_sm * P->cfg.blocks_per_sm);
    if (!P->cap) ANTS_CUDA_TRY(cudaStreamCreateWithFlags(&P->cap, cudaStreamNonBlocking), "plan stream");
    // the run is one graph: reset the work counter, launch the persistent kernel
    ANTS_CUDA_TRY(cudaStreamBeginCapture(P->cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaMemsetAsync(P->d_counter, 0, sizeof(int), P->cap);
    cgs_batched_kernel<<<blocks, threads, smem, P->cap>>>(P->d_items, P->d_units, P->n_units, P->d_counter,
                                                         P->warp_floats);
    cudaError_t e1 = cudaGetLastError();
    cudaError_t e2 = cudaStreamEndCapture(P->cap, &P->graph);
    if (e1 != cudaSuccess) return cuda_fail(e1, "batched launch (capture)");
    if (e2 != cudaSuccess) return cuda_fail(e2, "end capture");
    ANTS_CUDA_TRY(cudaGraphInstantiate(&P->exec, P->graph, 0), "graph instantiate");
    return ANTS_OK;
}

int check_config(const ants_batch_config &c)
{
    if (c.unit_events < 1 || c.unit_events > (1 << 20) || c.warps_per_block < 1 || c.warps_per_block > 8 ||
        c.blocks_per_sm < 1 || c.blocks_per_sm > 32)
        return fail(ANTS_E_ARG, "batch config: unit_events 1..2^20, warps_per_block 1..8, blocks_per_sm 1..32");
    return ANTS_OK;
}

std::string plan_signature(const ants_batch_plan *P)
{
    std::string sig;
    char buf[128];
    for (const auto &it : P->items) {
        snprintf(buf, sizeof buf, "%d:%d:%d:%d:%d:%d:%ld;", it.lrf->type, it.lrf->n_s, it.lrf->n_coef,
                 it.params.n_xy * it.params.n_xy * it.params.n_z, it.params.iters, 0, it.n_events);
        sig += buf;
    }
    return sig;
}

}  // namespace
}  // namespace ants

extern "C" {

ANTS_API int ants_batch_plan_create(ants_ctx *ctx, int n_items, const ants_batch_item *items,
                                    const ants_batch_config *cfg, ants_batch_plan **out)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_batch_plan_create");
    if (!out) return fail(ANTS_E_ARG, "ants_batch_plan_create: out is NULL");
    *out = nullptr;
    if (!ctx || n_items < 1 || n_items > 4096 || !items) return fail(ANTS_E_ARG, "ants_batch_plan_create: bad items");
    for (int k = 0; k < n_items; ++k) {
        const ants_batch_item &it = items[k];
        if (!it.lrf || it.lrf->ctx != ctx) return fail(ANTS_E_ARG, "batch item %d: LRF of another context", k);
        if (it.lrf->type > ANTS_LRF_XYZ || !it.lrf->ops.empty())
            return fail(ANTS_E_UNIMPLEMENTED, "batch item %d: RADIAL, XY and XYZ LRFs only (no XY classes)", k);
        if (it.n_events < 0) return fail(ANTS_E_ARG, "batch item %d: n_events < 0", k);
        if (it.n_events > 0 && (!it.signals_dev || !it.xyz_dev || !it.E_dev || !it.logL_dev || !it.status_dev))
            return fail(ANTS_E_ARG, "batch item %d: NULL buffer", k);
        int rc = check_cgs_params(it.lrf, &it.params);
        if (rc != ANTS_OK) return rc;
    }
    ants_batch_config c = cfg ? *cfg : ants_batch_config{16, 8, 4};
    int rc = check_config(c);
    if (rc != ANTS_OK) return rc;
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    ants_batch_plan *P = new (std::nothrow) ants_batch_plan();
    if (!P) return fail(ANTS_E_OOM, "ants_batch_plan_create: out of host memory");
    P->ctx = ctx;
    P->device = ctx->device;
    P->items.assign(items, items + n_items);
    P->cfg = c;
    rc = build_plan(P, 0);
    if (rc != ANTS_OK) {
        std::string keep = ants_last_error();
        ants_batch_plan_free(P);
        return fail(rc, "%s", keep.c_str());
    }
    *out = P;
    return ANTS_OK;
}

ANTS_API int ants_batch_run(ants_batch_plan *P, void *stream)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_batch_run");
    if (!P || !P->exec) return fail(ANTS_E_ARG, "ants_batch_run: no plan");
    ANTS_CUDA_TRY(cudaSetDevice(P->ctx->device), "cudaSetDevice");
    ANTS_CUDA_TRY(cudaGraphLaunch(P->exec, (cudaStream_t)stream), "graph launch");
    count_launch();
    return ANTS_OK;
}

ANTS_API int ants_batch_get_config(const ants_batch_plan *P, ants_batch_config *cfg)
{
    using namespace ants;
    begin_call();
    if (!P || !cfg) return fail(ANTS_E_ARG, "ants_batch_get_config: NULL argument");
    *cfg = P->cfg;
    return ANTS_OK;
}

ANTS_API int ants_batch_autotune(ants_batch_plan *P, const char *cache_path, long events_per_item,
                                 ants_batch_config *chosen)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_batch_autotune");
    if (!P) return fail(ANTS_E_ARG, "ants_batch_autotune: no plan");
    if (events_per_item < 1) events_per_item = 2048;
    ANTS_CUDA_TRY(cudaSetDevice(P->ctx->device), "cudaSetDevice");
    const std::string sig = plan_signature(P);
    // cached choice for this batch signature
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "r")) {
            char line[8192];
            while (fgets(line, sizeof line, f)) {
                char key[8000];
                ants_batch_config c;
                if (sscanf(line, "%7999s %d %d %d", key, &c.unit_events, &c.warps_per_block, &c.blocks_per_sm) == 4 &&
                    sig == key && check_config(c) == ANTS_OK) {
                    fclose(f);
                    P->cfg = c;
                    int rc = build_plan(P, 0);
                    if (rc == ANTS_OK && chosen) *chosen = c;
                    return rc;
                }
            }
            fclose(f);
        }
    }
    const int units[] = {4, 16, 64};
    const int warps[] = {4, 8};
    const int blocks[] = {2, 4, 8};
    ants_batch_config best = P->cfg;
    float best_ms = INFINITY;
    cudaEvent_t e0, e1;
    ANTS_CUDA_TRY(cudaEventCreate(&e0), "event");
    ANTS_CUDA_TRY(cudaEventCreate(&e1), "event");
    int rc = ANTS_OK;
    for (int u : units)
        for (int w : warps)
            for (int b : blocks) {
                if (rc != ANTS_OK) break;
                if (w * b > 64) continue;  // at most 64 warps per SM
                // blocks beyond what one SM holds at once only wait for an
                // empty queue: skip shapes whose blocks cannot all be resident
                int resident = 0;
                const size_t smem_b = (size_t)w * P->warp_floats * sizeof(float);
                if (smem_b <= P->ctx->smem_optin) {
                    cudaFuncSetAttribute(cgs_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_b);
                    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, cgs_batched_kernel, 32 * w, smem_b);
                }
                if (resident < b) continue;
                P->cfg = ants_batch_config{u, w, b};
                rc = build_plan(P, events_per_item);
                if (rc != ANTS_OK) break;
                float ms = 0.0f;
                cudaGraphLaunch(P->exec, P->cap);  // warm-up
                cudaEventRecord(e0, P->cap);
                cudaGraphLaunch(P->exec, P->cap);
                cudaGraphLaunch(P->exec, P->cap);
                cudaEventRecord(e1, P->cap);
                cudaError_t e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) {
                    rc = cuda_fail(e, "autotune timing");
                    break;
                }
                if (ms < best_ms) {
                    best_ms = ms;
                    best = P->cfg;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != ANTS_OK) return rc;
    P->cfg = best;
    rc = build_plan(P, 0);
    if (rc != ANTS_OK) return rc;
    if (chosen) *chosen = best;
    if (cache_path) {
        if (FILE *f = fopen(cache_path, "a")) {
            fprintf(f, "%s %d %d %d\n", sig.c_str(), best.unit_events, best.warps_per_block, best.blocks_per_sm);
            fclose(f);
        }
    }
    count_launch(0);
    return ANTS_OK;
}

ANTS_API void ants_batch_plan_free(ants_batch_plan *P)
{
    if (!P) return;
    cudaSetDevice(P->device);
    ants::release_plan_device(P);
    if (P->cap) cudaStreamDestroy(P->cap);
    delete P;
    (void)cudaGetLastError();
}

}  // extern "C"
