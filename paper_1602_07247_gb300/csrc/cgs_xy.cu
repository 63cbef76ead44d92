// Contracting-grid ML search for XY LRFs (Sec. 5.1.2.2 with the XY LRFs of
// Sec. 6.1.1), separable form, FP32.
//
// Decomposition: a team of TEAM warps reconstructs one event at a time
// (teams grid-stride over events; a block holds several teams and one
// shared copy of the coefficient table).  Team lane t < N*Q is
// (slot q = t / N, grid column j = t % N), Q = 32*TEAM / N.  Sensors are
// interleaved in pairs (float2 coefficients), and slot q owns pairs
// q, q+Q, q+2Q, ...; a lane processes them PPL at a time so that PPL
// independent dependency chains are in flight (11 x 11 grids: teams of three
// warps, Q = 8, four pairs per lane, 88 of 96 lanes busy; a grid row's fixed
// work is spread over eight evaluations per lane).  Only the grid rows inside
// the LRF box are swept (the others score -inf), and grids whose rows all
// share one 4-row window skip the window bookkeeping.
//
// Column trick: every node of column j shares x_j, so with
//   T[r] = sum_b wx_j[b] C[r][ix_j + b]          (x-contracted row r)
//   eta(x_j, y_k) = sum_a wy_k[a] T[iy_k + a],
// a 4-row window of T slides along y and only rows entering it are loaded.
//
// Per node and sensor, relative to the grid centre c (log2 units):
//   acc += s log2(eta / eta_c),  dH += eta - eta_c,
// and F = acc - S log2(1 + dH / H_c) is the Poisson log-likelihood with the
// energy E = S/H profiled out (Sec. 5.1.2.2), up to a per-event constant.
// On grids narrower than a quarter of a knot interval the nodes' scores differ
// by less than the error of the hardware log2 near 1 (about 2^-22 absolute per
// term) plus the rounding of eta/eta_c to single precision; there the term is
// log2(1 + u) with u = fma(eta, 1/eta_c, -1) (one rounding of the small
// difference) and a degree-4 Taylor polynomial (truncation below 9e-9 for
// |u| <= 1/32, below 1e-9 for the |u| <= 0.02 such grids see; larger |u|
// falls back to the hardware log2).  The rounding of 1/eta_c
// shifts every node of a grid by the same s log2(1 + d) and cancels in the
// argmax.
// Lanes store per-(node, slot) partial sums in shared memory; one thread per
// node adds the slots, and a team argmax (ties to the lowest flat index)
// picks the next centre.
#include <cmath>
#include <type_traits>

#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;
constexpr float kInvLn2 = 1.4426950408889634f;
constexpr int kXyThreads = 512;  // 16 warps per block (teams that fit: 15 with 3-warp teams), one block per SM

struct XyArgs {
    LrfDev L;
    int iters;
    float shrink, step_xy;
    float prec_halfwidth;  // grids whose half-width is at most this use the accurate log
    const float *sig;
    long n_e;
    int row_div;      // event e reads signal row e / row_div ...
    const int *rows;  // ... or rows[e] when given
    const float *start;
    float *xyz, *E, *logL;
    int32_t *status;
    int16_t *trace;
};

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 fmul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// 64-bit load of one coefficient pair: from shared memory by 32-bit address,
// or through the read-only path when the table stays in global memory
template <bool SMEM>
__device__ __forceinline__ float2 ldc(const float2 *gptr, unsigned saddr)
{
    if (SMEM) {
        float2 v;
        asm("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(saddr));
        return v;
    }
    return __ldg(gptr);
}

// log2(1 + u) for both lanes of a pair: Taylor series sum_k (-1)^(k+1) u^k /
// (k ln 2) to degree 4 (truncation below 9e-9 for |u| <= 1/32); the callers
// record an |u| beyond that and redo those terms with the hardware log2
constexpr float kNearOne = 0.03125f;
__device__ __forceinline__ float2 log2_1p_taylor(float2 u)
{
    float2 p = ffma2(u, make_float2(-0.36067376022224085f, -0.36067376022224085f),
                     make_float2(0.48089834696298783f, 0.48089834696298783f));
    p = ffma2(p, u, make_float2(-0.72134752044448170f, -0.72134752044448170f));
    p = ffma2(p, u, make_float2(1.4426950408889634f, 1.4426950408889634f));
    return fmul2(p, u);
}

// log2 of a positive ratio by the hardware approximation, subnormal inputs
// flushed.  Without the floor every LRF value lies between the smallest and
// the largest coefficient (B-spline partition of unity), and the host takes
// that path only when their ratio is at most 2^100, so every ratio of two
// values is a normal float.  With the floor the argument is first raised to
// the smallest normal float: a node whose value lies more than 2^126 below
// the centre's keeps a finite term (a sensor without signal adds 0).
template <bool FLOOR>
__device__ __forceinline__ float log2_ratio(float r)
{
    float y;
    if (FLOOR) r = fmaxf(r, 1.17549435e-38f);
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(r));
    return y;
}

__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
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

// eta of both sensors of pair p at one point inside the box
__device__ __forceinline__ float2 pair_eta(const LrfDev &L, const float2 *coef2, int p, float x, float y)
{
    float tx, ty, wx[4], wy[4];
    int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
    int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
    bs_weights(tx, wx);
    bs_weights(ty, wy);
    const float2 *c = coef2 + (size_t)p * L.pair_stride + jy * L.stride_y + jx;
    float2 f = make_float2(0.0f, 0.0f);
    const long lo_i = c - coef2, n_tab = (long)L.n_pairs * L.pair_stride;
    if (!ANTS_IN_RANGE(L.dbg, lo_i, n_tab, 101) || !ANTS_IN_RANGE(L.dbg, lo_i + 3 * L.stride_y + 3, n_tab, 102))
        return f;
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

// eta of both sensors of pair p at one point inside the box, from the
// pair-fastest copy (lanes taking consecutive pairs read contiguous runs)
__device__ __forceinline__ float2 pair_eta_pf(const LrfDev &L, int p, float x, float y)
{
    float tx, ty, wx[4], wy[4];
    const int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
    const int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
    bs_weights(tx, wx);
    bs_weights(ty, wy);
    const int np = L.n_pairs;
    const float2 *c = L.coef2_pf + ((size_t)jy * L.stride_y + jx) * np + p;
    float2 f = make_float2(0.0f, 0.0f);
    const long n_tab = (long)np * L.pair_stride, hi_i = ((long)(jy + 3) * L.stride_y + jx + 3) * np + p;
    if (!ANTS_IN_RANGE(L.dbg, hi_i, n_tab, 105)) return f;
    const int rs = L.stride_y * np;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        float2 fr = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int a = 0; a < 4; ++a) fr = ffma2(make_float2(wx[a], wx[a]), __ldg(c + b * rs + a * np), fr);
        f = ffma2(make_float2(wy[b], wy[b]), fr, f);
    }
    return f;
}

// x-contracted row: sum_b wx[b] C[r][ix+b] for both sensors of a pair;
// `g` / `sa` address C[r][ix] (global pointer / shared byte address)
template <bool SMEM>
__device__ __forceinline__ float2 trow(const float2 *g, unsigned sa, const float2 wx2[4], const float2 *base, long n,
                                       int *dbg)
{
    if (!ANTS_IN_RANGE(dbg, g - base, n - 3, 103)) return make_float2(0.0f, 0.0f);
    float2 v = fmul2(wx2[0], ldc<SMEM>(g, sa));
    v = ffma2(wx2[1], ldc<SMEM>(g + 1, sa + 8), v);
    v = ffma2(wx2[2], ldc<SMEM>(g + 2, sa + 16), v);
    v = ffma2(wx2[3], ldc<SMEM>(g + 3, sa + 24), v);
    return v;
}

template <int TEAM>
__device__ __forceinline__ void team_sync(int team)
{
    if (TEAM == 1) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(team + 1), "r"(TEAM * 32) : "memory");
    }
}

// per-team shared-memory layout (floats): signals, 1/eta_c, eta_c [n_pad each],
// row bases as duplicated pairs [N][8] (16-byte aligned) and iy [N], partial
// sums acc then dH, reduction scratch [32].  Teams of several warps keep one
// partial per grid row, warp and grid column ([N][warps][N]: the lanes of a
// warp that share a column are summed by shuffles first); one-warp teams keep
// one per grid row and lane ([N][LT+N]: row stride N mod 32, so a warp of node
// threads reads 32 different banks)
// (disjoint slots per phase: argmax 0..7, centre H 8..11, final H 12..15,
// prologue sums 16..31, final logL 16..19)
struct TeamSmem {
    int n_pad, part_stride;
    // the one place the layout is defined, for the launcher and the kernel
    __device__ __host__ static TeamSmem make(int n_pad, int lt, int n)
    {
        return TeamSmem{n_pad, lt > 32 ? (lt / 32) * n : lt + n};
    }
    __device__ __host__ int sig() const { return 0; }
    __device__ __host__ int ic() const { return n_pad; }
    __device__ __host__ int ec() const { return 2 * n_pad; }  // holds -eta_c
    __device__ __host__ int rows() const { return (3 * n_pad + 3) & ~3; }
    __device__ __host__ int part(int N) const { return rows() + 9 * N; }
    __device__ __host__ int red(int N) const { return part(N) + 2 * N * part_stride; }
    __device__ __host__ int total(int N) const { return (red(N) + 32 + 3) & ~3; }
};

template <int N, int TEAM, int PPL, bool SMEM, bool FLOOR>
__global__ void __launch_bounds__(kXyThreads, 1) cgs_xy_kernel(XyArgs a, int teams_per_block, int team_floats)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LT = 32 * TEAM;  // lanes per team
    constexpr int Q = LT / N;      // sensor slots
    constexpr int C = (N - 1) / 2;
    const LrfDev &L = a.L;
    const int n_s = L.n_s, n_pairs = L.n_pairs, n_pad = 2 * n_pairs;
    const size_t table = SMEM ? (size_t)n_pairs * L.pair_stride : 0;  // float2 entries
    float2 *cs = reinterpret_cast<float2 *>(smem_raw);
    const float2 *coef2 = L.coef2;
    const long n_tab = (long)n_pairs * L.pair_stride;  // float2 entries of the table (index checks)
    (void)n_tab;
    if (SMEM) {
        const float4 *src = reinterpret_cast<const float4 *>(L.coef2);
        float4 *dst = reinterpret_cast<float4 *>(cs);
        for (size_t k = threadIdx.x; k < table / 2; k += blockDim.x) dst[k] = src[k];
        if ((table & 1) && threadIdx.x == 0) cs[table - 1] = L.coef2[table - 1];
        __syncthreads();
        coef2 = cs;
    }
    const size_t table_even = (table + 1) & ~(size_t)1;  // team data stays 16-byte aligned
    const int team = threadIdx.x / LT;
    if (team >= teams_per_block) return;  // no block-wide barrier follows
    const int t = threadIdx.x - team * LT;  // lane within the team
    const int lane = threadIdx.x & 31, wit = t >> 5;
    const TeamSmem lay = TeamSmem::make(n_pad, LT, N);
    float *ts = reinterpret_cast<float *>(cs + table_even) + (size_t)team * team_floats;
    float *s_sig = ts + lay.sig(), *s_ic = ts + lay.ic(), *s_ec = ts + lay.ec();
    float4 *s_wy = reinterpret_cast<float4 *>(ts + lay.rows());  // [N][2]: (w0,w0,w1,w1), (w2,w2,w3,w3)
    int *s_iy = reinterpret_cast<int *>(ts + lay.rows() + 8 * N);
    float *s_part = ts + lay.part(N);
    float *s_red = ts + lay.red(N);
    const float2 *s_sig2 = reinterpret_cast<const float2 *>(s_sig);
    const float2 *s_ic2 = reinterpret_cast<const float2 *>(s_ic);
    const float2 *s_ec2 = reinterpret_cast<const float2 *>(s_ec);

    const int q = t / N, j = t - q * N;
    const bool active = q < Q;
    const int pairs_mine = active ? (n_pairs - q + Q - 1) / Q : 0;  // pairs q, q+Q, ... below n_pairs
    // every lane runs the same number of pair groups (the shuffles of the
    // partial sums need the whole warp); missing pairs contribute zero
    const int group_end = ((n_pairs + Q - 1) / Q + PPL - 1) / PPL * PPL;
    const float qnan = __int_as_float(0x7fc00000);
    const long team_stride = (long)gridDim.x * teams_per_block;

    for (long e = (long)blockIdx.x * teams_per_block + team; e < a.n_e; e += team_stride) {
        // ---- prologue: signals, S, centroid, status ----------------------------
        const float *sg = a.sig + (size_t)(a.rows ? (long)a.rows[e] : e / a.row_div) * n_s;
        float S = 0.0f, Sx = 0.0f, Sy = 0.0f, Sw = 0.0f;
        int bad = 0;
        for (int i = t; i < n_pad; i += LT) {
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
        if (TEAM > 1) {
            if (lane == 0) {
                s_red[16 + 4 * wit] = S;
                s_red[16 + 4 * wit + 1] = Sx;
                s_red[16 + 4 * wit + 2] = Sy;
                s_red[16 + 4 * wit + 3] = bad ? -1.0f : Sw;
            }
            team_sync<TEAM>(team);
            S = Sx = Sy = Sw = 0.0f;
            bad = 0;
            for (int w = 0; w < TEAM; ++w) {
                S += s_red[16 + 4 * w];
                Sx += s_red[16 + 4 * w + 1];
                Sy += s_red[16 + 4 * w + 2];
                float v = s_red[16 + 4 * w + 3];
                bad |= v < 0.0f;
                Sw += v;
            }
        }
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
            if (t == 0) {
                a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = qnan;
                a.E[e] = qnan;
                a.logL[e] = qnan;
                a.status[e] = st;
            }
            if (a.trace)
                for (int it = t; it < a.iters; it += LT) a.trace[e * a.iters + it] = -1;
            team_sync<TEAM>(team);
            continue;
        }

        float sxy = a.step_xy;
        for (int it = 0; it < a.iters; ++it) {
            // ---- phase 1: centre values and row bases -------------------------
            float hc = 0.0f;
            for (int p = t; p < n_pairs; p += LT) {
                float2 ec = pair_eta(L, coef2, p, cx, cy);
                if (FLOOR) {
                    ec.x = fmaxf(ec.x, kEtaFloor);
                    ec.y = fmaxf(ec.y, kEtaFloor);
                }
                s_ec[2 * p] = -ec.x;
                s_ec[2 * p + 1] = -ec.y;
                s_ic[2 * p] = __frcp_rn(ec.x);
                s_ic[2 * p + 1] = __frcp_rn(ec.y);
                hc += ec.x + (2 * p + 1 < n_s ? ec.y : 0.0f);
            }
            if (t < N) {
                float ty, w[4];
                float y = fmaf((float)(t - C), sxy, cy);
                int iy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
                bs_weights(ty, w);
                s_wy[2 * t] = make_float4(w[0], w[0], w[1], w[1]);
                s_wy[2 * t + 1] = make_float4(w[2], w[2], w[3], w[3]);
                s_iy[t] = iy;
            }
            // grid rows inside the LRF box (the node scores below apply the
            // same test): a contiguous range, the only rows swept
            unsigned rows_in = 0;
            if (wit == 0) {
                const float y = fmaf((float)(lane - C), sxy, cy);
                rows_in = __ballot_sync(kFull, lane < N && y >= L.lo[1] && y <= L.hi[1]);
            }
            hc = warp_sum(hc);
            if (TEAM > 1) {
                if (lane == 0) {
                    s_red[8 + wit] = hc;
                    if (wit == 0) s_red[12] = __uint_as_float(rows_in);
                }
                team_sync<TEAM>(team);
                hc = 0.0f;
                for (int w = 0; w < TEAM; ++w) hc += s_red[8 + w];
                rows_in = __float_as_uint(s_red[12]);
            } else {
                __syncwarp();
            }
            const float inv_hc = __frcp_rn(hc);
            const int k_first = rows_in ? __ffs(rows_in) - 1 : 0, k_last = rows_in ? 31 - __clz(rows_in) : -1;

            // ---- phase 2: each lane sums its column over its sensor pairs -----
            const float x = fmaf((float)(j - C), sxy, cx);
            float tx, wxs[4];
            const int ix = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
            bs_weights(tx, wxs);
            float2 wx2[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) wx2[b] = make_float2(wxs[b], wxs[b]);
            const int ps = lay.part_stride;
            const int sy = L.stride_y;
            const unsigned rowb = (unsigned)sy * 8u;  // bytes per table row
            // the sweep is compiled twice, with the hardware log2 of eta/eta_c
            // and with the accurate log2(1 + u); the choice is uniform per grid
            // with the accurate log, `umax` tracks the largest |u| (beyond the
            // Taylor range the warp sweeps again with the hardware log2)
            float umax = 0.0f;
            auto sweep = [&](auto accurate) {
                constexpr bool ACC = decltype(accurate)::value;
                for (int g = 0; g < group_end; g += PPL) {
                    const float2 *gb[PPL];
                    unsigned sb[PPL];
                    float2 sp[PPL], ic[PPL], nec[PPL];
                    bool on[PPL];
    #pragma unroll
                    for (int m = 0; m < PPL; ++m) {
                        on[m] = g + m < pairs_mine;
                        const int p = on[m] ? q + (g + m) * Q : 0;  // any valid pair when missing
                        gb[m] = coef2 + (size_t)p * L.pair_stride + ix;
                        sb[m] = SMEM ? (unsigned)__cvta_generic_to_shared(gb[m]) : 0u;
                        sp[m] = on[m] ? s_sig2[p] : make_float2(0.0f, 0.0f);
                        ic[m] = s_ic2[p];
                        nec[m] = s_ec2[p];
                    }
                    float2 W[PPL][4];
                    int top = s_iy[k_first];
    #pragma unroll
                    for (int m = 0; m < PPL; ++m)
    #pragma unroll
                        for (int a4 = 0; a4 < 4; ++a4)
                            W[m][a4] = trow<SMEM>(gb[m] + (top + a4) * sy, sb[m] + (unsigned)(top + a4) * rowb, wx2, coef2, n_tab, L.dbg);
                    // grids whose rows all share one window (the fine grids) skip
                    // the window bookkeeping
                    auto rows = [&](auto fixed_window) {
                        constexpr bool FIXED = decltype(fixed_window)::value;
        #pragma unroll 1
                        for (int k = k_first; k <= k_last; ++k) {
                            if (!FIXED) {
                                const int iyk = s_iy[k];
                                const int adv = iyk - top;
                                const int r4 = top + 4;  // first row not yet in the window
                                if (adv == 1) {
            #pragma unroll
                                    for (int m = 0; m < PPL; ++m) {
                                        W[m][0] = W[m][1];
                                        W[m][1] = W[m][2];
                                        W[m][2] = W[m][3];
                                        W[m][3] = trow<SMEM>(gb[m] + r4 * sy, sb[m] + (unsigned)r4 * rowb, wx2, coef2, n_tab, L.dbg);
                                    }
                                } else if (adv == 2) {
            #pragma unroll
                                    for (int m = 0; m < PPL; ++m) {
                                        W[m][0] = W[m][2];
                                        W[m][1] = W[m][3];
                                        W[m][2] = trow<SMEM>(gb[m] + r4 * sy, sb[m] + (unsigned)r4 * rowb, wx2, coef2, n_tab, L.dbg);
                                        W[m][3] = trow<SMEM>(gb[m] + (r4 + 1) * sy, sb[m] + (unsigned)(r4 + 1) * rowb, wx2, coef2, n_tab, L.dbg);
                                    }
                                } else if (adv == 3) {
            #pragma unroll
                                    for (int m = 0; m < PPL; ++m) {
                                        W[m][0] = W[m][3];
                                        W[m][1] = trow<SMEM>(gb[m] + r4 * sy, sb[m] + (unsigned)r4 * rowb, wx2, coef2, n_tab, L.dbg);
                                        W[m][2] = trow<SMEM>(gb[m] + (r4 + 1) * sy, sb[m] + (unsigned)(r4 + 1) * rowb, wx2, coef2, n_tab, L.dbg);
                                        W[m][3] = trow<SMEM>(gb[m] + (r4 + 2) * sy, sb[m] + (unsigned)(r4 + 2) * rowb, wx2, coef2, n_tab, L.dbg);
                                    }
                                } else if (adv >= 4) {
            #pragma unroll
                                    for (int m = 0; m < PPL; ++m)
            #pragma unroll
                                        for (int a4 = 0; a4 < 4; ++a4)
                                            W[m][a4] = trow<SMEM>(gb[m] + (iyk + a4) * sy, sb[m] + (unsigned)(iyk + a4) * rowb,
                                                                  wx2, coef2, n_tab, L.dbg);
                                }
                                top = iyk;
                            }
                            const float4 wa = s_wy[2 * k], wb = s_wy[2 * k + 1];
                            const float2 w0 = make_float2(wa.x, wa.y), w1 = make_float2(wa.z, wa.w);
                            const float2 w2 = make_float2(wb.x, wb.y), w3 = make_float2(wb.z, wb.w);
                            float2 acc = make_float2(0.0f, 0.0f), dh = make_float2(0.0f, 0.0f);
        #pragma unroll
                            for (int m = 0; m < PPL; ++m) {
                                float2 eta = fmul2(w0, W[m][0]);
                                eta = ffma2(w1, W[m][1], eta);
                                eta = ffma2(w2, W[m][2], eta);
                                eta = ffma2(w3, W[m][3], eta);
                                if (FLOOR) {
                                    eta.x = fmaxf(eta.x, kEtaFloor);
                                    eta.y = fmaxf(eta.y, kEtaFloor);
                                }
                                float2 lg;
                                if (ACC) {
                                    const float2 u = ffma2(eta, ic[m], make_float2(-1.0f, -1.0f));
                                    umax = fmaxf(umax, fmaxf(fabsf(u.x), fabsf(u.y)));
                                    lg = log2_1p_taylor(u);
                                } else {
                                    const float2 r = fmul2(eta, ic[m]);
                                    lg = make_float2(log2_ratio<FLOOR>(r.x), log2_ratio<FLOOR>(r.y));
                                }
                                acc = ffma2(sp[m], lg, acc);
                                if (on[m]) dh = fadd2(dh, fadd2(eta, nec[m]));
                            }
                            float va = acc.x + acc.y, vd = dh.x + dh.y;
                            if (TEAM > 1) {
                                // lanes l, l+N, l+2N, ... of a warp share grid column j:
                                // lane l < N adds the lanes' own values
                                const float a0 = va, d0 = vd;
        #pragma unroll
                                for (int o = N; o < 32; o += N) {
                                    const float xa = __shfl_down_sync(kFull, a0, o), xd = __shfl_down_sync(kFull, d0, o);
                                    if (lane + o < 32) {
                                        va += xa;
                                        vd += xd;
                                    }
                                }
                            }
                            if ((TEAM == 1 || lane < N) &&
                                ANTS_IN_RANGE(L.dbg, (N + k) * ps + (TEAM > 1 ? wit * N + j : t), 2 * N * ps, 104)) {
                                const int slot = TEAM > 1 ? wit * N + j : t;
                                float *pa = s_part + k * ps + slot, *pd = s_part + (N + k) * ps + slot;
                                if (g > 0) {
                                    va += *pa;
                                    vd += *pd;
                                }
                                *pa = va;
                                *pd = vd;
                            }
                        }
                    };
                    if (top == s_iy[k_last]) rows(std::true_type{});
                    else rows(std::false_type{});
                }
            };
            if (sxy * (float)C <= a.prec_halfwidth) {
                sweep(std::true_type{});
                // rare: a lane met an |u| beyond the Taylor range; this warp's
                // partial sums are rewritten from the start with the hardware log2
                if (__any_sync(kFull, umax > kNearOne)) sweep(std::false_type{});
            } else {
                sweep(std::false_type{});
            }
            team_sync<TEAM>(team);

            // ---- phase 3: node scores and team argmax --------------------------
            float bestF = -INFINITY;
            int bestk = 0x7fffffff;
            for (int node = t; node < N * N; node += LT) {
                const int k = node / N, jj = node - k * N;
                float sa = 0.0f, sd = 0.0f;
                // the partials of the warps (teams of several warps) or of the
                // sensor slots (one-warp teams) of this node's column
                constexpr int NPART = TEAM > 1 ? TEAM : Q;
#pragma unroll 4
                for (int w = 0; w < NPART; ++w) {
                    sa += s_part[k * lay.part_stride + w * N + jj];
                    sd += s_part[(N + k) * lay.part_stride + w * N + jj];
                }
                const float xn = fmaf((float)(jj - C), sxy, cx);
                const float yn = fmaf((float)(k - C), sxy, cy);
                const bool ok = xn >= L.lo[0] && xn <= L.hi[0] && yn >= L.lo[1] && yn <= L.hi[1];
                const float F = ok ? sa - S * (log1pf(sd * inv_hc) * kInvLn2) : -INFINITY;
                if (F > bestF) {
                    bestF = F;
                    bestk = node;
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
            if (TEAM > 1) {
                if (lane == 0) {
                    s_red[2 * wit] = bestF;
                    s_red[2 * wit + 1] = __int_as_float(bestk);
                }
                team_sync<TEAM>(team);
                bestF = s_red[0];
                bestk = __float_as_int(s_red[1]);
                for (int w = 1; w < TEAM; ++w) {
                    float F2 = s_red[2 * w];
                    int k2 = __float_as_int(s_red[2 * w + 1]);
                    if (F2 > bestF || (F2 == bestF && k2 < bestk)) {
                        bestF = F2;
                        bestk = k2;
                    }
                }
            }
            const int bj = bestk % N, bk = bestk / N;
            cx = fmaf((float)(bj - C), sxy, cx);
            cy = fmaf((float)(bk - C), sxy, cy);
            if (a.trace && t == 0) a.trace[e * a.iters + it] = (int16_t)bestk;
            sxy *= a.shrink;
        }

        // ---- energy and full Poisson log-likelihood at the result -------------
        float H = 0.0f, ll = 0.0f;
        for (int p = t; p < n_pairs; p += LT) {
            float2 v = pair_eta(L, coef2, p, cx, cy);
            v.x = fmaxf(v.x, kEtaFloor);
            v.y = fmaxf(v.y, kEtaFloor);
            H += v.x + (2 * p + 1 < n_s ? v.y : 0.0f);
        }
        H = warp_sum(H);
        if (TEAM > 1) {
            if (lane == 0) s_red[12 + wit] = H;
            team_sync<TEAM>(team);
            H = 0.0f;
            for (int w = 0; w < TEAM; ++w) H += s_red[12 + w];
        }
        const float E = S / H;
        for (int p = t; p < n_pairs; p += LT) {
            float2 v = pair_eta(L, coef2, p, cx, cy);
            float vv[2] = {fmaxf(v.x, kEtaFloor), fmaxf(v.y, kEtaFloor)};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int i = 2 * p + h;
                if (i >= n_s) continue;
                const float mu = E * vv[h];
                const float s = s_sig[i];
                ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + poisson_const(s) : -mu;
            }
        }
        ll = warp_sum(ll);
        if (TEAM > 1) {
            if (lane == 0) s_red[16 + wit] = ll;
            team_sync<TEAM>(team);
            ll = 0.0f;
            for (int w = 0; w < TEAM; ++w) ll += s_red[16 + w];
        }
        if (t == 0) {
            a.xyz[3 * e] = cx;
            a.xyz[3 * e + 1] = cy;
            a.xyz[3 * e + 2] = cz;
            a.E[e] = E;
            a.logL[e] = ll;
            a.status[e] = ANTS_EVT_OK;
        }
        team_sync<TEAM>(team);  // s_sig and s_red are reused by the next event
    }
}

// ---- small grids on a table in global memory: one sensor pair per lane ----
//
// When the whole grid spans less than two knot intervals per axis (the
// refines of the learned and precision forms), every node of a grid reads
// coefficients from one patch of at most kPatch x kPatch per sensor.  A team
// of TEAM warps reconstructs one event and its lane t owns sensor pair t
// (32 TEAM >= pairs).  The lane reads its pair's patch row by row from the
// pair-fastest copy (a warp's lanes read consecutive pairs: one contiguous
// 256-byte run per load), contracts each row along x for every grid column
// with the columns' B-spline weights placed in the patch ("dense" weights,
// zero outside the column's four), and adds the row into every node with the
// node rows' dense y weights.  The centre node gives eta_c; the pair's
// likelihood terms of every node (as in the team kernel above) go to shared
// memory and are summed over the team's lanes at the end of the grid.
constexpr int kPatch = 6;           // coefficient rows and columns a grid may touch
constexpr int kPatchThreads = 512;  // teams of TEAM warps, one block per SM

template <int N>
struct PatchSmem {
    static constexpr int NN = N * N;
    // floats per team of lt lanes: node terms [2 NN][lt + 1] (the odd row stride
    // keeps both the writes and the row sums free of bank conflicts), x weights
    // [N][kPatch], y weights [kPatch][N], half sums [2][2 NN], reduction slots [32]
    __device__ __host__ static int stride(int lt) { return lt + 1; }
    __device__ __host__ static int wx(int lt) { return 2 * NN * stride(lt); }
    __device__ __host__ static int wy(int lt) { return wx(lt) + N * kPatch; }
    __device__ __host__ static int tot(int lt) { return wy(lt) + kPatch * N; }
    __device__ __host__ static int red(int lt) { return tot(lt) + 4 * NN; }
    __device__ __host__ static int total(int lt) { return (red(lt) + 32 + 3) & ~3; }
};

template <int N, int TEAM, bool FLOOR>
__global__ void __launch_bounds__(kPatchThreads, 1) cgs_xy_patch_kernel(XyArgs a, int teams_per_block)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NN = N * N, C = (N - 1) / 2, LT = 32 * TEAM;
    // grid columns in register groups: all of a 5 x 5 grid at once; a 7 x 7 grid as
    // columns C-1..C+1 (holding the centre, needed first), then 0..C-2, then C+2..
    constexpr int NG = N <= 5 ? 1 : 3, JG = N <= 5 ? N : 3;
    using Lay = PatchSmem<N>;
    const LrfDev &L = a.L;
    const int n_s = L.n_s, n_pairs = L.n_pairs, sy = L.stride_y;
    const int team = threadIdx.x / LT;
    if (team >= teams_per_block) return;  // no block-wide barrier follows
    const int t = threadIdx.x - team * LT, lane = threadIdx.x & 31, wit = t >> 5;
    float *ts = reinterpret_cast<float *>(smem_raw) + (size_t)team * Lay::total(LT);
    float *s_part = ts, *s_wx = ts + Lay::wx(LT), *s_wy = ts + Lay::wy(LT);
    float *s_tot = ts + Lay::tot(LT), *s_red = ts + Lay::red(LT);
    const float2 *cpf = L.coef2_pf;
    const float qnan = __int_as_float(0x7fc00000);
    const long team_stride = (long)gridDim.x * teams_per_block;
    const bool mine = t < n_pairs;  // lane t owns pair t
    const int pp = mine ? t : 0;    // lanes past the last pair repeat pair 0 and add nothing

    for (long e = (long)blockIdx.x * teams_per_block + team; e < a.n_e; e += team_stride) {
        // ---- prologue: signals, S, centroid, status --------------------------
        const float *sg = a.sig + (size_t)(a.rows ? (long)a.rows[e] : e / a.row_div) * n_s;
        float S = 0.0f, Sx = 0.0f, Sy = 0.0f, Sw = 0.0f;
        int bad = 0;
        for (int i = t; i < n_s; i += LT) {
            const float v = sg[i];
            bad |= !(v >= 0.0f) || isinf(v);
            const float w = v * L.cog_w[i];
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
        if (TEAM > 1) {
            if (lane == 0) {
                s_red[16 + 4 * wit] = S;
                s_red[16 + 4 * wit + 1] = Sx;
                s_red[16 + 4 * wit + 2] = Sy;
                s_red[16 + 4 * wit + 3] = bad ? -1.0f : Sw;
            }
            team_sync<TEAM>(team);
            S = Sx = Sy = Sw = 0.0f;
            bad = 0;
            for (int w = 0; w < TEAM; ++w) {
                S += s_red[16 + 4 * w];
                Sx += s_red[16 + 4 * w + 1];
                Sy += s_red[16 + 4 * w + 2];
                const float v = s_red[16 + 4 * w + 3];
                bad |= v < 0.0f;
                Sw += v;
            }
        }
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
            if (t == 0) {
                a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = qnan;
                a.E[e] = qnan;
                a.logL[e] = qnan;
                a.status[e] = st;
            }
            if (a.trace)
                for (int it = t; it < a.iters; it += LT) a.trace[e * a.iters + it] = -1;
            team_sync<TEAM>(team);
            continue;
        }
        const float2 sp = mine ? make_float2(sg[2 * t], 2 * t + 1 < n_s ? sg[2 * t + 1] : 0.0f)
                               : make_float2(0.0f, 0.0f);

        float sxy = a.step_xy;
        for (int it = 0; it < a.iters; ++it) {
            // ---- the grid's patch and dense weights (every thread knows the
            //      patch origin; threads 0..N-1 write column weights, N..2N-1
            //      row weights)
            float t0;
            const int ix0 = bs_span(fmaf((float)(-C), sxy, cx), L.lo[0], L.inv_h[0], L.n_int[0], t0);
            const int iy0 = bs_span(fmaf((float)(-C), sxy, cy), L.lo[1], L.inv_h[1], L.n_int[1], t0);
            const int ixN = bs_span(fmaf((float)C, sxy, cx), L.lo[0], L.inv_h[0], L.n_int[0], t0);
            const int iyN = bs_span(fmaf((float)C, sxy, cy), L.lo[1], L.inv_h[1], L.n_int[1], t0);
            const int pw = ixN - ix0 + 4, ph = iyN - iy0 + 4;  // <= kPatch (checked on the host)
            if (t < 2 * N) {
                const bool col = t < N;
                const int jj = col ? t : t - N;
                float tt, w[4];
                const int spn = col ? bs_span(fmaf((float)(jj - C), sxy, cx), L.lo[0], L.inv_h[0], L.n_int[0], tt)
                                    : bs_span(fmaf((float)(jj - C), sxy, cy), L.lo[1], L.inv_h[1], L.n_int[1], tt);
                bs_weights(tt, w);
                const int off = spn - (col ? ix0 : iy0);
#pragma unroll
                for (int c = 0; c < kPatch; ++c) {
                    const int b = c - off;
                    const float v = b == 0 ? w[0] : b == 1 ? w[1] : b == 2 ? w[2] : b == 3 ? w[3] : 0.0f;
                    if (col) s_wx[jj * kPatch + c] = v;
                    else s_wy[c * N + jj] = v;
                }
            }
            team_sync<TEAM>(team);

            // ---- this lane's pair at every node, by groups of JG columns (the
            //      node accumulators of a group stay in registers) ------------
            const float2 *base = cpf + ((size_t)iy0 * sy + ix0) * n_pairs + pp;
            const int row_step = sy * n_pairs;  // float2 entries per table row (< 2^31)
            const bool acc_log = sxy * (float)C <= a.prec_halfwidth;
            constexpr int RS = LT + 1;
            bool far = false;  // some |u| beyond the Taylor range (accurate grids)
            float hc = 0.0f;
            float2 ic = make_float2(0.0f, 0.0f), nec = ic;
#pragma unroll 1
            for (int g = 0; g < NG; ++g) {
                constexpr int JGc = JG;
                const int j0 = N <= 5 ? 0 : g == 0 ? C - 1 : g == 1 ? 0 : C + 2;
                const int nj = N <= 5 ? N : g == 0 ? 3 : g == 1 ? C - 1 : N - C - 2;
                const int jc = C - j0;  // the centre column within group 0
                float wx[JGc][kPatch];
#pragma unroll
                for (int jj = 0; jj < JGc; ++jj)
#pragma unroll
                    for (int c = 0; c < kPatch; ++c) wx[jj][c] = jj < nj ? s_wx[(j0 + jj) * kPatch + c] : 0.0f;
                float2 eta[N * JGc];
#pragma unroll
                for (int q = 0; q < N * JGc; ++q) eta[q] = make_float2(0.0f, 0.0f);
                // the patch rows, compiled for each patch width (4, 5 or 6 columns;
                // uniform per grid): only the columns the grid touches are read
                // and contracted
                auto rows = [&](auto width) {
                    constexpr int PW = decltype(width)::value;
#pragma unroll
                    for (int r = 0; r < kPatch; ++r) {
                        if (r < ph) {
                            float2 seg[PW];
#pragma unroll
                            for (int c = 0; c < PW; ++c)
                                seg[c] = ANTS_IN_RANGE(L.dbg, ((long)(iy0 + r) * sy + ix0 + c) * n_pairs + pp,
                                                       (long)(L.n_int[1] + 3) * sy * n_pairs, 201)
                                             ? __ldg(base + (r * row_step + c * n_pairs))
                                             : make_float2(0.0f, 0.0f);
#pragma unroll
                            for (int jj = 0; jj < JGc; ++jj) {
                                if (jj < nj) {
                                    float2 T = make_float2(0.0f, 0.0f);
#pragma unroll
                                    for (int c = 0; c < PW; ++c)
                                        T = ffma2(make_float2(wx[jj][c], wx[jj][c]), seg[c], T);
#pragma unroll
                                    for (int k = 0; k < N; ++k) {
                                        const float w = s_wy[r * N + k];
                                        eta[k * JGc + jj] = ffma2(make_float2(w, w), T, eta[k * JGc + jj]);
                                    }
                                }
                            }
                        }
                    }
                };
                if (pw <= 4) rows(std::integral_constant<int, 4>{});
                else if (pw == 5) rows(std::integral_constant<int, 5>{});
                else rows(std::integral_constant<int, kPatch>{});
                if (g == 0) {  // the centre node (C, C) lies in the first group
                    float2 ec = eta[C * JGc + jc];
                    if (FLOOR) {
                        ec.x = fmaxf(ec.x, kEtaFloor);
                        ec.y = fmaxf(ec.y, kEtaFloor);
                    }
                    hc = mine ? ec.x + (2 * t + 1 < n_s ? ec.y : 0.0f) : 0.0f;
                    ic = make_float2(__frcp_rn(ec.x), __frcp_rn(ec.y));
                    nec = make_float2(-ec.x, -ec.y);
                }
                // the group's node terms, compiled once per log form (uniform per grid)
                auto terms = [&](auto accurate) {
                    constexpr bool ACC = decltype(accurate)::value;
#pragma unroll
                    for (int k = 0; k < N; ++k)
#pragma unroll
                        for (int jj = 0; jj < JGc; ++jj) {
                            if (jj >= nj) continue;
                            const int q = k * N + j0 + jj;
                            float2 v = eta[k * JGc + jj];
                            if (FLOOR) {
                                v.x = fmaxf(v.x, kEtaFloor);
                                v.y = fmaxf(v.y, kEtaFloor);
                            }
                            float2 lg;
                            if (ACC) {
                                const float2 u = ffma2(v, ic, make_float2(-1.0f, -1.0f));
                                far = far || fabsf(u.x) > kNearOne || fabsf(u.y) > kNearOne;
                                lg = log2_1p_taylor(u);
                            } else {
                                const float2 r2 = fmul2(v, ic);
                                lg = make_float2(log2_ratio<FLOOR>(r2.x), log2_ratio<FLOOR>(r2.y));
                            }
                            const float2 tt = fmul2(sp, lg);
                            const float2 d = fadd2(v, nec);
                            if (ANTS_IN_RANGE(L.dbg, (NN + q) * RS + t, Lay::wx(LT), 203)) {
                                s_part[q * RS + t] = tt.x + tt.y;
                                s_part[(NN + q) * RS + t] = mine ? d.x + d.y : 0.0f;
                            }
                        }
                };
                if (acc_log) terms(std::true_type{});
                else terms(std::false_type{});
            }
            if (acc_log && __any_sync(kFull, far)) {
                // rare: some |u| beyond the Taylor range; recompute this lane's
                // pair at every node (per node, 16 coefficients) and redo those
                // nodes' log terms with the hardware log2
#pragma unroll 1
                for (int q = 0; q < NN; ++q) {
                    const int k = q / N, jj = q - k * N;
                    const float xn = fminf(fmaxf(fmaf((float)(jj - C), sxy, cx), L.lo[0]), L.hi[0]);
                    const float yn = fminf(fmaxf(fmaf((float)(k - C), sxy, cy), L.lo[1]), L.hi[1]);
                    float2 v = pair_eta(L, L.coef2, pp, xn, yn);
                    if (FLOOR) {
                        v.x = fmaxf(v.x, kEtaFloor);
                        v.y = fmaxf(v.y, kEtaFloor);
                    }
                    const float2 u = ffma2(v, ic, make_float2(-1.0f, -1.0f));
                    if (fabsf(u.x) > kNearOne || fabsf(u.y) > kNearOne) {
                        float2 lg = log2_1p_taylor(u);
                        if (fabsf(u.x) > kNearOne) lg.x = __log2f(1.0f + u.x);
                        if (fabsf(u.y) > kNearOne) lg.y = __log2f(1.0f + u.y);
                        const float2 tt = fmul2(sp, lg);
                        s_part[q * RS + t] = tt.x + tt.y;
                    }
                }
            }
            hc = warp_sum(hc);
            if (TEAM > 1) {
                if (lane == 0) s_red[8 + wit] = hc;
            }
            team_sync<TEAM>(team);
            if (TEAM > 1) {
                hc = 0.0f;
                for (int w = 0; w < TEAM; ++w) hc += s_red[8 + w];
            }
            const float inv_hc = __frcp_rn(hc);

            // ---- node sums over the team's lanes: item k = sigma + 2 NN h adds
            //      half h of row sigma (consecutive threads take consecutive rows:
            //      distinct banks with the odd row stride)
            for (int k = t; k < 4 * NN; k += LT) {
                const int h = k >= 2 * NN, sigma = k - 2 * NN * h;
                const float *src = s_part + sigma * RS + h * (LT / 2);
                float v = 0.0f;
                if (ANTS_IN_RANGE(L.dbg, sigma * RS + h * (LT / 2) + LT / 2 - 1, Lay::wx(LT), 204)) {
#pragma unroll 16
                    for (int i = 0; i < LT / 2; ++i) v += src[i];
                }
                s_tot[k] = v;
            }
            team_sync<TEAM>(team);

            // ---- node scores and argmax (ties to the lowest index) ------------
            float bestF = -INFINITY;
            int bestk = 0x7fffffff;
            if (wit == 0) {
                for (int node = lane; node < NN; node += 32) {
                    const int k = node / N, jj = node - k * N;
                    const float xn = fmaf((float)(jj - C), sxy, cx);
                    const float yn = fmaf((float)(k - C), sxy, cy);
                    const bool ok = xn >= L.lo[0] && xn <= L.hi[0] && yn >= L.lo[1] && yn <= L.hi[1];
                    const float sa = s_tot[node] + s_tot[2 * NN + node];
                    const float sd = s_tot[NN + node] + s_tot[3 * NN + node];
                    const float F = ok ? sa - S * (log1pf(sd * inv_hc) * kInvLn2) : -INFINITY;
                    if (F > bestF) {
                        bestF = F;
                        bestk = node;
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
                if (lane == 0) s_red[0] = __int_as_float(bestk);
            }
            team_sync<TEAM>(team);
            bestk = __float_as_int(s_red[0]);
            const int bj = bestk % N, bk = bestk / N;
            cx = fmaf((float)(bj - C), sxy, cx);
            cy = fmaf((float)(bk - C), sxy, cy);
            if (a.trace && t == 0) a.trace[e * a.iters + it] = (int16_t)bestk;
            sxy *= a.shrink;
        }

        // ---- energy and full Poisson log-likelihood at the result -------------
        float H = 0.0f, ll = 0.0f;
        float2 v = make_float2(kEtaFloor, kEtaFloor);
        if (mine) {
            v = pair_eta_pf(L, t, cx, cy);
            v.x = fmaxf(v.x, kEtaFloor);
            v.y = fmaxf(v.y, kEtaFloor);
            H = v.x + (2 * t + 1 < n_s ? v.y : 0.0f);
        }
        H = warp_sum(H);
        if (TEAM > 1) {
            if (lane == 0) s_red[12 + wit] = H;
            team_sync<TEAM>(team);
            H = 0.0f;
            for (int w = 0; w < TEAM; ++w) H += s_red[12 + w];
        }
        const float E = S / H;
        if (mine) {
            const float vv[2] = {v.x, v.y};
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int i = 2 * t + hh;
                if (i >= n_s) continue;
                const float mu = E * vv[hh];
                const float s = sg[i];
                ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + poisson_const(s) : -mu;
            }
        }
        ll = warp_sum(ll);
        if (TEAM > 1) {
            if (lane == 0) s_red[16 + wit] = ll;
            team_sync<TEAM>(team);
            ll = 0.0f;
            for (int w = 0; w < TEAM; ++w) ll += s_red[16 + w];
        }
        if (t == 0) {
            a.xyz[3 * e] = cx;
            a.xyz[3 * e + 1] = cy;
            a.xyz[3 * e + 2] = cz;
            a.E[e] = E;
            a.logL[e] = ll;
            a.status[e] = ANTS_EVT_OK;
        }
        team_sync<TEAM>(team);  // s_red and the weights are reused by the next event
    }
}

// the patch kernel serves 5 x 5 and 7 x 7 grids on an XY LRF whose table stays
// in global memory, with at most 128 sensor pairs, when every grid of the
// search touches at most kPatch coefficients per axis
bool patch_fits(const ants_lrf *lrf, const ants_cgs_params &p)
{
    if (!lrf->dev.coef2_pf || (p.n_xy != 5 && p.n_xy != 7) || lrf->dev.n_pairs > 128 ||
        !(p.shrink > 0.0f && p.shrink <= 1.0f))
        return false;
    // a range of R covers at most floor(R/h) + 2 spans: patch <= floor(R/h) + 5
    const double R = (double)(p.n_xy - 1) * p.step_xy;
    const double hx = 1.0 / lrf->dev.inv_h[0], hy = 1.0 / lrf->dev.inv_h[1];
    return std::floor(R / hx + 1e-3) + 5 <= kPatch && std::floor(R / hy + 1e-3) + 5 <= kPatch;
}

template <int N, int TEAM, bool FLOOR>
int launch_patch(const ants_ctx *ctx, const XyArgs &a, cudaStream_t stream)
{
    constexpr int LT = 32 * TEAM;
    const int teams = kPatchThreads / LT;
    const size_t smem = (size_t)teams * PatchSmem<N>::total(LT) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(cgs_xy_patch_kernel<N, TEAM, FLOOR>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_xy_patch)");
    long blocks = (a.n_e + teams - 1) / teams;
    const long cap = (long)ctx->n_sm;
    if (blocks > cap) blocks = cap;
    cgs_xy_patch_kernel<N, TEAM, FLOOR><<<(unsigned)blocks, kPatchThreads, smem, stream>>>(a, teams);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cgs_xy_patch_kernel launch");
    count_launch();
    return ANTS_OK;
}

template <int N, bool FLOOR>
int launch_patch_n(const ants_ctx *ctx, const XyArgs &a, cudaStream_t stream)
{
    const int np = a.L.n_pairs;
    if (np <= 32) return launch_patch<N, 1, FLOOR>(ctx, a, stream);
    if (np <= 64) return launch_patch<N, 2, FLOOR>(ctx, a, stream);
    return launch_patch<N, 4, FLOOR>(ctx, a, stream);
}

template <int N, int TEAM, int PPL>
int launch_nt(const ants_ctx *ctx, const XyArgs &a, bool floor_needed, cudaStream_t stream)
{
    constexpr int LT = 32 * TEAM;
    const TeamSmem lay = TeamSmem::make(2 * a.L.n_pairs, LT, N);
    const int team_floats = lay.total(N);
    const size_t table = (((size_t)a.L.n_pairs * a.L.pair_stride + 1) & ~(size_t)1) * sizeof(float2);
    const size_t per_team = (size_t)team_floats * sizeof(float);
    const int max_teams = kXyThreads / LT;
    // keep the coefficient table in shared memory with as many teams as fit;
    // otherwise read it through L1/L2 with every team
    int teams = max_teams;
    while (teams > 0 && table + teams * per_team > ctx->smem_optin) --teams;
    const bool smem_table = teams > 0;
    if (!smem_table) teams = max_teams;
    const size_t smem = teams * per_team + (smem_table ? table : 0);
    if (smem > ctx->smem_optin) return fail(ANTS_E_UNIMPLEMENTED, "cgs_xy: %zu bytes of shared memory", smem);
    long blocks = (a.n_e + teams - 1) / teams;
    const long cap = (long)ctx->n_sm;
    if (blocks > cap) blocks = cap;
    cudaError_t e = cudaSuccess;
#define ANTS_XY_LAUNCH(SM, FL)                                                                                 \
    do {                                                                                                       \
        e = cudaFuncSetAttribute(cgs_xy_kernel<N, TEAM, PPL, SM, FL>, cudaFuncAttributeMaxDynamicSharedMemorySize,  \
                                 (int)smem);                                                                   \
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(cgs_xy)");                              \
        cgs_xy_kernel<N, TEAM, PPL, SM, FL><<<(unsigned)blocks, kXyThreads, smem, stream>>>(a, teams, team_floats); \
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

int launch_cgs_xy(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig, int row_div,
                  const int *rows,
                  long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status, int16_t *trace,
                  cudaStream_t stream)
{
    XyArgs a;
    a.row_div = row_div;
    a.rows = rows;
    a.L = lrf->dev;
    a.iters = p.iters;
    a.shrink = p.shrink;
    a.step_xy = p.step_xy;
    // a quarter of a knot interval (the smaller axis): on such grids the LRF
    // changes by a few per cent at most between a node and the centre, and the
    // last two grids of a halving search are the ones whose nodes' scores are
    // close enough for the logarithm's error to decide the argmax
    a.prec_halfwidth = 0.25f * fminf(1.0f / lrf->dev.inv_h[0], 1.0f / lrf->dev.inv_h[1]);
    a.sig = sig;
    a.n_e = n_e;
    a.start = start;
    a.xyz = xyz;
    a.E = E;
    a.logL = logL;
    a.status = status;
    a.trace = trace;
    // the floor is needed when an LRF value can be <= 0 or the coefficients
    // span more than 2^100, or to neutralise the zero-coefficient padding
    // sensor of an odd sensor count
    bool floor_needed = !lrf->dev.positive || (lrf->n_s & 1);
    // tables too large for shared memory: small grids take the patch kernel
    const size_t table_bytes = (size_t)lrf->dev.n_pairs * lrf->dev.pair_stride * sizeof(float2);
    if (table_bytes + 4096 > ctx->smem_optin && patch_fits(lrf, p))
        return p.n_xy == 5 ? (floor_needed ? launch_patch_n<5, true>(ctx, a, stream)
                                           : launch_patch_n<5, false>(ctx, a, stream))
                           : (floor_needed ? launch_patch_n<7, true>(ctx, a, stream)
                                           : launch_patch_n<7, false>(ctx, a, stream));
    switch (p.n_xy) {
    case 5: return launch_nt<5, 1, 3>(ctx, a, floor_needed, stream);
    case 7: return launch_nt<7, 1, 3>(ctx, a, floor_needed, stream);
    case 9: return launch_nt<9, 4, 3>(ctx, a, floor_needed, stream);
    case 11: return launch_nt<11, 3, 4>(ctx, a, floor_needed, stream);
    case 13: return launch_nt<13, 4, 3>(ctx, a, floor_needed, stream);
    default: return launch_nt<15, 4, 3>(ctx, a, floor_needed, stream);
    }
}

}  // namespace ants
