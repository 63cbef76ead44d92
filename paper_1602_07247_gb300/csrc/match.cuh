// The per-event set-up shared by the search variants and the continuous
// minimisation: signals, status, start position and the sensors in the
// match (Sec. 5.1.2: sensors below a signal threshold or farther than a
// given distance from the start can be left out; Sec. 5.1.2.1 / 5.1.2.2: the
// start is the centroid or the strongest sensor; Sec. 5.3: passive sensors
// are ignored).  One warp per event.
#pragma once

#include <type_traits>

#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

constexpr int kMaxMatchSensors = 1024;

struct MatchArgs {
    int start;                                  // ANTS_START_COG / ANTS_START_MAX_SENSOR
    float min_signal, max_distance, z0;
    double gain[kMaxMatchSensors];              // relative gains (start)
    float inv_gain[kMaxMatchSensors];           // their reciprocals (single-precision start)
    unsigned char passive[kMaxMatchSensors];    // 1 = passive
};

__device__ __forceinline__ float match_warp_sum(float v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double match_warp_sum_d(double v)
{
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Collectives of a group of G lanes (G = 8, 16 or 32; groups are aligned
// blocks of the warp).  Every lane of the warp calls them together (the
// callers keep the groups in lockstep), so the full mask is used; butterfly
// offsets below G stay inside the group, and every lane of a group ends with
// the same sum.
template <int G> struct Group {
    static __device__ __forceinline__ unsigned mask(int lane)
    {
        return G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    }
    static __device__ __forceinline__ float sum(float v)
    {
        for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    static __device__ __forceinline__ double sumd(double v)
    {
        for (int o = G / 2; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    }
    static __device__ __forceinline__ double sum_any(double v) { return sumd(v); }
    static __device__ __forceinline__ float sum_any(float v) { return sum(v); }
    static __device__ __forceinline__ bool any(bool p, int lane)
    {
        return (__ballot_sync(0xffffffffu, p) & mask(lane)) != 0u;
    }
    static __device__ __forceinline__ bool all(bool p, int lane)
    {
        const unsigned m = mask(lane);
        return (__ballot_sync(0xffffffffu, p) & m) == m;
    }
};

// The set-up of event e by a group of G lanes (glane = lane within the
// group): loads the signals into s_sig (0 for passive sensors), picks the
// start (given: start_xyz, nullable), marks the sensors in the match in
// s_act (1 / 0) and returns ANTS_EVT_OK with their signal sum S and the
// start, or the event's failure status.  EXACT: the sums and comparisons
// that pick the start or a sensor are made in FP64 (s / g as the oracle
// forms it, for searches whose path depends on the start's last bit); else
// in FP32 with s times 1 / g (a minimisation converges to the same optimum).
// Every lane of the warp runs every collective; an inactive group (no
// event) reads nothing and returns ANTS_EVT_ZERO_SIGNAL.
template <int TYPE, int G, bool EXACT = true>
__device__ __forceinline__ int match_prologue_g(const LrfDev &L, const MatchArgs &m, const float *sig, long e,
                                                bool active, const float *start_xyz, float *s_sig, float *s_act,
                                                int lane, float &S, float &cx, float &cy, float &cz)
{
    using A = typename std::conditional<EXACT, double, float>::type;
    const int n_s = L.n_s, glane = lane & (G - 1);
    bool bad = false;
    A tot = 0, W = 0, X = 0, Y = 0, bv = -1;
    int bi = 0x7fffffff;
    for (int i = glane; active && i < n_s; i += G) {
        float s = sig[e * n_s + i];
        if (m.passive[i]) s = 0.0f;
        else if (!isfinite(s) || s < 0.0f) bad = true;
        s_sig[i] = s;
        const A w = EXACT ? (A)((double)s / m.gain[i]) : (A)(s * m.inv_gain[i]);
        tot += (A)s;
        W += w;
        X += (A)L.sxy[2 * i] * w;
        Y += (A)L.sxy[2 * i + 1] * w;
        if (!m.passive[i] && w > bv) {  // lanes visit increasing i: the first maximum
            bv = w;
            bi = i;
        }
    }
    bad = Group<G>::any(bad, lane);
    tot = Group<G>::sum_any(tot);
    int st = !active ? ANTS_EVT_ZERO_SIGNAL : bad ? ANTS_EVT_BAD_SIGNAL : !(tot > A(0)) ? ANTS_EVT_ZERO_SIGNAL
                                                                                       : ANTS_EVT_OK;
    cz = lrf_is_3d(TYPE) ? m.z0 : 0.0f;
    for (int o = G / 2; o; o >>= 1) {  // the largest s/g, ties to the lowest index
        const A v2 = __shfl_xor_sync(0xffffffffu, bv, o);
        const int i2 = __shfl_xor_sync(0xffffffffu, bi, o);
        if (v2 > bv || (v2 == bv && i2 < bi)) {
            bv = v2;
            bi = i2;
        }
    }
    W = Group<G>::sum_any(W);
    X = Group<G>::sum_any(X);
    Y = Group<G>::sum_any(Y);
    if (start_xyz && active) {
        cx = start_xyz[3 * e];
        cy = start_xyz[3 * e + 1];
        cz = start_xyz[3 * e + 2];
    } else if (m.start == 1) {
        cx = bi < n_s ? L.sxy[2 * bi] : 0.0f;
        cy = bi < n_s ? L.sxy[2 * bi + 1] : 0.0f;
    } else {
        cx = (float)(X / W);
        cy = (float)(Y / W);
    }
    if (lrf_has_box(TYPE) && !start_xyz) {
        cx = fminf(fmaxf(cx, L.lo[0]), L.hi[0]);
        cy = fminf(fmaxf(cy, L.lo[1]), L.hi[1]);
    }
    float Sp = 0.0f;
    for (int i = glane; st == ANTS_EVT_OK && i < n_s; i += G) {
        bool in = !m.passive[i];
        if (m.min_signal > 0.0f && s_sig[i] < m.min_signal) in = false;
        if (m.max_distance > 0.0f) {
            const double dx = (double)L.sxy[2 * i] - (double)cx, dy = (double)L.sxy[2 * i + 1] - (double)cy;
            if (sqrt(dx * dx + dy * dy) > (double)m.max_distance) in = false;
        }
        s_act[i] = in ? 1.0f : 0.0f;
        if (in) Sp += s_sig[i];
    }
    S = Group<G>::sum(Sp);
    __syncwarp();
    if (st != ANTS_EVT_OK) return st;
    if (!(S > 0.0f)) return ANTS_EVT_ZERO_SIGNAL;
    if (!lrf_defined(L, s_act, cx, cy, cz)) return ANTS_EVT_OUT_OF_DOMAIN;
    return ANTS_EVT_OK;
}

// the same for one event per warp (G = 32)
template <int TYPE>
__device__ __forceinline__ int match_prologue(const LrfDev &L, const MatchArgs &m, const float *sig, long e,
                                              const float *start_xyz, float *s_sig, float *s_act, int lane, float &S,
                                              float &cx, float &cy, float &cz)
{
    return match_prologue_g<TYPE, 32>(L, m, sig, e, true, start_xyz, s_sig, s_act, lane, S, cx, cy, cz);
}

}  // namespace ants
