// Continuous minimisation of the match (Sec. 5.1.2.1: the match, maximum
// likelihood or least squares, is minimised over the two or three source
// coordinates by a gradient method, from the centroid or the strongest
// sensor; the paper uses Minuit2's Migrad).  Here: damped Fisher scoring
// (Levenberg-Marquardt) with the energy profiled out, E = S / H.
//
// One warp per event.  Each trial evaluates every sensor in the match at the
// trial point in two passes over the lanes' sensors (eta and its gradient,
// kept in shared memory; then, with H and grad H reduced, the Fisher
// information J and the scoring direction g); the butterfly reductions
// leave identical sums in every lane, so every lane solves the same 2 x 2 or
// 3 x 3 system and takes the same decisions.  The change of the match
// between the current point p and the trial q is formed relative to p: for
// maximum likelihood sum s log2(eta_q / eta_p) - S log1p(sum (eta_q - eta_p)
// / H_p), which keeps single precision near the optimum; inside a rounding
// band tau = 2^-18 S the decision falls to the trapezoid rule on the
// gradients, (g_p + g_q) . (q - p) >= 0.  Coordinates on a bound of the
// domain's box whose step points out of it are held (a projected step), and
// a step that overshot the optimum along its line raises the damping.
#include <cmath>

#include "bspline.cuh"
#include "internal.cuh"
#include "match.cuh"

namespace ants {

namespace {

constexpr float kEtaFloor = 1e-30f;
constexpr int kMinWarps = 8;
constexpr float kLambdaMin = 1e-12f, kLambdaMax = 1e8f;

struct MinArgs {
    LrfDev L;
    int criterion, max_iter;
    float tol, lambda0;
    const float *sig;
    long n_e;
    const float *start_xyz;  // nullable [n_e][3]
    float *xyz, *E, *logL;
    int32_t *status;
    int16_t *n_iter;  // nullable [n_e]
    MatchArgs m;
};

// the sums of one trial point (identical in every lane after the reductions)
struct PointSums {
    float H, dH[3];
    float g[3];
    float J[6];   // J00, J01, J02, J11, J12, J22
    float chi2;   // least squares: Pearson's chi^2
    float lsum;   // maximum likelihood: sum s log2(eta / eta_p)
    float dHrel;  // sum (eta - eta_p)
};

// s ln s - s - lgamma(s + 1) for s > 0 (Stirling series from s = 10)
__device__ __forceinline__ float poisson_const(float s)
{
    if (s >= 10.0f) {
        float r = 1.0f / s, r2 = r * r;
        float series = r * (-1.0f / 12.0f + r2 * (1.0f / 360.0f - r2 * (1.0f / 1260.0f)));
        return -0.5f * logf(6.283185307179586f * s) + series;
    }
    return s * logf(s) - s - lgammaf(s + 1.0f);
}

// every LRF in the match defined at (x, y, z), checked across the group
// (every lane of the warp calls it; a lane with live = false checks nothing)
template <int TYPE, int G>
__device__ __forceinline__ bool defined_group(const LrfDev &L, const float *s_act, float x, float y, float z, int lane,
                                              bool live)
{
    bool ok = true;
    if (TYPE == ANTS_LRF_RADIAL || TYPE == ANTS_LRF_COMPOSITE || TYPE == ANTS_LRF_AXIAL_Z) {
        const float rhi = TYPE == ANTS_LRF_COMPOSITE ? L.hi_r : L.hi[0];
        for (int i = lane & (G - 1); live && i < L.n_s; i += G)
            if (s_act[i] != 0.0f && plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]) > rhi) ok = false;
    }
    if (TYPE == kLrfXYSym) {
        // symmetry classes: every sensor's mapped point inside the box
        for (int i = lane & (G - 1); live && i < L.n_s; i += G) {
            if (s_act[i] == 0.0f) continue;
            float m[4];
            sym_op(__ldg(L.op_of + i), m);
            const float dx = x - L.sym_c[0], dy = y - L.sym_c[1];
            const float u = fmaf(m[0], dx, fmaf(m[2], dy, L.sym_c[0]));
            const float v = fmaf(m[1], dx, fmaf(m[3], dy, L.sym_c[1]));
            if (!in_box(L, u, v, z)) ok = false;
        }
        return Group<G>::all(ok, lane);
    }
    ok = Group<G>::all(ok, lane);
    if (TYPE == ANTS_LRF_AXIAL_Z) return ok && z >= L.lo[1] && z <= L.hi[1];
    if (TYPE == ANTS_LRF_RADIAL) return ok;
    return ok && in_box(L, x, y, z);
}

// the box bounds of coordinate k: x and y in the XY box (XY, XYZ,
// composite, sliced), z in the z range (XYZ, sliced, axial+z); false when
// the coordinate has none
template <int TYPE>
__device__ __forceinline__ bool box_bounds(const LrfDev &L, int k, float &lo, float &hi)
{
    if (k < 2) {
        if (!lrf_has_box(TYPE)) return false;
        lo = L.lo[k];
        hi = L.hi[k];
        return true;
    }
    if (!lrf_is_3d(TYPE)) return false;
    const int kz = TYPE == ANTS_LRF_AXIAL_Z ? 1 : 2;
    lo = L.lo[kz];
    hi = L.hi[kz];
    return true;
}

// a trial point moved onto the domain's box
template <int TYPE>
__device__ __forceinline__ void clamp_box(const LrfDev &L, float q[3])
{
    for (int k = 0; k < 3; ++k) {
        float lo, hi;
        if (box_bounds<TYPE>(L, k, lo, hi)) q[k] = fminf(fmaxf(q[k], lo), hi);
    }
}

// the coordinates (bit k) on a bound of the box while the step points out
// of it: held in the next solve (a projected step)
template <int TYPE, int D>
__device__ __forceinline__ int active_set(const LrfDev &L, const float p[3], const float delta[3])
{
    int fixed = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float lo, hi;
        if (!box_bounds<TYPE>(L, k, lo, hi)) continue;
        if ((p[k] == lo && delta[k] < 0.0f) || (p[k] == hi && delta[k] > 0.0f)) fixed |= 1 << k;
    }
    return fixed;
}

// The two passes at point q over the sensors in the match: eta (floored,
// gradient 0 where floored) into s_eq and its gradient into s_g, then J, g
// and chi^2; rel: the sums relative to eta_p in s_ep as well.
template <int TYPE, int D, int G>
__device__ __forceinline__ PointSums point_pass(const MinArgs &a, const float *s_sig, const float *s_act,
                                                const float *s_ep, float *s_eq, float *s_g, const float q[3], float S,
                                                bool rel, int lane, bool live)
{
    const LrfDev &L = a.L;
    const int n_s = L.n_s, glane = lane & (G - 1);
    PointSums P;
    float H = 0.0f, d0 = 0.0f, d1 = 0.0f, d2 = 0.0f, ls = 0.0f, dh = 0.0f;
    // XY sets share the knot grid: the span and the weights of the point are
    // computed once, not per sensor (the same arithmetic as lrf_eta_grad_t)
    int jx = 0, jy = 0;
    float wx[4], wy[4], dwx[4], dwy[4];
    if (TYPE == ANTS_LRF_XY) {
        float tx, ty;
        jx = bs_span(q[0], L.lo[0], L.inv_h[0], L.n_int[0], tx);
        jy = bs_span(q[1], L.lo[1], L.inv_h[1], L.n_int[1], ty);
        bs_weights(tx, wx);
        bs_weights(ty, wy);
        bs_dweights(tx, dwx);
        bs_dweights(ty, dwy);
    }
    for (int i = glane; live && i < n_s; i += G) {
        if (s_act[i] == 0.0f) continue;
        bool ok;
        float gx, gy, gz = 0.0f, eta;
        if (TYPE == ANTS_LRF_XY) {
            // sensor-minor copy: the group's lanes read neighbouring sensors
            const float *c = L.coef_t + (size_t)(jy * L.stride_y + jx) * n_s + i;
            const size_t rs = (size_t)L.stride_y * n_s;
            float f = 0.0f, fx = 0.0f, fy = 0.0f;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float *row = c + b * rs;
                float fr = 0.0f, frx = 0.0f;
#pragma unroll
                for (int a2 = 0; a2 < 4; ++a2) {
                    const float cv = __ldg(row + (size_t)a2 * n_s);
                    fr = fmaf(cv, wx[a2], fr);
                    frx = fmaf(cv, dwx[a2], frx);
                }
                f = fmaf(fr, wy[b], f);
                fx = fmaf(frx, wy[b], fx);
                fy = fmaf(fr, dwy[b], fy);
            }
            eta = f;
            gx = fx * L.inv_h[0];
            gy = fy * L.inv_h[1];
        } else {
            eta = lrf_eta_grad_t<TYPE>(L, i, q[0], q[1], q[2], ok, gx, gy, gz);
        }
        if (!(eta > kEtaFloor)) {
            eta = kEtaFloor;
            gx = gy = gz = 0.0f;
        }
        s_eq[i] = eta;
        s_g[3 * i] = gx;
        s_g[3 * i + 1] = gy;
        s_g[3 * i + 2] = gz;
        H += eta;
        d0 += gx;
        d1 += gy;
        if (D == 3) d2 += gz;
        if (rel) {
            const float ep = s_ep[i];
            if (s_sig[i] != 0.0f) ls = fmaf(s_sig[i], log2f(eta / ep), ls);
            dh += eta - ep;
        }
    }
    P.H = Group<G>::sum(H);
    P.dH[0] = Group<G>::sum(d0);
    P.dH[1] = Group<G>::sum(d1);
    P.dH[2] = D == 3 ? Group<G>::sum(d2) : 0.0f;
    P.lsum = rel ? Group<G>::sum(ls) : 0.0f;
    P.dHrel = rel ? Group<G>::sum(dh) : 0.0f;
    const float E = S / P.H, invH = 1.0f / P.H;
    float g[3] = {0.0f, 0.0f, 0.0f}, J[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, chi = 0.0f;
    for (int i = glane; live && i < n_s; i += G) {
        if (s_act[i] == 0.0f) continue;
        const float eta = s_eq[i], s = s_sig[i], mu = E * eta;
        float gi[3] = {s_g[3 * i], s_g[3 * i + 1], D == 3 ? s_g[3 * i + 2] : 0.0f}, dmu[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < D; ++k) dmu[k] = E * fmaf(-eta * invH, P.dH[k], gi[k]);
        const float imu = 1.0f / mu;
        J[0] = fmaf(dmu[0] * imu, dmu[0], J[0]);
        J[1] = fmaf(dmu[0] * imu, dmu[1], J[1]);
        J[3] = fmaf(dmu[1] * imu, dmu[1], J[3]);
        if (D == 3) {
            J[2] = fmaf(dmu[0] * imu, dmu[2], J[2]);
            J[4] = fmaf(dmu[1] * imu, dmu[2], J[4]);
            J[5] = fmaf(dmu[2] * imu, dmu[2], J[5]);
        }
        const float r = s - mu;
        if (a.criterion == 0) {
            const float w = r / eta;
#pragma unroll
            for (int k = 0; k < D; ++k) g[k] = fmaf(w, gi[k], g[k]);
        } else {
            const float sm = s * imu, w = -0.5f * (1.0f - sm * sm);
#pragma unroll
            for (int k = 0; k < D; ++k) g[k] = fmaf(w, dmu[k], g[k]);
            chi = fmaf(r * r, imu, chi);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) P.g[k] = k < D ? Group<G>::sum(g[k]) : 0.0f;
    P.J[0] = Group<G>::sum(J[0]);
    P.J[1] = Group<G>::sum(J[1]);
    P.J[3] = Group<G>::sum(J[3]);
    P.J[2] = D == 3 ? Group<G>::sum(J[2]) : 0.0f;
    P.J[4] = D == 3 ? Group<G>::sum(J[4]) : 0.0f;
    P.J[5] = D == 3 ? Group<G>::sum(J[5]) : 0.0f;
    P.chi2 = a.criterion == 0 ? 0.0f : Group<G>::sum(chi);
    return P;
}

// (J + lambda D) delta = g, D = diag(J) floored at 1e-12 of its largest
// entry, by Cramer's rule; the coordinates in `fixed` are held (their rows
// and columns those of the identity, right-hand side 0); false when singular
template <int D>
__device__ __forceinline__ bool solve_step(const PointSums &P, float lambda, int fixed, float delta[3])
{
    delta[0] = delta[1] = delta[2] = 0.0f;
    float dmax = fmaxf(P.J[0], P.J[3]);
    if (D == 3) dmax = fmaxf(dmax, P.J[5]);
    if (!(dmax > 0.0f)) return false;
    const float fl = 1e-12f * dmax;
    const bool f0 = fixed & 1, f1 = fixed & 2, f2 = fixed & 4;
    const float g0 = f0 ? 0.0f : P.g[0], g1 = f1 ? 0.0f : P.g[1], g2 = f2 ? 0.0f : P.g[2];
    const float a00 = f0 ? 1.0f : fmaf(lambda, fmaxf(P.J[0], fl), P.J[0]);
    const float a11 = f1 ? 1.0f : fmaf(lambda, fmaxf(P.J[3], fl), P.J[3]);
    const float a01 = f0 || f1 ? 0.0f : P.J[1];
    if (D == 2) {
        const float det = a00 * a11 - a01 * a01;
        if (!(fabsf(det) > 0.0f)) return false;
        delta[0] = (g0 * a11 - a01 * g1) / det;
        delta[1] = (a00 * g1 - g0 * a01) / det;
        return true;
    }
    const float a22 = f2 ? 1.0f : fmaf(lambda, fmaxf(P.J[5], fl), P.J[5]);
    const float a02 = f0 || f2 ? 0.0f : P.J[2], a12 = f1 || f2 ? 0.0f : P.J[4];
    const float c00 = a11 * a22 - a12 * a12, c01 = a02 * a12 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    const float det = a00 * c00 + a01 * c01 + a02 * c02;
    if (!(fabsf(det) > 0.0f)) return false;
    const float c11 = a00 * a22 - a02 * a02, c12 = a01 * a02 - a00 * a12, c22 = a00 * a11 - a01 * a01;
    const float inv = 1.0f / det;
    delta[0] = (c00 * g0 + c01 * g1 + c02 * g2) * inv;
    delta[1] = (c01 * g0 + c11 * g1 + c12 * g2) * inv;
    delta[2] = (c02 * g0 + c12 * g1 + c22 * g2) * inv;
    return true;
}

// G lanes per event, 32 / G events per warp in lockstep: every lane runs
// every collective; groups whose event is finished (or absent) keep running
// the loop without evaluating sensors or changing their state
template <int TYPE, int D, int G>
__global__ void __launch_bounds__(32 * kMinWarps, 2) minimize_kernel(const __grid_constant__ MinArgs a)
{
    extern __shared__ float smem[];
    constexpr int EPW = 32 / G;
    const LrfDev &L = a.L;
    const int n_s = L.n_s;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, grp = lane / G, glane = lane & (G - 1);
    float *s_sig = smem + ((size_t)wib * EPW + grp) * 7 * n_s;  // signals (0 for passive sensors)
    float *s_act = s_sig + n_s;                                  // 1 in the match, 0 out
    float *s_ep = s_act + n_s;                                   // eta at the current point
    float *s_eq = s_ep + n_s;                                    // eta at the trial point
    float *s_g = s_eq + n_s;                                     // its gradient [n_s][3]
    const long warps = (long)gridDim.x * (blockDim.x >> 5);
    for (long base = ((long)blockIdx.x * (blockDim.x >> 5) + wib) * EPW; base < a.n_e; base += warps * EPW) {
        const long e = base + grp;
        const bool active = e < a.n_e;
        float S, p[3];
        const int st = match_prologue_g<TYPE, G, false>(L, a.m, a.sig, e, active, a.start_xyz, s_sig, s_act, lane, S,
                                                        p[0], p[1], p[2]);
        bool done = st != ANTS_EVT_OK;
        if (active && done && glane == 0) {
            const float nan = __int_as_float(0x7fc00000);
            a.xyz[3 * e] = a.xyz[3 * e + 1] = a.xyz[3 * e + 2] = nan;
            a.E[e] = a.logL[e] = nan;
            a.status[e] = st;
            if (a.n_iter) a.n_iter[e] = 0;
        }
        const float tau = ldexpf(S, -18);
        PointSums P = point_pass<TYPE, D, G>(a, s_sig, s_act, s_ep, s_eq, s_g, p, S, false, lane, !done);
        for (int i = glane; !done && i < n_s; i += G) s_ep[i] = s_eq[i];
        float lambda = a.lambda0;
        int used = -a.max_iter;
        for (int it = 1; it <= a.max_iter; ++it) {
            if (__all_sync(0xffffffffu, done)) break;
            float delta[3];
            bool okd = solve_step<D>(P, lambda, 0, delta);
            const int fixed = okd ? active_set<TYPE, D>(L, p, delta) : 0;
            if (fixed) okd = solve_step<D>(P, lambda, fixed, delta);
            float q[3] = {p[0] + delta[0], p[1] + delta[1], p[2] + delta[2]};
            clamp_box<TYPE>(L, q);
            const bool cand = !done && okd && isfinite(q[0]) && isfinite(q[1]) && isfinite(q[2]);
            bool acc = defined_group<TYPE, G>(L, s_act, q[0], q[1], q[2], lane, cand) && cand;
            PointSums Q = point_pass<TYPE, D, G>(a, s_sig, s_act, s_ep, s_eq, s_g, q, S, true, lane, acc);
            if (acc) {
                const float dC = a.criterion == 0 ? 0.6931471805599453f * Q.lsum - S * log1pf(Q.dHrel / P.H)
                                                  : P.chi2 - Q.chi2;
                if (fabsf(dC) > tau) {
                    acc = dC > 0.0f;
                } else {
                    float t = 0.0f;
                    for (int k = 0; k < 3; ++k) t = fmaf(P.g[k] + Q.g[k], q[k] - p[k], t);
                    acc = t >= 0.0f;
                }
            }
            if (done) continue;
            if (acc) {
                const float dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
                const float step = sqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                // slopes along the step at both ends: when their sign changed
                // the step overshot the line's optimum (at t* = a0 / (a0 - a1)
                // for a quadratic), and the next damping shortens by t*
                const float a0 = fmaf(P.g[0], dx, fmaf(P.g[1], dy, P.g[2] * dz));
                const float a1 = fmaf(Q.g[0], dx, fmaf(Q.g[1], dy, Q.g[2] * dz));
                float next = fmaxf(lambda * 0.1f, kLambdaMin);
                if (a0 > 0.0f && a1 < 0.0f) next = fmaxf(next, (a0 - a1) / a0 - 1.0f);
                p[0] = q[0];
                p[1] = q[1];
                p[2] = q[2];
                P = Q;
                for (int i = glane; i < n_s; i += G) s_ep[i] = s_eq[i];
                lambda = next;
                if (step < a.tol) {
                    used = it;
                    done = true;
                }
            } else {
                lambda *= 10.0f;
                if (lambda > kLambdaMax) {
                    used = it;
                    done = true;
                }
            }
        }
        // energy and full Poisson log-likelihood over the match at p
        const bool ok = st == ANTS_EVT_OK;
        const float En = S / P.H;
        float ll = 0.0f;
        for (int i = glane; ok && i < n_s; i += G) {
            if (s_act[i] == 0.0f) continue;
            const float mu = En * s_ep[i], s = s_sig[i];
            ll += s > 0.0f ? fmaf(s, logf(mu / s), s - mu) + poisson_const(s) : -mu;
        }
        ll = Group<G>::sum(ll);
        if (ok && glane == 0) {
            a.xyz[3 * e] = p[0];
            a.xyz[3 * e + 1] = p[1];
            a.xyz[3 * e + 2] = p[2];
            a.E[e] = En;
            a.logL[e] = ll;
            a.status[e] = ANTS_EVT_OK;
            if (a.n_iter) a.n_iter[e] = (int16_t)used;
        }
        __syncwarp();
    }
}

}  // namespace

int check_minimize_params(const ants_lrf *lrf, const ants_minimize_params *P)
{
    if (!P) return fail(ANTS_E_ARG, "minimize parameters are NULL");
    if (P->criterion != ANTS_CRIT_ML && P->criterion != ANTS_CRIT_LS)
        return fail(ANTS_E_ARG, "minimize: unknown criterion %d", P->criterion);
    if (P->start != ANTS_START_COG && P->start != ANTS_START_MAX_SENSOR)
        return fail(ANTS_E_ARG, "minimize: unknown start %d", P->start);
    if (P->max_iter < 1 || P->max_iter > 32767) return fail(ANTS_E_ARG, "minimize: max_iter must be in 1..32767");
    if (!(P->tol > 0.0f) || !(P->lambda0 >= 0.0f)) return fail(ANTS_E_ARG, "minimize: tol must be > 0, lambda0 >= 0");
    if (!(P->min_signal >= 0.0f) || !(P->max_distance >= 0.0f))
        return fail(ANTS_E_ARG, "minimize: min_signal and max_distance must be >= 0");
    if (P->fit_z != 0 && P->fit_z != 1) return fail(ANTS_E_ARG, "minimize: fit_z must be 0 or 1");
    if (lrf->n_s > kMaxMatchSensors)
        return fail(ANTS_E_UNIMPLEMENTED, "minimize: at most %d sensors", kMaxMatchSensors);
    return ANTS_OK;
}

int reconstruct_minimize(const ants_ctx *ctx, const ants_lrf *lrf, const ants_minimize_params &P, const float *sig,
                         long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                         int16_t *n_iter, cudaStream_t s)
{
    MinArgs a;
    a.L = lrf->dev;
    a.criterion = P.criterion;
    a.max_iter = P.max_iter;
    a.tol = P.tol;
    a.lambda0 = P.lambda0;
    a.sig = sig;
    a.n_e = n_e;
    a.start_xyz = start;
    a.xyz = xyz;
    a.E = E;
    a.logL = logL;
    a.status = status;
    a.n_iter = n_iter;
    a.m.start = P.start;
    a.m.min_signal = P.min_signal;
    a.m.max_distance = P.max_distance;
    a.m.z0 = P.z0;
    const int n_s = lrf->n_s;
    for (int i = 0; i < kMaxMatchSensors; ++i) {
        a.m.gain[i] = i < n_s ? lrf->rel_gain[i] : 1.0;
        a.m.inv_gain[i] = (float)(1.0 / a.m.gain[i]);
        a.m.passive[i] = i < n_s && P.passive_host && P.passive_host[i] ? 1 : 0;
    }
    // 8 lanes per event (4 events per warp) up to 96 sensors, else a warp
    // per event; as many warps per block as fit 7 n_s floats per event in 48 KB
    const int G = n_s <= 96 ? 8 : 32, epw = 32 / G;
    int wpb = (int)(48 * 1024 / (28 * (size_t)n_s * epw));
    wpb = wpb < 1 ? 1 : (wpb > kMinWarps ? kMinWarps : wpb);
    const size_t smem = (size_t)wpb * epw * 28 * n_s;
    const long per_block = (long)wpb * epw;
    long blocks = (n_e + per_block - 1) / per_block;
    const long cap = (long)ctx->n_sm * 16;
    if (blocks > cap) blocks = cap;
    const bool z = P.fit_z != 0;
    const unsigned g = (unsigned)blocks, t = 32u * wpb;
#define ANTS_MIN_LAUNCH(T, D)                                                         \
    (G == 8    ? minimize_kernel<T, D, 8><<<g, t, smem, s>>>(a)                                \
     : G == 16 ? minimize_kernel<T, D, 16><<<g, t, smem, s>>>(a)                              \
               : minimize_kernel<T, D, 32><<<g, t, smem, s>>>(a))
    switch (lrf->type) {
    case ANTS_LRF_RADIAL: ANTS_MIN_LAUNCH(ANTS_LRF_RADIAL, 2); break;
    case ANTS_LRF_XY:
        if (lrf->dev.set_of) ANTS_MIN_LAUNCH(kLrfXYSym, 2);
        else ANTS_MIN_LAUNCH(ANTS_LRF_XY, 2);
        break;
    case ANTS_LRF_COMPOSITE: ANTS_MIN_LAUNCH(ANTS_LRF_COMPOSITE, 2); break;
    case ANTS_LRF_XYZ:
        if (z) ANTS_MIN_LAUNCH(ANTS_LRF_XYZ, 3);
        else ANTS_MIN_LAUNCH(ANTS_LRF_XYZ, 2);
        break;
    case ANTS_LRF_AXIAL_Z:
        if (z) ANTS_MIN_LAUNCH(ANTS_LRF_AXIAL_Z, 3);
        else ANTS_MIN_LAUNCH(ANTS_LRF_AXIAL_Z, 2);
        break;
    default:
        if (z) ANTS_MIN_LAUNCH(ANTS_LRF_SLICED, 3);
        else ANTS_MIN_LAUNCH(ANTS_LRF_SLICED, 2);
        break;
    }
#undef ANTS_MIN_LAUNCH
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return cuda_fail(err, "minimize_kernel launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace ants
