// Uniform cubic B-spline evaluation on the device (LRFs of Sec. 6, 6.1).
//
// On a uniform knot grid the four basis functions that are non-zero on a span
// are fixed cubic polynomials of the local parameter t in [0, 1]; the kernels
// evaluate them in that segment form (the CPU oracle uses the Cox-de Boor
// recursion instead).
#pragma once

#include "internal.cuh"

namespace ants {

// the four non-zero uniform cubic B-spline weights at local parameter t
__device__ __forceinline__ void bs_weights(float t, float w[4])
{
    const float k = 1.0f / 6.0f;
    float t2 = t * t, t3 = t2 * t, u = 1.0f - t;
    w[0] = k * u * u * u;
    w[1] = k * fmaf(3.0f, t3, fmaf(-6.0f, t2, 4.0f));
    w[2] = k * fmaf(-3.0f, t3, fmaf(3.0f, t2, fmaf(3.0f, t, 1.0f)));
    w[3] = k * t3;
}

// the same weights in FP64 (LRF fits and the gain refit)
__device__ __forceinline__ void bs_weights_f64(double t, double w[4])
{
    const double k = 1.0 / 6.0;
    double t2 = t * t, t3 = t2 * t, u = 1.0 - t;
    w[0] = k * u * u * u;
    w[1] = k * (3.0 * t3 - 6.0 * t2 + 4.0);
    w[2] = k * (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0);
    w[3] = k * t3;
}

// span index j in [0, n-1] of x and its local parameter t; x == hi falls in
// the last span with t = 1
__device__ __forceinline__ int bs_span(float x, float lo, float inv_h, int n, float &t)
{
    float u = (x - lo) * inv_h;
    int j = (int)floorf(u);
    j = j < 0 ? 0 : (j > n - 1 ? n - 1 : j);
    t = u - (float)j;
    return j;
}

__device__ __forceinline__ bool in_box(const LrfDev &L, float x, float y, float z)
{
    bool ok = x >= L.lo[0] && x <= L.hi[0] && y >= L.lo[1] && y <= L.hi[1];
    if (L.type == ANTS_LRF_XYZ || L.type == ANTS_LRF_SLICED) ok = ok && z >= L.lo[2] && z <= L.hi[2];
    return ok;
}

// a tensor spline of two axes (axis 0 fastest in c, row stride n0 + 3) at
// (u, v), both inside their ranges
__device__ __forceinline__ float spline2(const float *c, float u, float lo0, float inv_h0, int n0, float v, float lo1,
                                         float inv_h1, int n1)
{
    float tu, tv, wu[4], wv[4];
    const int ju = bs_span(u, lo0, inv_h0, n0, tu);
    const int jv = bs_span(v, lo1, inv_h1, n1, tv);
    bs_weights(tu, wu);
    bs_weights(tv, wv);
    const int st = n0 + 3;
    float f = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float *row = c + (jv + b) * st + ju;
        float fr = row[0] * wu[0];
        fr = fmaf(row[1], wu[1], fr);
        fr = fmaf(row[2], wu[2], fr);
        fr = fmaf(row[3], wu[3], fr);
        f = fmaf(fr, wv[b], f);
    }
    return f;
}

// distance in the sensor plane as r^2 times the reciprocal square root of
// r^2 (rsqrtf: within 2 ulp); the floor on the argument makes it 0 at the
// sensor itself
__device__ __forceinline__ float plane_dist(float dx, float dy)
{
    const float r2 = fmaf(dx, dx, dy * dy);
    return r2 * rsqrtf(fmaxf(r2, 1e-30f));
}

// an axial profile at 0 <= r <= hi: its span (the same span and local
// parameter as bs_span with lo = 0, since r >= 0), the span's cubic in the
// power basis of the local parameter, Horner's rule
__device__ __forceinline__ float radial_profile(const float4 *poly, float inv_h, int n, float r)
{
    const float u = r * inv_h;
    const int j = min((int)u, n - 1);
    const float t = u - (float)j;
    const float4 p = __ldg(poly + j);
    return fmaf(t, fmaf(t, fmaf(t, p.w, p.z), p.y), p.x);
}

// the power-basis cubics of sensor i's axial LRF
__device__ __forceinline__ const float4 *radial_poly(const LrfDev &L, int i)
{
    return L.rpoly + (L.shared ? 0 : (L.set_of ? __ldg(L.set_of + i) : i)) * L.n_int[0];
}

// axial LRF of sensor i at distance r (caller checks r <= hi)
__device__ __forceinline__ float radial_eta(const LrfDev &L, int i, float r)
{
    return __ldg(L.gain + i) * radial_profile(radial_poly(L, i), L.inv_h[0], L.n_int[0], r);
}

// eta_i at one point; ok = false outside the domain (used by the evaluation
// entry point and by per-event prologue/epilogue code)
template <int TYPE>
__device__ __forceinline__ float lrf_eta_t(const LrfDev &L, int i, float x, float y, float z, bool &ok)
{
    if (TYPE == ANTS_LRF_RADIAL) {
        const float r = plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]);
        ok = r <= L.hi[0];
        return ok ? radial_eta(L, i, r) : 0.0f;
    }
    if (TYPE == ANTS_LRF_COMPOSITE) {
        // the axial part at r plus the XY part
        const float r = plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]);
        ok = r <= L.hi_r && in_box(L, x, y, z);
        if (!ok) return 0.0f;
        const float *c = L.coef + (size_t)i * L.n_coef + (L.n_int_r + 3);
        return radial_profile(L.rpoly + i * L.n_int_r, L.inv_h_r, L.n_int_r, r) +
               spline2(c, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1], L.n_int[1]);
    }
    if (TYPE == ANTS_LRF_AXIAL_Z) {
        // one spline of (r, z)
        const float r = plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]);
        ok = r <= L.hi[0] && z >= L.lo[1] && z <= L.hi[1];
        if (!ok) return 0.0f;
        return spline2(L.coef + (size_t)i * L.n_coef, r, 0.0f, L.inv_h[0], L.n_int[0], z, L.lo[1], L.inv_h[1],
                       L.n_int[1]);
    }
    if (TYPE == ANTS_LRF_SLICED) {
        // the XY splines of the two closest planes, blended linearly in z
        ok = in_box(L, x, y, z);
        if (!ok) return 0.0f;
        const float u = (z - L.lo[2]) * L.inv_h[2];
        const int j = min(max((int)floorf(u), 0), L.n_planes - 2);
        const float w = u - (float)j;
        const float *c = L.coef + (size_t)i * L.n_coef + (size_t)j * L.n_coef_xy;
        const float f0 = spline2(c, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1], L.n_int[1]);
        const float f1 =
            spline2(c + L.n_coef_xy, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1], L.n_int[1]);
        return fmaf(w, f1, (1.0f - w) * f0);
    }
    const float *c = L.coef + (size_t)i * L.n_coef;
    float gs = 1.0f;
    if (TYPE == kLrfXYSym) {
        // a symmetry class: the representative's LRF at M^T (p - c) + c, times the gain
        float m[4];
        sym_op(__ldg(L.op_of + i), m);
        const float dx = x - L.sym_c[0], dy = y - L.sym_c[1];
        x = fmaf(m[0], dx, fmaf(m[2], dy, L.sym_c[0]));
        y = fmaf(m[1], dx, fmaf(m[3], dy, L.sym_c[1]));
        c = L.coef + (size_t)__ldg(L.set_of + i) * L.n_coef;
        gs = __ldg(L.gain + i);
    }
    ok = in_box(L, x, y, z);
    if (!ok) return 0.0f;
    float tx, ty, tz = 0.0f, wx[4], wy[4], wz[4] = {1.0f, 0.0f, 0.0f, 0.0f};
    int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
    int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
    int jz = 0, nz = 1;
    bs_weights(tx, wx);
    bs_weights(ty, wy);
    if (TYPE == ANTS_LRF_XYZ) {
        jz = bs_span(z, L.lo[2], L.inv_h[2], L.n_int[2], tz);
        bs_weights(tz, wz);
        nz = 4;
    }
    float f = 0.0f;
    for (int cz = 0; cz < nz; ++cz) {
        float fz = 0.0f;
        for (int b = 0; b < 4; ++b) {
            const float *row = c + (jz + cz) * L.stride_z + (jy + b) * L.stride_y + jx;
            float fr = row[0] * wx[0];
            fr = fmaf(row[1], wx[1], fr);
            fr = fmaf(row[2], wx[2], fr);
            fr = fmaf(row[3], wx[3], fr);
            fz = fmaf(fr, wy[b], fz);
        }
        f = fmaf(fz, wz[cz], f);
    }
    return gs * f;
}

// the same with the type read at run time
__device__ __forceinline__ float lrf_eta_point(const LrfDev &L, int i, float x, float y, float z, bool &ok)
{
    switch (L.type) {
    case ANTS_LRF_RADIAL: return lrf_eta_t<ANTS_LRF_RADIAL>(L, i, x, y, z, ok);
    case ANTS_LRF_XY: return L.set_of ? lrf_eta_t<kLrfXYSym>(L, i, x, y, z, ok) : lrf_eta_t<ANTS_LRF_XY>(L, i, x, y, z, ok);
    case ANTS_LRF_XYZ: return lrf_eta_t<ANTS_LRF_XYZ>(L, i, x, y, z, ok);
    case ANTS_LRF_COMPOSITE: return lrf_eta_t<ANTS_LRF_COMPOSITE>(L, i, x, y, z, ok);
    case ANTS_LRF_AXIAL_Z: return lrf_eta_t<ANTS_LRF_AXIAL_Z>(L, i, x, y, z, ok);
    default: return lrf_eta_t<ANTS_LRF_SLICED>(L, i, x, y, z, ok);
    }
}

// derivatives of the four weights along the local parameter t
__device__ __forceinline__ void bs_dweights(float t, float d[4])
{
    const float u = 1.0f - t;
    d[0] = -0.5f * u * u;
    d[1] = 0.5f * t * fmaf(3.0f, t, -4.0f);
    d[2] = 0.5f * fmaf(t, fmaf(-3.0f, t, 2.0f), 1.0f);
    d[3] = 0.5f * t * t;
}

// spline2 with its partial derivatives along u and v
__device__ __forceinline__ float spline2_grad(const float *c, float u, float lo0, float inv_h0, int n0, float v,
                                              float lo1, float inv_h1, int n1, float &du, float &dv)
{
    float tu, tv, wu[4], wv[4], du4[4], dv4[4];
    const int ju = bs_span(u, lo0, inv_h0, n0, tu);
    const int jv = bs_span(v, lo1, inv_h1, n1, tv);
    bs_weights(tu, wu);
    bs_weights(tv, wv);
    bs_dweights(tu, du4);
    bs_dweights(tv, dv4);
    const int st = n0 + 3;
    float f = 0.0f, fu = 0.0f, fv = 0.0f;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const float *row = c + (jv + b) * st + ju;
        float fr = 0.0f, fru = 0.0f;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            fr = fmaf(row[a], wu[a], fr);
            fru = fmaf(row[a], du4[a], fru);
        }
        f = fmaf(fr, wv[b], f);
        fu = fmaf(fru, wv[b], fu);
        fv = fmaf(fr, dv4[b], fv);
    }
    du = fu * inv_h0;
    dv = fv * inv_h1;
    return f;
}

// an axial profile and its derivative along r (power-basis cubic of the span)
__device__ __forceinline__ float radial_profile_grad(const float4 *poly, float inv_h, int n, float r, float &dr)
{
    const float u = r * inv_h;
    const int j = min((int)u, n - 1);
    const float t = u - (float)j;
    const float4 p = __ldg(poly + j);
    dr = fmaf(t, fmaf(3.0f * t, p.w, 2.0f * p.z), p.y) * inv_h;
    return fmaf(t, fmaf(t, fmaf(t, p.w, p.z), p.y), p.x);
}

// eta_i at one point and its gradient (gx, gy, gz) = (d/dx, d/dy, d/dz),
// gz = 0 for 2D LRFs; an axial part's direction (dx, dy) / r is 0 at the
// sensor itself; ok = false outside the domain
template <int TYPE>
__device__ __forceinline__ float lrf_eta_grad_t(const LrfDev &L, int i, float x, float y, float z, bool &ok, float &gx,
                                                float &gy, float &gz)
{
    gx = gy = gz = 0.0f;
    const float dx = x - L.sxy[2 * i], dy = y - L.sxy[2 * i + 1];
    const float r2 = fmaf(dx, dx, dy * dy), rinv = rsqrtf(fmaxf(r2, 1e-30f)), r = r2 * rinv;
    if (TYPE == ANTS_LRF_RADIAL) {
        ok = r <= L.hi[0];
        if (!ok) return 0.0f;
        float dr;
        const float g = __ldg(L.gain + i);
        const float f = radial_profile_grad(radial_poly(L, i), L.inv_h[0], L.n_int[0], r, dr);
        gx = g * dr * dx * rinv;
        gy = g * dr * dy * rinv;
        return g * f;
    }
    if (TYPE == ANTS_LRF_COMPOSITE) {
        ok = r <= L.hi_r && in_box(L, x, y, z);
        if (!ok) return 0.0f;
        float dr, fx, fy;
        const float fa = radial_profile_grad(L.rpoly + i * L.n_int_r, L.inv_h_r, L.n_int_r, r, dr);
        const float *c = L.coef + (size_t)i * L.n_coef + (L.n_int_r + 3);
        const float fxy = spline2_grad(c, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1], L.n_int[1], fx, fy);
        gx = fmaf(dr * dx, rinv, fx);
        gy = fmaf(dr * dy, rinv, fy);
        return fa + fxy;
    }
    if (TYPE == ANTS_LRF_AXIAL_Z) {
        ok = r <= L.hi[0] && z >= L.lo[1] && z <= L.hi[1];
        if (!ok) return 0.0f;
        float fr, fz;
        const float f = spline2_grad(L.coef + (size_t)i * L.n_coef, r, 0.0f, L.inv_h[0], L.n_int[0], z, L.lo[1],
                                     L.inv_h[1], L.n_int[1], fr, fz);
        gx = fr * dx * rinv;
        gy = fr * dy * rinv;
        gz = fz;
        return f;
    }
    if (TYPE == ANTS_LRF_SLICED) {
        ok = in_box(L, x, y, z);
        if (!ok) return 0.0f;
        const float u = (z - L.lo[2]) * L.inv_h[2];
        const int j = min(max((int)floorf(u), 0), L.n_planes - 2);
        const float w = u - (float)j;
        const float *c = L.coef + (size_t)i * L.n_coef + (size_t)j * L.n_coef_xy;
        float f0x, f0y, f1x, f1y;
        const float f0 = spline2_grad(c, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1], L.n_int[1], f0x, f0y);
        const float f1 = spline2_grad(c + L.n_coef_xy, x, L.lo[0], L.inv_h[0], L.n_int[0], y, L.lo[1], L.inv_h[1],
                                      L.n_int[1], f1x, f1y);
        gx = fmaf(w, f1x, (1.0f - w) * f0x);
        gy = fmaf(w, f1y, (1.0f - w) * f0y);
        gz = (f1 - f0) * L.inv_h[2];
        return fmaf(w, f1, (1.0f - w) * f0);
    }
    const float *c = L.coef + (size_t)i * L.n_coef;
    float gs = 1.0f, m[4] = {1.0f, 0.0f, 0.0f, 1.0f};
    if (TYPE == kLrfXYSym) {
        sym_op(__ldg(L.op_of + i), m);
        const float dx = x - L.sym_c[0], dy = y - L.sym_c[1];
        x = fmaf(m[0], dx, fmaf(m[2], dy, L.sym_c[0]));
        y = fmaf(m[1], dx, fmaf(m[3], dy, L.sym_c[1]));
        c = L.coef + (size_t)__ldg(L.set_of + i) * L.n_coef;
        gs = __ldg(L.gain + i);
    }
    ok = in_box(L, x, y, z);
    if (!ok) return 0.0f;
    float tx, ty, tz = 0.0f, wx[4], wy[4], wz[4] = {1.0f, 0.0f, 0.0f, 0.0f};
    float ddx[4], ddy[4], ddz[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    const int jx = bs_span(x, L.lo[0], L.inv_h[0], L.n_int[0], tx);
    const int jy = bs_span(y, L.lo[1], L.inv_h[1], L.n_int[1], ty);
    int jz = 0, nz = 1;
    bs_weights(tx, wx);
    bs_weights(ty, wy);
    bs_dweights(tx, ddx);
    bs_dweights(ty, ddy);
    if (TYPE == ANTS_LRF_XYZ) {
        jz = bs_span(z, L.lo[2], L.inv_h[2], L.n_int[2], tz);
        bs_weights(tz, wz);
        bs_dweights(tz, ddz);
        nz = 4;
    }
    float f = 0.0f, fx = 0.0f, fy = 0.0f, fz = 0.0f;
    for (int cz = 0; cz < nz; ++cz) {
        float a0 = 0.0f, ax = 0.0f, ay = 0.0f;
        for (int b = 0; b < 4; ++b) {
            const float *row = c + (jz + cz) * L.stride_z + (jy + b) * L.stride_y + jx;
            float fr = 0.0f, frx = 0.0f;
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                fr = fmaf(row[a], wx[a], fr);
                frx = fmaf(row[a], ddx[a], frx);
            }
            a0 = fmaf(fr, wy[b], a0);
            ax = fmaf(frx, wy[b], ax);
            ay = fmaf(fr, ddy[b], ay);
        }
        f = fmaf(a0, wz[cz], f);
        fx = fmaf(ax, wz[cz], fx);
        fy = fmaf(ay, wz[cz], fy);
        fz = fmaf(a0, ddz[cz], fz);
    }
    gx = fx * L.inv_h[0];
    gy = fy * L.inv_h[1];
    gz = TYPE == ANTS_LRF_XYZ ? fz * L.inv_h[2] : 0.0f;
    if (TYPE == kLrfXYSym) {
        // the gradient of F(M^T (p - c) + c) is M grad F
        const float ux = gx, uy = gy;
        gx = gs * fmaf(m[0], ux, m[1] * uy);
        gy = gs * fmaf(m[2], ux, m[3] * uy);
    }
    return gs * f;
}

// every LRF of the sensors with s_act[i] != 0 (all sensors when s_act is
// NULL) defined at the point: within reach of each sensor for the axial
// parts, inside the XY box, inside the z range
__device__ __forceinline__ bool lrf_defined(const LrfDev &L, const float *s_act, float x, float y, float z)
{
    if (L.type == ANTS_LRF_RADIAL || L.type == ANTS_LRF_COMPOSITE || L.type == ANTS_LRF_AXIAL_Z) {
        const float rhi = L.type == ANTS_LRF_COMPOSITE ? L.hi_r : L.hi[0];
        for (int i = 0; i < L.n_s; ++i)
            if ((!s_act || s_act[i] != 0.0f) && plane_dist(x - L.sxy[2 * i], y - L.sxy[2 * i + 1]) > rhi) return false;
    }
    if (L.type == ANTS_LRF_AXIAL_Z) return z >= L.lo[1] && z <= L.hi[1];
    if (L.type == ANTS_LRF_RADIAL) return true;
    if (L.type == ANTS_LRF_XY && L.set_of) {
        // symmetry classes: every sensor's mapped point inside the box
        for (int i = 0; i < L.n_s; ++i) {
            if (s_act && s_act[i] == 0.0f) continue;
            float m[4];
            sym_op(__ldg(L.op_of + i), m);
            const float dx = x - L.sym_c[0], dy = y - L.sym_c[1];
            const float u = fmaf(m[0], dx, fmaf(m[2], dy, L.sym_c[0]));
            const float v = fmaf(m[1], dx, fmaf(m[3], dy, L.sym_c[1]));
            if (!in_box(L, u, v, z)) return false;
        }
        return true;
    }
    return in_box(L, x, y, z);
}

}  // namespace ants
