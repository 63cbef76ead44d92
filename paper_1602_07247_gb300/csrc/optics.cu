// Optical photon transport in a stack of horizontal slabs (Sec. 4.2.3 photon
// tracing, 4.2.4 detection, 4.2.6 pre-rejection; Sec. 3.5 custom interface
// properties).  One thread per photon: isotropic emission from the source,
// then tracing cycles (distance to the next interface; absorption and
// Rayleigh ranges drawn from exponentials; at an interface the custom
// properties, then unpolarised Fresnel reflection or Snell refraction) until
// the photon is absorbed, leaves the stack, enters a sensor window on the
// bottom boundary (detection test: QE times the angular response) or runs
// out of cycles.  Each photon draws from its own Philox4x32-10 stream, counter
// (photon, source, tag, block), in a fixed order, so the results do not depend
// on the launch shape.  Templated on the arithmetic type: the FP64 instance
// takes every decision in the precision of the CPU oracle, the FP32 one is the
// fast mode.  A lane whose photon ends starts its next one in the same loop
// iteration.  Detections are counted per block in shared memory and added to
// the global counts once per block and sensor.
#include <cmath>

#include "internal.cuh"
#include "philox.cuh"

namespace ants {

namespace {

constexpr int kMaxLayers = ANTS_OPT_MAX_LAYERS;
constexpr int kMaxOptSensors = 256;
constexpr int kMaxAng = 64;
constexpr uint32_t kTag = 0x0F7105u;
constexpr int kOptThreads = 256;

// the geometry in the kernel's arithmetic type (converted once on the host,
// so the FP32 kernel does no double-precision work)
template <typename R>
struct OptArgs {
    int n_layers, n_s, n_ang, max_cycles, pre_reject;
    R z[kMaxLayers + 1], n[kMaxLayers], abs_len[kMaxLayers], ray_len[kMaxLayers];
    R n_below, n_above, half_x, half_y;
    R p_abs[kMaxLayers + 1], p_spec[kMaxLayers + 1], p_diff[kMaxLayers + 1];
    R sensor_half, n_sensor, p_max;
    R sx[kMaxOptSensors], sy[kMaxOptSensors], qe[kMaxOptSensors];
    R ang[kMaxAng];
    uint32_t k0, k1;
    const float *src;
    long n_src, n_ph;
    int32_t *counts;
    int16_t *outcome;
};

template <typename R> struct M;
template <> struct M<float> {
    static __device__ __forceinline__ float log(float x) { return logf(x); }
    static __device__ __forceinline__ float sqrt(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float cbrt(float x) { return cbrtf(x); }
    static __device__ __forceinline__ float acos(float x) { return acosf(x); }
    static __device__ __forceinline__ void sincos(float x, float *s, float *c) { sincosf(x, s, c); }
    static __device__ __forceinline__ float u(uint32_t w) { return u01(w); }
};
template <> struct M<double> {
    static __device__ __forceinline__ double log(double x) { return ::log(x); }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double cbrt(double x) { return ::cbrt(x); }
    static __device__ __forceinline__ double acos(double x) { return ::acos(x); }
    static __device__ __forceinline__ void sincos(double x, double *s, double *c) { ::sincos(x, s, c); }
    static __device__ __forceinline__ double u(uint32_t w) { return u01d(w); }
};

// the photon's uniform stream: Philox blocks of counter (photon, source, tag, n)
struct PhotonStream {
    uint32_t k0, k1, p, q, n, buf[4];
    int pos;
    template <typename R> __device__ __forceinline__ R next()
    {
        if (pos == 4) {
            buf[0] = p;
            buf[1] = q;
            buf[2] = kTag;
            buf[3] = n++;
            philox10(k0, k1, buf);
            pos = 0;
        }
        // a select chain keeps the block in registers (no dynamic indexing)
        const uint32_t w = pos == 0 ? buf[0] : pos == 1 ? buf[1] : pos == 2 ? buf[2] : buf[3];
        ++pos;
        return M<R>::u(w);
    }
};

// unpolarised Fresnel reflection coefficient from n1 into n2 at incidence
// cosine ci (1 beyond the critical angle)
template <typename R>
__device__ __forceinline__ R fresnel(R n1, R n2, R ci)
{
    const R si2 = R(1) - ci * ci, st2 = (n1 / n2) * (n1 / n2) * si2;
    if (st2 >= R(1)) return R(1);
    const R ct = M<R>::sqrt(R(1) - st2);
    const R rs = (n1 * ci - n2 * ct) / (n1 * ci + n2 * ct);
    const R rp = (n1 * ct - n2 * ci) / (n1 * ct + n2 * ci);
    return R(0.5) * (rs * rs + rp * rp);
}

// a unit direction at angle acos(mu) from d and azimuth phi about it
template <typename R>
__device__ __forceinline__ void turn(R d[3], R mu, R phi)
{
    R sp, cp;
    M<R>::sincos(phi, &sp, &cp);
    const R s = M<R>::sqrt(fmax(R(0), R(1) - mu * mu));
    R nx, ny, nz;
    if (fabs(d[2]) > R(0.99999)) {
        const R sg = d[2] > R(0) ? R(1) : R(-1);
        nx = s * cp;
        ny = s * sp;
        nz = sg * mu;
    } else {
        const R a = M<R>::sqrt(R(1) - d[2] * d[2]);
        nx = mu * d[0] + s * (d[0] * d[2] * cp - d[1] * sp) / a;
        ny = mu * d[1] + s * (d[1] * d[2] * cp + d[0] * sp) / a;
        nz = mu * d[2] - s * a * cp;
    }
    d[0] = nx;
    d[1] = ny;
    d[2] = nz;
}

template <typename R>
__device__ __forceinline__ R ang_resp(const OptArgs<R> &a, R ci)
{
    if (a.n_ang < 2) return R(1);
    const R th = M<R>::acos(fmin(R(1), fmax(R(0), ci))) / R(0.5 * 3.14159265358979323846) * R(a.n_ang - 1);
    const int j = (int)floor(th);
    if (j >= a.n_ang - 1) return R(a.ang[a.n_ang - 1]);
    const R w = th - R(j);
    return (R(1) - w) * R(a.ang[j]) + w * R(a.ang[j + 1]);
}

constexpr int kGoOn = 1000;  // a photon still in flight

// the state of a photon in flight
template <typename R>
struct Photon {
    PhotonStream st;
    R r[3], d[3], u_det;
    int k, cyc;
};

// emission of photon p of source q: ANTS_PH_REJECTED or kGoOn
template <typename R>
__device__ __forceinline__ int photon_start(const OptArgs<R> &a, Photon<R> &ph, uint32_t q, uint32_t p)
{
    ph.st = PhotonStream{a.k0, a.k1, p, q, 0u, {0u, 0u, 0u, 0u}, 4};
    ph.u_det = R(-1);
    ph.cyc = 0;
    if (a.pre_reject) {
        ph.u_det = ph.st.template next<R>();
        if (!(ph.u_det < a.p_max)) return ANTS_PH_REJECTED;
    }
    const R x0 = R(a.src[3 * (size_t)q]), y0 = R(a.src[3 * (size_t)q + 1]), z0 = R(a.src[3 * (size_t)q + 2]);
    int k = 0;
    while (k < a.n_layers - 1 && z0 >= a.z[k + 1]) ++k;
    ph.k = k;
    ph.r[0] = x0;
    ph.r[1] = y0;
    ph.r[2] = z0;
    const R mu = R(2) * ph.st.template next<R>() - R(1), phi = R(2 * 3.14159265358979323846) * ph.st.template next<R>();
    R sp, cp;
    M<R>::sincos(phi, &sp, &cp);
    const R s = M<R>::sqrt(fmax(R(0), R(1) - mu * mu));
    ph.d[0] = s * cp;
    ph.d[1] = s * sp;
    ph.d[2] = mu;
    return kGoOn;
}

// one tracing cycle of a photon in flight: its outcome, or kGoOn
template <typename R>
__device__ __forceinline__ int photon_cycle(const OptArgs<R> &a, const R *s_sx, const R *s_sy, Photon<R> &ph)
{
    if (ph.cyc >= a.max_cycles) return ANTS_PH_MAX_CYCLES;
    ++ph.cyc;
    R *r = ph.r, *d = ph.d;
    int &k = ph.k;
    PhotonStream &st = ph.st;
    R &u_det = ph.u_det;
    const R hx = a.half_x, hy = a.half_y, inf = R(INFINITY), half = a.sensor_half;
    R tz = inf, tw = inf;
    int b = -1;
    if (d[2] > R(0)) {
        tz = (R(a.z[k + 1]) - r[2]) / d[2];
        b = k + 1;
    } else if (d[2] < R(0)) {
        tz = (R(a.z[k]) - r[2]) / d[2];
        b = k;
    }
    if (d[0] != R(0)) tw = ((d[0] > R(0) ? hx : -hx) - r[0]) / d[0];
    if (d[1] != R(0)) {
        const R ty = ((d[1] > R(0) ? hy : -hy) - r[1]) / d[1];
        tw = ty < tw ? ty : tw;
    }
    const R ua = st.next<R>(), ur = st.next<R>();
    const R sa = a.abs_len[k] > R(0) ? -a.abs_len[k] * M<R>::log(ua) : inf;
    const R sr = a.ray_len[k] > R(0) ? -a.ray_len[k] * M<R>::log(ur) : inf;
    const R t = tz < tw ? tz : tw, s = sa < sr ? sa : sr;
    if (s < t) {
        for (int c = 0; c < 3; ++c) r[c] += s * d[c];
        if (sa <= sr) return ANTS_PH_ABSORBED;
        const R uq = st.next<R>();
        const R qq = R(4) * uq - R(2), rr = M<R>::sqrt(qq * qq + R(1));
        const R mu = M<R>::cbrt(qq + rr) + M<R>::cbrt(qq - rr);
        turn<R>(d, mu, R(2 * 3.14159265358979323846) * st.next<R>());
        return kGoOn;
    }
    if (tw <= tz) return ANTS_PH_ESCAPED;
    for (int c = 0; c < 3; ++c) r[c] += tz * d[c];
    r[2] = R(a.z[b]);
    const R ci = fabs(d[2]);
    int sens = -1;
    if (b == 0)
        for (int i = 0; i < a.n_s; ++i)
            if (fabs(r[0] - s_sx[i]) <= half && fabs(r[1] - s_sy[i]) <= half) {
                sens = i;
                break;
            }
    if (sens >= 0) {
        if (st.next<R>() < fresnel<R>(R(a.n[k]), R(a.n_sensor), ci)) {
            d[2] = -d[2];
            return kGoOn;
        }
        const R pd = R(a.qe[sens]) * ang_resp<R>(a, ci);
        if (u_det < R(0)) u_det = st.next<R>();
        return u_det < pd ? sens : ANTS_PH_UNDETECTED;
    }
    const R pa = R(a.p_abs[b]), ps = R(a.p_spec[b]), pf = R(a.p_diff[b]);
    if (pa + ps + pf > R(0)) {
        const R u = st.next<R>();
        if (u < pa) return ANTS_PH_ABSORBED;
        if (u < pa + ps) {
            d[2] = -d[2];
            return kGoOn;
        }
        if (u < pa + ps + pf) {
            const R mu = M<R>::sqrt(st.next<R>()), phi = R(2 * 3.14159265358979323846) * st.next<R>();
            R sp, cp;
            M<R>::sincos(phi, &sp, &cp);
            const R sn = M<R>::sqrt(fmax(R(0), R(1) - mu * mu));
            d[0] = sn * cp;
            d[1] = sn * sp;
            d[2] = b == k + 1 ? -mu : mu;
            return kGoOn;
        }
    }
    const R n1 = R(a.n[k]);
    const R n2 = b == k + 1 ? (b == a.n_layers ? R(a.n_above) : R(a.n[k + 1])) : (b == 0 ? R(a.n_below) : R(a.n[k - 1]));
    if (st.next<R>() < fresnel<R>(n1, n2, ci)) {
        d[2] = -d[2];
        return kGoOn;
    }
    if (b == 0 || b == a.n_layers) return ANTS_PH_ESCAPED;
    const R eta = n1 / n2, ct = M<R>::sqrt(fmax(R(0), R(1) - eta * eta * (R(1) - ci * ci)));
    d[0] *= eta;
    d[1] *= eta;
    d[2] = d[2] > R(0) ? ct : -ct;
    k = b == k + 1 ? k + 1 : k - 1;
    return kGoOn;
}

// grid (photon blocks, sources): each block traces a strided share of one
// source's photons and adds its per-sensor counts once
template <typename R>
__global__ void __launch_bounds__(kOptThreads) trace_kernel(const __grid_constant__ OptArgs<R> a)
{
    __shared__ int hist[kMaxOptSensors];
    __shared__ R s_sx[kMaxOptSensors], s_sy[kMaxOptSensors];
    const uint32_t q = blockIdx.y;
    for (int i = threadIdx.x; i < a.n_s; i += blockDim.x) {
        hist[i] = 0;
        s_sx[i] = R(a.sx[i]);
        s_sy[i] = R(a.sy[i]);
    }
    __syncthreads();
    // a lane whose photon ends starts its next one at once, so the lanes of a
    // warp stay busy however long the individual paths are
    const long stride = (long)gridDim.x * blockDim.x;
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    Photon<R> ph;
    bool have = p < a.n_ph;
    int o = have ? photon_start<R>(a, ph, q, (uint32_t)p) : kGoOn;
    while (have) {
        if (o == kGoOn) o = photon_cycle<R>(a, s_sx, s_sy, ph);
        if (o != kGoOn) {
            if (o >= 0) atomicAdd(&hist[o], 1);
            if (a.outcome) a.outcome[(size_t)q * a.n_ph + p] = (int16_t)o;
            p += stride;
            have = p < a.n_ph;
            if (have) o = photon_start<R>(a, ph, q, (uint32_t)p);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < a.n_s; i += blockDim.x)
        if (hist[i]) atomicAdd(&a.counts[(size_t)q * a.n_s + i], hist[i]);
}

__global__ void counts_to_eta(const int32_t *counts, long n, float inv_ph, float *eta)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
        eta[i] = (float)counts[i] * inv_ph;
}

// the FP32 kernel's arguments: every geometry value rounded to float
OptArgs<float> to_float(const OptArgs<double> &d)
{
    OptArgs<float> f;
    f.n_layers = d.n_layers;
    f.n_s = d.n_s;
    f.n_ang = d.n_ang;
    f.max_cycles = d.max_cycles;
    f.pre_reject = d.pre_reject;
    for (int b = 0; b <= kMaxLayers; ++b) {
        f.z[b] = (float)d.z[b];
        f.p_abs[b] = (float)d.p_abs[b];
        f.p_spec[b] = (float)d.p_spec[b];
        f.p_diff[b] = (float)d.p_diff[b];
    }
    for (int k = 0; k < kMaxLayers; ++k) {
        f.n[k] = (float)d.n[k];
        f.abs_len[k] = (float)d.abs_len[k];
        f.ray_len[k] = (float)d.ray_len[k];
    }
    f.n_below = (float)d.n_below;
    f.n_above = (float)d.n_above;
    f.half_x = (float)d.half_x;
    f.half_y = (float)d.half_y;
    f.sensor_half = (float)d.sensor_half;
    f.n_sensor = (float)d.n_sensor;
    f.p_max = (float)d.p_max;
    for (int i = 0; i < kMaxOptSensors; ++i) {
        f.sx[i] = (float)d.sx[i];
        f.sy[i] = (float)d.sy[i];
        f.qe[i] = (float)d.qe[i];
    }
    for (int j = 0; j < kMaxAng; ++j) f.ang[j] = (float)d.ang[j];
    f.k0 = d.k0;
    f.k1 = d.k1;
    f.src = d.src;
    f.n_src = d.n_src;
    f.n_ph = d.n_ph;
    f.counts = d.counts;
    f.outcome = d.outcome;
    return f;
}

}  // namespace

extern "C" ANTS_API int ants_trace_photons(ants_ctx *ctx, const ants_optics_params *P, const float *src_xyz_dev,
                                           long n_src, long n_photons, uint64_t seed, int precision,
                                           int32_t *counts_dev, int16_t *outcome_dev, float *eta_dev, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_trace_photons");
    if (!ctx || !P) return fail(ANTS_E_ARG, "ants_trace_photons: NULL ctx or params");
    if (n_src < 0 || n_photons < 0) return fail(ANTS_E_ARG, "ants_trace_photons: negative counts");
    if (n_src > 65535) return fail(ANTS_E_ARG, "ants_trace_photons: at most 65535 sources per call");
    if (n_photons > 2147483647L) return fail(ANTS_E_ARG, "ants_trace_photons: at most 2^31 - 1 photons per source");
    if (precision != ANTS_F32 && precision != ANTS_F64)
        return fail(ANTS_E_ARG, "ants_trace_photons: precision must be ANTS_F32 or ANTS_F64");
    const int K = P->n_layers;
    if (K < 1 || K > kMaxLayers) return fail(ANTS_E_ARG, "ants_trace_photons: 1..%d layers", kMaxLayers);
    for (int b = 0; b < K; ++b)
        if (!(P->z[b + 1] > P->z[b])) return fail(ANTS_E_ARG, "ants_trace_photons: boundaries must increase");
    for (int k = 0; k < K; ++k)
        if (!(P->n[k] > 0.0) || !(P->abs_len[k] >= 0.0) || !(P->ray_len[k] >= 0.0))
            return fail(ANTS_E_ARG, "ants_trace_photons: layer %d needs n > 0 and lengths >= 0", k);
    for (int b = 0; b <= K; ++b) {
        const double pa = P->p_abs[b], ps = P->p_spec[b], pf = P->p_diff[b];
        if (!(pa >= 0.0 && ps >= 0.0 && pf >= 0.0 && pa + ps + pf <= 1.0))
            return fail(ANTS_E_ARG, "ants_trace_photons: interface %d probabilities must be >= 0 and sum <= 1", b);
    }
    if (!(P->n_below > 0.0) || !(P->n_above > 0.0) || !(P->n_sensor > 0.0) || !(P->half_x > 0.0) ||
        !(P->half_y > 0.0) || !(P->sensor_size > 0.0))
        return fail(ANTS_E_ARG, "ants_trace_photons: indices, extents and the window size must be > 0");
    if (P->n_sensors < 1 || P->n_sensors > kMaxOptSensors || !P->sensor_xy_host || !P->qe_host)
        return fail(ANTS_E_ARG, "ants_trace_photons: 1..%d sensors with positions and QE", kMaxOptSensors);
    if (P->n_ang < 0 || P->n_ang == 1 || P->n_ang > kMaxAng || (P->n_ang > 0 && !P->ang_host))
        return fail(ANTS_E_ARG, "ants_trace_photons: angular response needs 0 or 2..%d samples", kMaxAng);
    if (P->max_cycles < 1) return fail(ANTS_E_ARG, "ants_trace_photons: max_cycles must be >= 1");
    if (n_src > 0 && n_photons > 0 && (!src_xyz_dev || !counts_dev))
        return fail(ANTS_E_ARG, "ants_trace_photons: NULL source or count buffer");
    OptArgs<double> a;
    a.n_layers = K;
    a.n_s = P->n_sensors;
    a.n_ang = P->n_ang;
    a.max_cycles = P->max_cycles;
    a.pre_reject = P->pre_reject != 0;
    for (int b = 0; b <= kMaxLayers; ++b) {
        a.z[b] = b <= K ? P->z[b] : 0.0;
        a.p_abs[b] = b <= K ? P->p_abs[b] : 0.0;
        a.p_spec[b] = b <= K ? P->p_spec[b] : 0.0;
        a.p_diff[b] = b <= K ? P->p_diff[b] : 0.0;
    }
    for (int k = 0; k < kMaxLayers; ++k) {
        a.n[k] = k < K ? P->n[k] : 1.0;
        a.abs_len[k] = k < K ? P->abs_len[k] : 0.0;
        a.ray_len[k] = k < K ? P->ray_len[k] : 0.0;
    }
    a.n_below = P->n_below;
    a.n_above = P->n_above;
    a.half_x = P->half_x;
    a.half_y = P->half_y;
    a.sensor_half = 0.5 * P->sensor_size;
    a.n_sensor = P->n_sensor;
    double qmax = 0.0, amax = P->n_ang < 2 ? 1.0 : 0.0;
    for (int i = 0; i < kMaxOptSensors; ++i) {
        const bool in = i < a.n_s;
        a.sx[i] = in ? P->sensor_xy_host[2 * i] : 0.0;
        a.sy[i] = in ? P->sensor_xy_host[2 * i + 1] : 0.0;
        a.qe[i] = in ? P->qe_host[i] : 0.0;
        if (in && !(a.qe[i] >= 0.0 && a.qe[i] <= 1.0)) return fail(ANTS_E_ARG, "ants_trace_photons: QE in [0, 1]");
        if (in && a.qe[i] > qmax) qmax = a.qe[i];
    }
    for (int j = 0; j < kMaxAng; ++j) {
        a.ang[j] = j < a.n_ang ? P->ang_host[j] : 0.0;
        if (j < a.n_ang && !(a.ang[j] >= 0.0 && a.ang[j] <= 1.0))
            return fail(ANTS_E_ARG, "ants_trace_photons: angular response in [0, 1]");
        if (j < a.n_ang && a.ang[j] > amax) amax = a.ang[j];
    }
    a.p_max = qmax * amax;
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.src = src_xyz_dev;
    a.n_src = n_src;
    a.n_ph = n_photons;
    a.counts = counts_dev;
    a.outcome = outcome_dev;
    if (n_src == 0) return ANTS_OK;
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    ANTS_CUDA_TRY(cudaMemsetAsync(counts_dev, 0, (size_t)n_src * a.n_s * sizeof(int32_t), s), "memset counts");
    if (n_photons > 0) {
        // enough blocks per source to fill the GPU several times over
        long per = ((long)ctx->n_sm * 8 + n_src - 1) / n_src;
        const long need = (n_photons + kOptThreads - 1) / kOptThreads;
        per = per < 1 ? 1 : (per > need ? need : per);
        const dim3 grid((unsigned)per, (unsigned)n_src);
        if (precision == ANTS_F64) {
            trace_kernel<double><<<grid, kOptThreads, 0, s>>>(a);
        } else {
            trace_kernel<float><<<grid, kOptThreads, 0, s>>>(to_float(a));
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "trace_kernel launch");
        count_launch();
    }
    if (eta_dev) {
        const long n = n_src * a.n_s;
        counts_to_eta<<<(unsigned)((n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024), 256, 0, s>>>(
            counts_dev, n, n_photons > 0 ? 1.0f / (float)n_photons : 0.0f, eta_dev);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e, "counts_to_eta launch");
        count_launch();
    }
    return ANTS_OK;
}

}  // namespace ants
