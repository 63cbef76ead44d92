// Event filters (Sec. 5.2) and iterative LRF reconstruction (Sec. 8).
//
// One cycle of the iterative procedure, all on the device:
//   reconstruct every flood event with the current LRFs (contracting grids)
//   -> chi-squared of each reconstruction -> cuts -> compacted list of kept
//   events -> samples (position, s_i / E) of the kept events, optionally
//   with a seeded normal shift of the position -> FP64 least-squares refit
//   (fit.cu) -> for a radial group, the relative gains refitted with the new
//   profile fixed (Sec. 6.3).
// Reductions over sensors or events run in a fixed order (warp butterflies,
// fixed-size block trees, a fixed number of blocks), so every result is
// reproducible bit for bit.
#include <algorithm>
#include <cmath>
#include <vector>

#include "bspline.cuh"
#include "internal.cuh"
#include "philox.cuh"

namespace ants {

namespace {

struct DBuf {
    void *p = nullptr;
    DBuf() = default;
    DBuf(const DBuf &) = delete;
    DBuf &operator=(const DBuf &) = delete;
    ~DBuf() { cudaFree(p); }
};

template <class T>
int dmalloc(DBuf &b, size_t count, const char *what)
{
    cudaFree(b.p);
    b.p = nullptr;
    cudaError_t e = cudaMalloc(&b.p, count * sizeof(T) + 16);
    if (e != cudaSuccess) return fail(ANTS_E_OOM, "cudaMalloc(%s): %s", what, cudaGetErrorString(e));
    return ANTS_OK;
}

#define IT_TRY(x)                        \
    do {                                 \
        int _rc = (x);                   \
        if (_rc != ANTS_OK) return _rc;  \
    } while (0)

constexpr int kEvWarps = 8;  // events (one warp each) per block
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Sec. 5.1.1 centroid with weights s_i / g_i, and the signal sum
__global__ void centroid_kernel(const double *sxy, const double *gain, const float *sig, long n_e, int n_s,
                                float *xyz, float *ssum)
{
    const int lane = threadIdx.x & 31;
    const long e = (long)blockIdx.x * kEvWarps + (threadIdx.x >> 5);
    if (e >= n_e) return;  // warp-uniform
    const float *s = sig + e * n_s;
    double S = 0.0, W = 0.0, X = 0.0, Y = 0.0;
    for (int i = lane; i < n_s; i += 32) {
        const double v = (double)s[i], w = v / gain[i];
        S += v;
        W += w;
        X += sxy[2 * i] * w;
        Y += sxy[2 * i + 1] * w;
    }
    S = warp_sum(S);
    W = warp_sum(W);
    X = warp_sum(X);
    Y = warp_sum(Y);
    if (lane == 0) {
        const float nan = __int_as_float(0x7fc00000);
        xyz[3 * e] = W > 0.0 ? (float)(X / W) : nan;
        xyz[3 * e + 1] = W > 0.0 ? (float)(Y / W) : nan;
        xyz[3 * e + 2] = 0.0f;
        if (ssum) ssum[e] = (float)S;
    }
}

// Pearson chi-squared per degree of freedom at (xyz, E), and the signal sum
__global__ void chi2_kernel(LrfDev L, const float *sig, long n_e, const float *xyz, const float *E, float *chi2,
                            float *ssum)
{
    const int lane = threadIdx.x & 31;
    const long e = (long)blockIdx.x * kEvWarps + (threadIdx.x >> 5);
    if (e >= n_e) return;  // warp-uniform
    const float x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2], En = E[e];
    const bool fin = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(En);
    const float *s = sig + e * L.n_s;
    // FP32 throughout (FP64 is scarce): s - mu is exact whenever s is within a
    // factor 2 of mu (Sterbenz), so the terms carry the rounding of mu only,
    // and the warp's butterfly sum is pairwise
    float acc = 0.0f, S = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) {
        const float si = s[i];
        S += si;
        if (fin) {
            bool ok;
            const float mu = En * lrf_eta_point(L, i, x, y, z, ok);
            if (ok && mu > 0.0f) {
                const float d = si - mu;
                acc += __fdividef(d * d, mu);
            }
        }
    }
    acc = warp_sum_f(acc);
    S = warp_sum_f(S);
    if (lane == 0) {
        const float dof = L.n_s > 3 ? (float)(L.n_s - 3) : 1.0f;
        chi2[e] = fin ? acc / dof : __int_as_float(0x7fc00000);
        if (ssum) ssum[e] = S;
    }
}

__global__ void filter_flags(long n_e, const int32_t *status, const float *xyz, const float *E, const float *chi2,
                             const float *ssum, ants_event_cuts c, int *flag)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_e) return;
    const float x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2], En = E[e], q = chi2[e];
    bool k = status[e] == ANTS_EVT_OK && isfinite(x) && isfinite(y) && isfinite(z) && isfinite(En) && isfinite(q);
    if (k && c.chi2_max > 0.0) k = (double)q <= c.chi2_max;
    if (k && c.e_hi > c.e_lo) k = (double)En >= c.e_lo && (double)En <= c.e_hi;
    if (k && c.sum_hi > c.sum_lo) k = (double)ssum[e] >= c.sum_lo && (double)ssum[e] <= c.sum_hi;
    if (k && c.r_max > 0.0) {
        const double dx = (double)x - c.cx, dy = (double)y - c.cy;
        // no contraction into an FMA: the same rounding as a plain C evaluation
        k = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= __dmul_rn(c.r_max, c.r_max);
    }
    flag[e] = k ? 1 : 0;
}

__global__ void compact_kernel(const int *flag, const int *pos, long n, int32_t *index)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n && flag[e]) index[pos[e]] = (int32_t)e;
}

// sums of chi2 and E over the kept events: a fixed grid of kStatBlocks
// blocks, each summing a fixed stride pattern, then a fixed tree
constexpr int kStatBlocks = 256, kStatThreads = 256;

__global__ void __launch_bounds__(kStatThreads) kept_sums(const int32_t *index, long n_kept, const float *chi2,
                                                          const float *E, double *part)
{
    __shared__ double s_a[kStatThreads], s_b[kStatThreads];
    double a = 0.0, b = 0.0;
    for (long k = (long)blockIdx.x * kStatThreads + threadIdx.x; k < n_kept; k += (long)kStatBlocks * kStatThreads) {
        const long e = index[k];
        a += (double)chi2[e];
        b += (double)E[e];
    }
    s_a[threadIdx.x] = a;
    s_b[threadIdx.x] = b;
    __syncthreads();
    for (int o = kStatThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_a[0];
        part[2 * blockIdx.x + 1] = s_b[0];
    }
}

// sums over the kept events (at their reconstructed positions) and the
// sensors of (eta_B - eta_A)^2 and eta_A^2, where both are defined
__global__ void __launch_bounds__(kStatThreads) change_sums(LrfDev A, LrfDev B, const int32_t *index, long n_kept,
                                                            const float *xyz, double *part)
{
    __shared__ double s_a[kStatThreads], s_b[kStatThreads];
    const long total = n_kept * A.n_s;
    // a convergence monitor: FP32 partial sums per thread, the tree in FP64
    float d2 = 0.0f, a2 = 0.0f;
    for (long t = (long)blockIdx.x * kStatThreads + threadIdx.x; t < total; t += (long)kStatBlocks * kStatThreads) {
        const long k = t / A.n_s;
        const int i = (int)(t - k * A.n_s);
        const long e = index[k];
        const float x = xyz[3 * e], y = xyz[3 * e + 1], z = xyz[3 * e + 2];
        bool oka, okb;
        const float a = lrf_eta_point(A, i, x, y, z, oka), b = lrf_eta_point(B, i, x, y, z, okb);
        if (oka && okb) {
            const float d = b - a;
            d2 = fmaf(d, d, d2);
            a2 = fmaf(a, a, a2);
        }
    }
    s_a[threadIdx.x] = (double)d2;
    s_b[threadIdx.x] = (double)a2;
    __syncthreads();
    for (int o = kStatThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s_a[0];
        part[2 * blockIdx.x + 1] = s_b[0];
    }
}

// the fixed-order total of the per-block pairs of kept_sums / change_sums
int read_pairs(const double *d_part, std::vector<double> &part, cudaStream_t st, double &a, double &b)
{
    ANTS_CUDA_TRY(cudaMemcpyAsync(part.data(), d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, st),
                  "statistics download");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "statistics");
    a = 0.0;
    b = 0.0;
    for (size_t k = 0; k + 1 < part.size(); k += 2) {
        a += part[k];
        b += part[k + 1];
    }
    return ANTS_OK;
}

// the random shift of Sec. 8: a normal pair of standard deviation sigma from
// the Philox block at counter (e_lo, e_hi, 0xFFFFFFFE, cycle), Box-Muller in FP64
struct ShiftArgs {
    double sigma;
    uint32_t k0, k1, cycle;
};

__device__ __forceinline__ void shift_of(long e, const ShiftArgs &sh, double &dx, double &dy)
{
    dx = 0.0;
    dy = 0.0;
    if (!(sh.sigma > 0.0)) return;
    uint32_t c[4] = {(uint32_t)e, (uint32_t)((unsigned long long)e >> 32), 0xFFFFFFFEu, sh.cycle};
    philox10(sh.k0, sh.k1, c);
    const double ua = u01d(c[0]), ub = u01d(c[1]);
    const double rho = sqrt(-2.0 * log(ua)), th = 6.283185307179586 * ub;
    double sn, cs;
    sincos(th, &sn, &cs);
    dx = sh.sigma * rho * cs;
    dy = sh.sigma * rho * sn;
}

// XY / XYZ samples, one thread per kept event: pts [k][dims], vals [k][n_s]
// = s / E (FP64 is scarce: one division per event, a product per sensor)
__global__ void samples_box(const int32_t *index, long n_kept, int dims, int n_s, const float *xyz, const float *sig,
                            const float *E, ShiftArgs sh, double *pts, double *vals)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_kept) return;
    const long e = index ? index[k] : k;
    double dx, dy;
    shift_of(e, sh, dx, dy);
    pts[k * dims] = (double)xyz[3 * e] + dx;
    pts[k * dims + 1] = (double)xyz[3 * e + 1] + dy;
    if (dims == 3) pts[k * 3 + 2] = (double)xyz[3 * e + 2];
    const double inv_e = 1.0 / (double)E[e];
    for (int i = 0; i < n_s; ++i) vals[k * n_s + i] = (double)sig[e * n_s + i] * inv_e;
}

// XY symmetry-class samples, one thread per kept event: for every sensor i
// its row row_of[i] (the members of a class in consecutive rows) receives
// the event's position mapped into the class representative's frame, M^T (p
// - c) + c (opm: the operations' 2 x 2 matrices, row-major), and the value
// v / g_i
__global__ void samples_sym(const double *pts, const double *vals, long n_kept, int n_s, const int *row_of,
                            const int *op_of, const double *opm, double cx, double cy, const double *inv_g, double *P,
                            double *V)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_kept) return;
    const double dx = pts[2 * k] - cx, dy = pts[2 * k + 1] - cy;
    for (int i = 0; i < n_s; ++i) {
        const double *M = opm + 4 * op_of[i];
        const long o = (long)row_of[i] * n_kept + k;
        P[2 * o] = M[0] * dx + M[2] * dy + cx;
        P[2 * o + 1] = M[1] * dx + M[3] * dy + cy;
        V[o] = vals[k * n_s + i] * inv_g[i];
    }
}

// RADIAL samples, one thread per kept event: r = distance to sensor i,
// v = s / E (times inv_g[i] when given); by_sensor stores [i][k], otherwise
// [k][i]
__global__ void samples_radial(const int32_t *index, long n_kept, int n_s, const float *xyz, const float *sig,
                               const float *E, const double *sxy, const double *inv_g, ShiftArgs sh, int by_sensor,
                               const int *row_of, double *r, double *v)
{
    const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_kept) return;
    const long e = index ? index[k] : k;
    double dx, dy;
    shift_of(e, sh, dx, dy);
    const double x = (double)xyz[3 * e] + dx, y = (double)xyz[3 * e + 1] + dy;
    const double inv_e = 1.0 / (double)E[e];
    for (int i = 0; i < n_s; ++i) {
        const double ddx = x - sxy[2 * i], ddy = y - sxy[2 * i + 1];
        const double rr = sqrt(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)));
        double vv = (double)sig[e * n_s + i] * inv_e;
        if (inv_g) vv *= inv_g[i];
        const long o = by_sensor ? (long)(row_of ? row_of[i] : i) * n_kept + k : k * n_s + i;
        r[o] = rr;
        v[o] = vv;
    }
}

// Sec. 6.3 gain of sensor i with the profile fixed: sum f(r) v / sum f(r)^2
// over the samples with r inside [0, hi]; one block per sensor
constexpr int kGainThreads = 256;

// (samples event-major, or by sensor in rows row_of[i] when row_of is given;
// sensor i's profile at coef + set_of[i] * nc when set_of is given)
__global__ void __launch_bounds__(kGainThreads) gain_sums(const double *coef_all, int n_int, double hi, long n_kept,
                                                          int n_s, const double *r, const int32_t *index,
                                                          const float *sig, const float *E, const int *row_of,
                                                          const int *set_of, int nc, double *g)
{
    __shared__ double s_a[kGainThreads], s_b[kGainThreads];
    const int i = blockIdx.x;
    const double *coef = coef_all + (set_of ? (size_t)set_of[i] * nc : 0);
    const double inv_h = (double)n_int / hi;
    double fv = 0.0, ff = 0.0;
    for (long k = threadIdx.x; k < n_kept; k += kGainThreads) {
        const double rr = row_of ? r[(long)row_of[i] * n_kept + k] : r[k * n_s + i];
        if (!(rr >= 0.0 && rr <= hi)) continue;
        const double u = rr * inv_h;
        int j = (int)floor(u);
        j = j < 0 ? 0 : (j > n_int - 1 ? n_int - 1 : j);
        double w[4];
        bs_weights_f64(u - (double)j, w);
        const double f = coef[j] * w[0] + coef[j + 1] * w[1] + coef[j + 2] * w[2] + coef[j + 3] * w[3];
        const long e = index ? index[k] : k;
        const double vv = (double)sig[e * n_s + i] * (1.0 / (double)E[e]);
        fv += f * vv;
        ff += f * f;
    }
    s_a[threadIdx.x] = fv;
    s_b[threadIdx.x] = ff;
    __syncthreads();
    for (int o = kGainThreads / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            s_a[threadIdx.x] += s_a[threadIdx.x + o];
            s_b[threadIdx.x] += s_b[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) g[i] = s_b[0] > 0.0 ? s_a[0] / s_b[0] : __longlong_as_double(0x7ff8000000000000LL);
}

unsigned blocks_for(long n, int per) { return (unsigned)((n + per - 1) / per); }

// an LRF set on the input's knot grid and sensors from FP64 coefficients
int make_like(ants_ctx *ctx, const ants_lrf *like, int shared, const std::vector<double> &coef,
              const std::vector<double> *gain, ants_lrf **out)
{
    ants_detector det;
    det.n_s = like->n_s;
    det.xy = like->sxy;
    det.gain = like->rel_gain;
    const long launches = ants_last_launch_count();
    const int rc = like->groups.empty()
                       ? ants_lrf_create(ctx, &det, like->type, like->n_int, like->lo, like->hi, shared, coef.data(),
                                         gain ? gain->data() : nullptr, out)
                       : lrf_create_impl(ctx, &det, ANTS_LRF_RADIAL, like->n_int, like->lo, like->hi, 0, coef.data(),
                                         gain ? gain->data() : nullptr, 0, 0.0, 0, out, like->n_sets,
                                         like->groups.data());
    count_launch(launches);
    return rc;
}

// XY symmetry classes: one fit per class to its members' mapped samples
// (the points outside the box are left out by the fit), gains kept
int refit_symmetric(ants_ctx *ctx, const ants_lrf *lrf, const double *A, const double *B, long n_kept,
                    const ants_refit_params &p, cudaStream_t st, ants_lrf **out)
{
    const int n_s = lrf->n_s, n_sets = lrf->n_sets, nc = lrf->n_coef;
    std::vector<int> row(n_s), first(n_sets + 1, 0);
    for (int i = 0; i < n_s; ++i) first[lrf->groups[i] + 1]++;
    for (int j = 0; j < n_sets; ++j) first[j + 1] += first[j];
    std::vector<int> fill(first.begin(), first.end() - 1);
    for (int i = 0; i < n_s; ++i) row[i] = fill[lrf->groups[i]]++;
    std::vector<double> opm(24 * 4), inv_g(n_s);
    for (int k = 0; k < 24; ++k) {
        const double t = (double)(k % 12) * (3.14159265358979323846 / 6.0);
        double c = std::cos(t), sn = std::sin(t);
        if (k % 3 == 0) {
            const int q = (k % 12) / 3;
            c = q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
            sn = q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
        }
        const double f = k >= 12 ? -1.0 : 1.0;
        opm[4 * k] = c;
        opm[4 * k + 1] = -sn * f;
        opm[4 * k + 2] = sn;
        opm[4 * k + 3] = c * f;
    }
    for (int i = 0; i < n_s; ++i) inv_g[i] = 1.0 / lrf->gain[i];
    const long total = n_kept * (long)n_s;
    Carve cv;
    const size_t o_p = cv.take<double>(2 * (size_t)total), o_v = cv.take<double>(total);
    const size_t o_row = cv.take<int>(n_s), o_op = cv.take<int>(n_s), o_m = cv.take<double>(96),
                 o_g = cv.take<double>(n_s);
    char *base = (char *)ctx_scratch(ctx, 12, cv.off);  // not a slot of the fit
    if (!base) return ANTS_E_OOM;
    double *P = (double *)(base + o_p), *V = (double *)(base + o_v), *d_m = (double *)(base + o_m);
    double *d_g = (double *)(base + o_g);
    int *d_row = (int *)(base + o_row), *d_op = (int *)(base + o_op);
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_row, row.data(), n_s * sizeof(int), cudaMemcpyHostToDevice, st), "refit: rows");
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_op, lrf->ops.data(), n_s * sizeof(int), cudaMemcpyHostToDevice, st),
                  "refit: operations");
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_m, opm.data(), 96 * sizeof(double), cudaMemcpyHostToDevice, st),
                  "refit: matrices");
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_g, inv_g.data(), n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "refit: gains");
    if (n_kept > 0) {
        samples_sym<<<blocks_for(n_kept, 256), 256, 0, st>>>(A, B, n_kept, n_s, d_row, d_op, d_m, lrf->sym_c[0],
                                                             lrf->sym_c[1], d_g, P, V);
        ANTS_CUDA_TRY(cudaGetLastError(), "refit class samples launch");
        count_launch();
    }
    std::vector<double> coef((size_t)n_sets * nc);
    for (int j = 0; j < n_sets; ++j) {
        const long np = (long)(first[j + 1] - first[j]) * n_kept;
        IT_TRY(lrf_fit_samples(ctx, 2, lrf->n_int, lrf->lo, lrf->hi, np, P + 2 * (size_t)first[j] * n_kept, 1,
                               V + (size_t)first[j] * n_kept, p.ridge, coef.data() + (size_t)j * nc, nullptr, st));
    }
    ants_detector det;
    det.n_s = n_s;
    det.xy = lrf->sxy;
    det.gain = lrf->rel_gain;
    const long launches = ants_last_launch_count();
    const int rc = ants_lrf_create_symmetric(ctx, &det, lrf->n_int, lrf->lo, lrf->hi, n_sets, lrf->groups.data(),
                                             lrf->ops.data(), lrf->sym_c, coef.data(), lrf->gain.data(), out);
    count_launch(launches);
    return rc;
}

int refit_lrf(ants_ctx *ctx, const ants_lrf *lrf, const float *sig, const float *xyz, const float *E,
              const int32_t *index, long n_kept, const ants_refit_params &p, cudaStream_t st, ants_lrf **out)
{
    const int n_s = lrf->n_s, dims = lrf_dims(lrf->type);
    const ShiftArgs sh{p.shift_sigma, (uint32_t)p.seed, (uint32_t)(p.seed >> 32), (uint32_t)p.cycle};
    const long total = n_kept * (long)n_s;
    const int T = 256;
    const int nc = lrf->n_coef;
    // the samples and the small per-call tables live in scratch slot 10
    Carve cv;
    const size_t o_a = cv.take<double>(lrf->type == ANTS_LRF_RADIAL ? total : (size_t)n_kept * dims);
    const size_t o_b = cv.take<double>(total);
    const size_t o_sxy = cv.take<double>(2 * (size_t)n_s), o_g = cv.take<double>(n_s);
    const bool grouped = !lrf->groups.empty();
    const int n_sets = lrf->n_sets;
    const size_t o_coef = cv.take<double>((size_t)nc * n_sets), o_graw = cv.take<double>(n_s);
    const size_t o_row = cv.take<int>(n_s), o_set = cv.take<int>(n_s);
    char *base = (char *)ctx_scratch(ctx, 10, cv.off);
    if (!base) return ANTS_E_OOM;
    double *A = (double *)(base + o_a), *B = (double *)(base + o_b);
    if (lrf->type != ANTS_LRF_RADIAL) {
        if (total > 0) {
            samples_box<<<blocks_for(n_kept, T), T, 0, st>>>(index, n_kept, dims, n_s, xyz, sig, E, sh, A, B);
            ANTS_CUDA_TRY(cudaGetLastError(), "refit samples launch");
            count_launch();
        }
        if (!lrf->ops.empty()) return refit_symmetric(ctx, lrf, A, B, n_kept, p, st, out);
        std::vector<double> coef((size_t)n_s * nc);
        IT_TRY(lrf_fit_samples(ctx, dims, lrf->n_int, lrf->lo, lrf->hi, n_kept, A, n_s, B, p.ridge, coef.data(),
                               nullptr, st));
        return make_like(ctx, lrf, 0, coef, nullptr, out);
    }
    double *d_sxy = (double *)(base + o_sxy), *d_g = (double *)(base + o_g);
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_sxy, lrf->sxy.data(), 2 * n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "refit: upload sensors");
    // a per-sensor input has no group gains: its values are divided by 1
    std::vector<double> g_in(n_s, 1.0), inv_g(n_s);
    if (lrf->shared || grouped) g_in = lrf->gain;
    // grouped: the samples of each group's sensors in consecutive rows
    std::vector<int> row(n_s), first(n_sets + 1, 0);
    int *d_row = (int *)(base + o_row), *d_set = (int *)(base + o_set);
    if (grouped) {
        for (int i = 0; i < n_s; ++i) first[lrf->groups[i] + 1]++;
        for (int j = 0; j < n_sets; ++j) first[j + 1] += first[j];
        std::vector<int> fill(first.begin(), first.end() - 1);
        for (int i = 0; i < n_s; ++i) row[i] = fill[lrf->groups[i]]++;
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_row, row.data(), n_s * sizeof(int), cudaMemcpyHostToDevice, st),
                      "refit: upload rows");
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_set, lrf->groups.data(), n_s * sizeof(int), cudaMemcpyHostToDevice, st),
                      "refit: upload groups");
    }
    for (int i = 0; i < n_s; ++i) inv_g[i] = 1.0 / g_in[i];
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_g, inv_g.data(), n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "refit: upload gains");
    double *r = A, *v = B;
    if (total > 0) {
        samples_radial<<<blocks_for(n_kept, T), T, 0, st>>>(index, n_kept, n_s, xyz, sig, E, d_sxy,
                                                            p.shared || grouped ? d_g : nullptr, sh,
                                                            p.shared && !grouped ? 0 : 1, grouped ? d_row : nullptr,
                                                            r, v);
        ANTS_CUDA_TRY(cudaGetLastError(), "refit samples launch");
        count_launch();
    }
    if (grouped) {
        std::vector<double> coef((size_t)n_sets * nc);
        for (int j = 0; j < n_sets; ++j) {
            const long np = (long)(first[j + 1] - first[j]) * n_kept;
            if (np == 0) return fail(ANTS_E_LRF, "refit: group %d has no sensor", j);
            IT_TRY(lrf_fit_samples(ctx, 1, lrf->n_int, lrf->lo, lrf->hi, np, r + (size_t)first[j] * n_kept, 1,
                                   v + (size_t)first[j] * n_kept, p.ridge, coef.data() + (size_t)j * nc, nullptr,
                                   st));
        }
        std::vector<double> gains = g_in;
        if (p.refit_gains) {
            double *d_coef = (double *)(base + o_coef), *d_graw = (double *)(base + o_graw);
            ANTS_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), coef.size() * sizeof(double), cudaMemcpyHostToDevice,
                                          st),
                          "refit: upload profiles");
            gain_sums<<<n_s, kGainThreads, 0, st>>>(d_coef, lrf->n_int[0], lrf->hi[0], n_kept, n_s, r, index, sig, E,
                                                    d_row, d_set, nc, d_graw);
            ANTS_CUDA_TRY(cudaGetLastError(), "gain refit launch");
            count_launch();
            ANTS_CUDA_TRY(cudaMemcpyAsync(gains.data(), d_graw, n_s * sizeof(double), cudaMemcpyDeviceToHost, st),
                          "refit: download gains");
            ANTS_CUDA_TRY(cudaStreamSynchronize(st), "gain refit");
            std::vector<double> gm(n_sets, 0.0);
            for (int i = 0; i < n_s; ++i) {
                if (!std::isfinite(gains[i]) || !(gains[i] > 0.0))
                    return fail(ANTS_E_LRF, "gain refit: sensor %d has no usable samples", i);
                gm[lrf->groups[i]] += gains[i];
            }
            for (int j = 0; j < n_sets; ++j) gm[j] /= (double)(first[j + 1] - first[j]);
            for (int i = 0; i < n_s; ++i) gains[i] /= gm[lrf->groups[i]];
            for (int j = 0; j < n_sets; ++j)
                for (int c = 0; c < nc; ++c) coef[(size_t)j * nc + c] *= gm[j];
        }
        return make_like(ctx, lrf, 0, coef, &gains, out);
    }
    if (!p.shared) {
        std::vector<double> coef((size_t)n_s * nc);
        for (int i = 0; i < n_s; ++i)
            IT_TRY(lrf_fit_samples(ctx, 1, lrf->n_int, lrf->lo, lrf->hi, n_kept, r + (size_t)i * n_kept, 1,
                                   v + (size_t)i * n_kept, p.ridge, coef.data() + (size_t)i * nc, nullptr, st));
        return make_like(ctx, lrf, 0, coef, nullptr, out);
    }
    std::vector<double> coef(nc);
    IT_TRY(lrf_fit_samples(ctx, 1, lrf->n_int, lrf->lo, lrf->hi, total, r, 1, v, p.ridge, coef.data(), nullptr, st));
    std::vector<double> gains = g_in;
    if (p.refit_gains) {
        double *d_coef = (double *)(base + o_coef), *d_graw = (double *)(base + o_graw);
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_coef, coef.data(), nc * sizeof(double), cudaMemcpyHostToDevice, st),
                      "refit: upload profile");
        gain_sums<<<n_s, kGainThreads, 0, st>>>(d_coef, lrf->n_int[0], lrf->hi[0], n_kept, n_s, r, index, sig, E,
                                                nullptr, nullptr, nc, d_graw);
        ANTS_CUDA_TRY(cudaGetLastError(), "gain refit launch");
        count_launch();
        ANTS_CUDA_TRY(cudaMemcpyAsync(gains.data(), d_graw, n_s * sizeof(double), cudaMemcpyDeviceToHost, st),
                      "refit: download gains");
        ANTS_CUDA_TRY(cudaStreamSynchronize(st), "gain refit");
        double gm = 0.0;
        for (int i = 0; i < n_s; ++i) {
            if (!std::isfinite(gains[i]) || !(gains[i] > 0.0))
                return fail(ANTS_E_LRF, "gain refit: sensor %d has no usable samples", i);
            gm += gains[i];
        }
        gm /= (double)n_s;
        for (auto &gg : gains) gg /= gm;
        for (auto &c : coef) c *= gm;
    }
    return make_like(ctx, lrf, 1, coef, &gains, out);
}

int check_cuts(const ants_event_cuts *c)
{
    if (!c) return fail(ANTS_E_ARG, "event cuts are NULL");
    const double v[8] = {c->chi2_max, c->e_lo, c->e_hi, c->sum_lo, c->sum_hi, c->r_max, c->cx, c->cy};
    for (double x : v)
        if (std::isnan(x)) return fail(ANTS_E_ARG, "event cuts: NaN bound");
    return ANTS_OK;
}

int filter_events(ants_ctx *ctx, long n_e, const int32_t *status, const float *xyz, const float *E, const float *chi2,
                  const float *ssum, const ants_event_cuts &c, int32_t *index, long *n_kept, cudaStream_t st)
{
    // flags, positions, scan scratch and the count live in scratch slot 11;
    // the call waits for the count, so nothing is in flight on return
    Carve cv;
    const size_t o_flag = cv.take<int>(n_e), o_pos = cv.take<int>(n_e);
    const size_t o_tmp = cv.take<char>(exclusive_scan_tmp_bytes(n_e)), o_tot = cv.take<int>(1);
    char *base = (char *)ctx_scratch(ctx, 11, cv.off);
    if (!base) return ANTS_E_OOM;
    int *flag = (int *)(base + o_flag), *pos = (int *)(base + o_pos), *tot = (int *)(base + o_tot);
    const int T = 256;
    filter_flags<<<blocks_for(n_e, T), T, 0, st>>>(n_e, status, xyz, E, chi2, ssum, c, flag);
    count_launch();
    IT_TRY(exclusive_scan(flag, pos, n_e, tot, base + o_tmp, st));
    compact_kernel<<<blocks_for(n_e, T), T, 0, st>>>(flag, pos, n_e, index);
    count_launch();
    ANTS_CUDA_TRY(cudaGetLastError(), "filter launch");
    int h = 0;
    ANTS_CUDA_TRY(cudaMemcpyAsync(&h, tot, sizeof(int), cudaMemcpyDeviceToHost, st), "filter: count");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "filter");
    *n_kept = h;
    return ANTS_OK;
}

int check_refit(const ants_lrf *lrf, const ants_refit_params *p)
{
    if (!p) return fail(ANTS_E_ARG, "refit parameters are NULL");
    if (!(p->shift_sigma >= 0.0) || !(p->ridge >= 0.0)) return fail(ANTS_E_ARG, "refit: shift_sigma, ridge >= 0");
    if (p->cycle < 0) return fail(ANTS_E_ARG, "refit: cycle < 0");
    if (lrf->type > ANTS_LRF_XYZ) return fail(ANTS_E_UNIMPLEMENTED, "refit: RADIAL, XY and XYZ LRFs only");
    if (lrf->type != ANTS_LRF_RADIAL && p->shared) return fail(ANTS_E_ARG, "refit: groups are RADIAL only");
    if (p->refit_gains && !(lrf->type == ANTS_LRF_RADIAL && (p->shared || !lrf->groups.empty())))
        return fail(ANTS_E_ARG, "refit: gains are refitted for RADIAL groups only");
    return ANTS_OK;
}

}  // namespace

}  // namespace ants

using namespace ants;

extern "C" ANTS_API int ants_event_centroid(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev,
                                            long n_events, float *xyz_dev, float *sum_dev, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_event_centroid");
    if (!ctx || !lrf || lrf->ctx != ctx || n_events < 0) return fail(ANTS_E_ARG, "ants_event_centroid: bad arguments");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !xyz_dev) return fail(ANTS_E_ARG, "ants_event_centroid: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    const int n_s = lrf->n_s;
    DBuf d_sxy, d_g;
    IT_TRY(dmalloc<double>(d_sxy, (size_t)2 * n_s, "sensor positions"));
    IT_TRY(dmalloc<double>(d_g, (size_t)n_s, "relative gains"));
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_sxy.p, lrf->sxy.data(), 2 * n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "centroid: upload");
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_g.p, lrf->rel_gain.data(), n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "centroid: upload");
    centroid_kernel<<<blocks_for(n_events, kEvWarps), 32 * kEvWarps, 0, st>>>(
        (const double *)d_sxy.p, (const double *)d_g.p, signals_dev, n_events, n_s, xyz_dev, sum_dev);
    ANTS_CUDA_TRY(cudaGetLastError(), "centroid launch");
    count_launch();
    // the staging buffers are freed on return: finish with them first
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "centroid");
    return ANTS_OK;
}

extern "C" ANTS_API int ants_event_chi2(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                                        const float *xyz_dev, const float *E_dev, float *chi2_dev, float *sum_dev,
                                        void *stream)
{
    begin_call();
    ANTS_NVTX("ants_event_chi2");
    if (!ctx || !lrf || lrf->ctx != ctx || n_events < 0) return fail(ANTS_E_ARG, "ants_event_chi2: bad arguments");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !xyz_dev || !E_dev || !chi2_dev) return fail(ANTS_E_ARG, "ants_event_chi2: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    chi2_kernel<<<blocks_for(n_events, kEvWarps), 32 * kEvWarps, 0, (cudaStream_t)stream>>>(
        lrf->dev, signals_dev, n_events, xyz_dev, E_dev, chi2_dev, sum_dev);
    ANTS_CUDA_TRY(cudaGetLastError(), "chi2 launch");
    count_launch();
    return ANTS_OK;
}

extern "C" ANTS_API int ants_event_filter(ants_ctx *ctx, long n_events, const int32_t *status_dev,
                                          const float *xyz_dev, const float *E_dev, const float *chi2_dev,
                                          const float *sum_dev, const ants_event_cuts *cuts, int32_t *index_dev,
                                          long *n_kept_host, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_event_filter");
    if (!ctx || n_events < 0 || !n_kept_host) return fail(ANTS_E_ARG, "ants_event_filter: bad arguments");
    IT_TRY(check_cuts(cuts));
    *n_kept_host = 0;
    if (n_events == 0) return ANTS_OK;
    if (n_events > 0x7fffffffL) return fail(ANTS_E_ARG, "ants_event_filter: more than 2^31 - 1 events");
    if (!status_dev || !xyz_dev || !E_dev || !chi2_dev || !index_dev)
        return fail(ANTS_E_ARG, "ants_event_filter: NULL buffer");
    if (cuts->sum_hi > cuts->sum_lo && !sum_dev)
        return fail(ANTS_E_ARG, "ants_event_filter: the signal-sum cut needs sum_dev");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    return filter_events(ctx, n_events, status_dev, xyz_dev, E_dev, chi2_dev, sum_dev, *cuts, index_dev, n_kept_host,
                         (cudaStream_t)stream);
}

extern "C" ANTS_API int ants_lrf_refit(ants_ctx *ctx, const ants_lrf *lrf, const float *signals_dev, long n_events,
                                       const float *xyz_dev, const float *E_dev, const int32_t *index_dev,
                                       long n_kept, const ants_refit_params *p, ants_lrf **out)
{
    begin_call();
    ANTS_NVTX("ants_lrf_refit");
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_refit: out is NULL");
    *out = nullptr;
    if (!ctx || !lrf || lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_lrf_refit: bad context or LRF");
    IT_TRY(check_refit(lrf, p));
    if (n_events < 0 || n_kept < 0 || (!index_dev && n_kept != n_events) || n_kept > n_events)
        return fail(ANTS_E_ARG, "ants_lrf_refit: bad event counts");
    if ((long)lrf->n_s * n_kept > (1L << 30)) return fail(ANTS_E_ARG, "ants_lrf_refit: more than 2^30 samples");
    if (n_kept > 0 && (!signals_dev || !xyz_dev || !E_dev)) return fail(ANTS_E_ARG, "ants_lrf_refit: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    return refit_lrf(ctx, lrf, signals_dev, xyz_dev, E_dev, index_dev, n_kept, *p, ctx->stream[0], out);
}

extern "C" ANTS_API int ants_lrf_iterate(ants_ctx *ctx, const ants_lrf *lrf_init, const float *signals_dev,
                                         long n_events, const ants_iter_params *p, ants_iter_stats *stats_host,
                                         ants_lrf **out)
{
    begin_call();
    ANTS_NVTX("ants_lrf_iterate");
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_iterate: out is NULL");
    *out = nullptr;
    if (!ctx || !lrf_init || lrf_init->ctx != ctx || !p) return fail(ANTS_E_ARG, "ants_lrf_iterate: bad arguments");
    if (p->cycles < 1 || p->shift_cycles < 0 || n_events < 1 || n_events > 0x7fffffffL || !signals_dev)
        return fail(ANTS_E_ARG, "ants_lrf_iterate: cycles >= 1, shift_cycles >= 0, 1 <= n_events < 2^31");
    IT_TRY(check_cuts(&p->cuts));
    if (p->method == ANTS_MINIMIZE) {
        IT_TRY(check_minimize_params(lrf_init, &p->minimize));
    } else if (p->method == ANTS_CGS_PLAIN) {
        IT_TRY(check_cgs_params(lrf_init, &p->cgs));
    } else {
        return fail(ANTS_E_ARG, "ants_lrf_iterate: method must be ANTS_CGS_PLAIN or ANTS_MINIMIZE");
    }
    ants_refit_params rp{lrf_init->shared, p->refit_gains, p->shift_sigma, p->seed, 0, p->ridge};
    IT_TRY(check_refit(lrf_init, &rp));
    if ((long)lrf_init->n_s * n_events > (1L << 30))
        return fail(ANTS_E_ARG, "ants_lrf_iterate: more than 2^30 samples");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = ctx->stream[0];
    const long n = n_events;
    DBuf d_xyz, d_E, d_logL, d_status, d_chi2, d_sum, d_index, d_part;
    IT_TRY(dmalloc<float>(d_xyz, (size_t)3 * n, "positions"));
    IT_TRY(dmalloc<float>(d_E, (size_t)n, "energies"));
    IT_TRY(dmalloc<float>(d_logL, (size_t)n, "logL"));
    IT_TRY(dmalloc<int32_t>(d_status, (size_t)n, "status"));
    IT_TRY(dmalloc<float>(d_chi2, (size_t)n, "chi2"));
    IT_TRY(dmalloc<float>(d_sum, (size_t)n, "signal sums"));
    IT_TRY(dmalloc<int32_t>(d_index, (size_t)n, "kept events"));
    IT_TRY(dmalloc<double>(d_part, (size_t)2 * kStatBlocks, "statistics"));
    float *xyz = (float *)d_xyz.p, *E = (float *)d_E.p, *chi2 = (float *)d_chi2.p, *ssum = (float *)d_sum.p;
    int32_t *status = (int32_t *)d_status.p, *index = (int32_t *)d_index.p;
    const ants_lrf *cur = lrf_init;
    ants_lrf *owned = nullptr;
    int rc = ANTS_OK;
    std::vector<double> part(2 * kStatBlocks);
    for (int c = 0; c < p->cycles && rc == ANTS_OK; ++c) {
        rc = p->method == ANTS_MINIMIZE
                 ? reconstruct_minimize(ctx, cur, p->minimize, signals_dev, n, nullptr, xyz, E, (float *)d_logL.p,
                                        status, nullptr, st)
                 : launch_cgs_plain(ctx, cur, p->cgs, signals_dev, n, nullptr, xyz, E, (float *)d_logL.p, status,
                                    nullptr, st);
        if (rc != ANTS_OK) break;
        chi2_kernel<<<blocks_for(n, kEvWarps), 32 * kEvWarps, 0, st>>>(cur->dev, signals_dev, n, xyz, E, chi2, ssum);
        count_launch();
        long n_kept = 0;
        rc = filter_events(ctx, n, status, xyz, E, chi2, ssum, p->cuts, index, &n_kept, st);
        if (rc != ANTS_OK) break;
        if (n_kept == 0) {
            rc = fail(ANTS_E_LRF, "ants_lrf_iterate: cycle %d kept no event", c);
            break;
        }
        kept_sums<<<kStatBlocks, kStatThreads, 0, st>>>(index, n_kept, chi2, E, (double *)d_part.p);
        count_launch();
        double sa = 0.0, sb = 0.0;
        rc = read_pairs((const double *)d_part.p, part, st, sa, sb);
        if (rc != ANTS_OK) break;
        rp.shift_sigma = c < p->shift_cycles ? p->shift_sigma : 0.0;
        rp.cycle = c;
        ants_lrf *next = nullptr;
        rc = refit_lrf(ctx, cur, signals_dev, xyz, E, index, n_kept, rp, st, &next);
        if (rc != ANTS_OK) break;
        if (stats_host) {
            change_sums<<<kStatBlocks, kStatThreads, 0, st>>>(cur->dev, next->dev, index, n_kept, xyz,
                                                              (double *)d_part.p);
            count_launch();
            double d2 = 0.0, a2 = 0.0;
            rc = read_pairs((const double *)d_part.p, part, st, d2, a2);
            if (rc != ANTS_OK) {
                ants_lrf_free(next);
                break;
            }
            stats_host[c].n_kept = n_kept;
            stats_host[c].mean_chi2 = sa / (double)n_kept;
            stats_host[c].mean_E = sb / (double)n_kept;
            stats_host[c].rel_change = a2 > 0.0 ? std::sqrt(d2 / a2) : NAN;
        }
        if (owned) ants_lrf_free(owned);
        owned = next;
        cur = next;
    }
    if (rc != ANTS_OK) {
        if (owned) {
            const std::string keep = ants_last_error();
            ants_lrf_free(owned);
            fail(rc, "%s", keep.c_str());
        }
        return rc;
    }
    *out = owned;
    return ANTS_OK;
}
