// FP64 fits of the composite, axial+z and sliced LRF sets (Sec. 6.1.1,
// 6.1.2) on the device, from host samples (positions, one value per sensor).
//   composite: per sensor the axial part is fitted first to (r_i, v_i); the
//     XY part of all sensors is then fitted to the residuals v_i - A_i(r_i)
//     (a sample beyond the axial part's reach gives a zero residual);
//   axial+z: per sensor one fit of the spline of (r_i, z);
//   sliced: plane j's XY splines are fitted to the samples whose nearest
//     plane is j.
// The sample sets are built by small kernels; every solve is the FP64 fit of
// fit.cu, so the results are bitwise reproducible.
#include <cmath>
#include <vector>

#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

struct SBuf {
    void *p = nullptr;
    SBuf() = default;
    SBuf(const SBuf &) = delete;
    SBuf &operator=(const SBuf &) = delete;
    ~SBuf() { cudaFree(p); }
};

template <class T>
int smalloc(SBuf &b, size_t count, const char *what)
{
    cudaError_t e = cudaMalloc(&b.p, count * sizeof(T) + 16);
    if (e != cudaSuccess) return fail(ANTS_E_OOM, "scheme fit: cudaMalloc(%s): %s", what, cudaGetErrorString(e));
    return ANTS_OK;
}

#define SC_TRY(x)                        \
    do {                                 \
        int _rc = (x);                   \
        if (_rc != ANTS_OK) return _rc;  \
    } while (0)

__device__ __forceinline__ double dist_xy(double x, double y, double sx, double sy)
{
    const double dx = x - sx, dy = y - sy;
    return sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
}

// sensor i's sample column: r (and z) as points, its values
__global__ void scheme_column(const double *pts, long n, int d, double sx, double sy, int with_z, const double *vals,
                              int n_s, int i, double *cp, double *cv)
{
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double r = dist_xy(pts[p * d], pts[p * d + 1], sx, sy);
    if (with_z) {
        cp[2 * p] = r;
        cp[2 * p + 1] = pts[p * d + 2];
    } else {
        cp[p] = r;
    }
    cv[p] = vals[p * n_s + i];
}

// v - A_i(r) per (sample, sensor); 0 where r is beyond the axial part
__global__ void composite_residual(const double *pts, long n, const double *sxy, const double *vals, int n_s,
                                   const double *cr, int nr, double hi_r, double *res)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n_s) return;
    const long p = t / n_s;
    const int i = (int)(t - p * n_s);
    const double r = dist_xy(pts[2 * p], pts[2 * p + 1], sxy[2 * i], sxy[2 * i + 1]);
    if (!(r <= hi_r)) {
        res[t] = 0.0;
        return;
    }
    const double u = r * ((double)nr / hi_r);
    int j = (int)floor(u);
    j = j < 0 ? 0 : (j > nr - 1 ? nr - 1 : j);
    double w[4];
    bs_weights_f64(u - (double)j, w);
    const double *c = cr + (size_t)i * (nr + 3) + j;
    res[t] = vals[t] - (c[0] * w[0] + c[1] * w[1] + c[2] * w[2] + c[3] * w[3]);
}

// 1 when the sample's nearest plane is j: floor((z - z_lo) / dz + 0.5), clamped
__global__ void plane_flags(const double *pts, long n, double z_lo, double dz, int m, int j, int *flag)
{
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    double k = floor((pts[3 * p + 2] - z_lo) / dz + 0.5);
    k = k < 0.0 ? 0.0 : (k > (double)(m - 1) ? (double)(m - 1) : k);
    flag[p] = (int)k == j ? 1 : 0;
}

// the flagged samples' (x, y) and value rows, in index order
__global__ void gather_plane(const double *pts, const double *vals, long n, int n_s, const int *flag, const int *pos,
                             double *gp, double *gv)
{
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n || !flag[p]) return;
    const long k = pos[p];
    gp[2 * k] = pts[3 * p];
    gp[2 * k + 1] = pts[3 * p + 1];
    for (int s = 0; s < n_s; ++s) gv[k * n_s + s] = vals[p * n_s + s];
}

unsigned nblocks(long n) { return (unsigned)((n + 255) / 256); }

int fit_composite(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo, const double *hi,
                  int nr, double hi_r, long n, const double *pts, const double *vals, double ridge,
                  std::vector<double> &coef, cudaStream_t st)
{
    const int n_s = det->n_s, ncr = nr + 3, ncxy = (n_int[0] + 3) * (n_int[1] + 3);
    SBuf cp, cv, d_cr, d_sxy, res;
    SC_TRY(smalloc<double>(cp, (size_t)n, "column points"));
    SC_TRY(smalloc<double>(cv, (size_t)n, "column values"));
    SC_TRY(smalloc<double>(d_cr, (size_t)n_s * ncr, "axial coefficients"));
    SC_TRY(smalloc<double>(d_sxy, (size_t)2 * n_s, "sensor positions"));
    SC_TRY(smalloc<double>(res, (size_t)n * n_s, "residuals"));
    std::vector<double> cr((size_t)n_s * ncr), cxy((size_t)n_s * ncxy);
    const int nr1[1] = {nr};
    const double lo1[1] = {0.0}, hi1[1] = {hi_r};
    for (int i = 0; i < n_s; ++i) {
        scheme_column<<<nblocks(n), 256, 0, st>>>(pts, n, 2, det->xy[2 * i], det->xy[2 * i + 1], 0, vals, n_s, i,
                                                  (double *)cp.p, (double *)cv.p);
        ANTS_CUDA_TRY(cudaGetLastError(), "composite column launch");
        count_launch();
        SC_TRY(lrf_fit_samples(ctx, 1, nr1, lo1, hi1, n, (const double *)cp.p, 1, (const double *)cv.p, ridge,
                               cr.data() + (size_t)i * ncr, nullptr, st));
    }
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_cr.p, cr.data(), cr.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                  "composite: upload axial part");
    ANTS_CUDA_TRY(cudaMemcpyAsync(d_sxy.p, det->xy.data(), 2 * n_s * sizeof(double), cudaMemcpyHostToDevice, st),
                  "composite: upload sensors");
    composite_residual<<<nblocks(n * n_s), 256, 0, st>>>(pts, n, (const double *)d_sxy.p, vals, n_s,
                                                         (const double *)d_cr.p, nr, hi_r, (double *)res.p);
    ANTS_CUDA_TRY(cudaGetLastError(), "composite residual launch");
    count_launch();
    SC_TRY(lrf_fit_samples(ctx, 2, n_int, lo, hi, n, pts, n_s, (const double *)res.p, ridge, cxy.data(), nullptr,
                           st));
    coef.assign((size_t)n_s * (ncr + ncxy), 0.0);
    for (int i = 0; i < n_s; ++i) {
        std::copy(cr.begin() + (size_t)i * ncr, cr.begin() + (size_t)(i + 1) * ncr,
                  coef.begin() + (size_t)i * (ncr + ncxy));
        std::copy(cxy.begin() + (size_t)i * ncxy, cxy.begin() + (size_t)(i + 1) * ncxy,
                  coef.begin() + (size_t)i * (ncr + ncxy) + ncr);
    }
    return ANTS_OK;
}

int fit_axial_z(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo, const double *hi,
                long n, const double *pts, const double *vals, double ridge, std::vector<double> &coef,
                cudaStream_t st)
{
    const int n_s = det->n_s, nc = (n_int[0] + 3) * (n_int[1] + 3);
    SBuf cp, cv;
    SC_TRY(smalloc<double>(cp, (size_t)2 * n, "column points"));
    SC_TRY(smalloc<double>(cv, (size_t)n, "column values"));
    coef.assign((size_t)n_s * nc, 0.0);
    for (int i = 0; i < n_s; ++i) {
        scheme_column<<<nblocks(n), 256, 0, st>>>(pts, n, 3, det->xy[2 * i], det->xy[2 * i + 1], 1, vals, n_s, i,
                                                  (double *)cp.p, (double *)cv.p);
        ANTS_CUDA_TRY(cudaGetLastError(), "axial+z column launch");
        count_launch();
        SC_TRY(lrf_fit_samples(ctx, 2, n_int, lo, hi, n, (const double *)cp.p, 1, (const double *)cv.p, ridge,
                               coef.data() + (size_t)i * nc, nullptr, st));
    }
    return ANTS_OK;
}

int fit_sliced(ants_ctx *ctx, const ants_detector *det, const int *n_int, const double *lo, const double *hi, int m,
               long n, const double *pts, const double *vals, double ridge, std::vector<double> &coef,
               cudaStream_t st)
{
    const int n_s = det->n_s, ncxy = (n_int[0] + 3) * (n_int[1] + 3);
    const double dz = (hi[2] - lo[2]) / (double)(m - 1);
    SBuf flag, pos, tmp, tot, gp, gv;
    SC_TRY(smalloc<int>(flag, (size_t)n, "plane flags"));
    SC_TRY(smalloc<int>(pos, (size_t)n, "plane positions"));
    SC_TRY(smalloc<char>(tmp, exclusive_scan_tmp_bytes(n), "scan scratch"));
    SC_TRY(smalloc<int>(tot, 1, "count"));
    SC_TRY(smalloc<double>(gp, (size_t)2 * n, "plane points"));
    SC_TRY(smalloc<double>(gv, (size_t)n * n_s, "plane values"));
    coef.assign((size_t)n_s * m * ncxy, 0.0);
    std::vector<double> cj((size_t)n_s * ncxy);
    for (int j = 0; j < m; ++j) {
        plane_flags<<<nblocks(n), 256, 0, st>>>(pts, n, lo[2], dz, m, j, (int *)flag.p);
        count_launch();
        SC_TRY(exclusive_scan((const int *)flag.p, (int *)pos.p, n, (int *)tot.p, tmp.p, st));
        gather_plane<<<nblocks(n), 256, 0, st>>>(pts, vals, n, n_s, (const int *)flag.p, (const int *)pos.p,
                                                 (double *)gp.p, (double *)gv.p);
        count_launch();
        ANTS_CUDA_TRY(cudaGetLastError(), "sliced gather launch");
        int k = 0;
        ANTS_CUDA_TRY(cudaMemcpyAsync(&k, tot.p, sizeof(int), cudaMemcpyDeviceToHost, st), "sliced: count");
        ANTS_CUDA_TRY(cudaStreamSynchronize(st), "sliced: gather");
        if (k == 0) return fail(ANTS_E_LRF, "sliced fit: no sample near plane %d", j);
        SC_TRY(lrf_fit_samples(ctx, 2, n_int, lo, hi, k, (const double *)gp.p, n_s, (const double *)gv.p, ridge,
                               cj.data(), nullptr, st));
        for (int i = 0; i < n_s; ++i)
            std::copy(cj.begin() + (size_t)i * ncxy, cj.begin() + (size_t)(i + 1) * ncxy,
                      coef.begin() + ((size_t)i * m + j) * ncxy);
    }
    return ANTS_OK;
}

}  // namespace

}  // namespace ants

extern "C" ANTS_API int ants_lrf_fit_scheme(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                            const double *lo, const double *hi, int n_int_r, double hi_r,
                                            int n_planes, long n_pts, const double *pts_host,
                                            const double *vals_host, double ridge, ants_lrf **out)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_lrf_fit_scheme");
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: out is NULL");
    *out = nullptr;
    if (!ctx || !det || !n_int || !lo || !hi || (n_pts > 0 && (!pts_host || !vals_host)))
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: NULL argument");
    if (type != ANTS_LRF_COMPOSITE && type != ANTS_LRF_AXIAL_Z && type != ANTS_LRF_SLICED)
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: type %d is not a composite, axial+z or sliced LRF", type);
    if (n_pts < 0 || n_pts > (1L << 30) || (long)det->n_s * n_pts > (1L << 31))
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: n_pts out of range");
    if (!(ridge >= 0.0)) return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: ridge must be >= 0");
    if (n_pts == 0) return fail(ANTS_E_LRF, "ants_lrf_fit_scheme: no samples");
    for (int a = 0; a < 2; ++a)
        if (n_int[a] < 1 || n_int[a] > 256 || !(lo[a] < hi[a]))
            return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: axis %d needs 1 <= n_int <= 256, lo < hi", a);
    if (type == ANTS_LRF_AXIAL_Z && lo[0] != 0.0)
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: an axial+z LRF starts at r = 0");
    if (type == ANTS_LRF_COMPOSITE && (n_int_r < 1 || n_int_r > 256 || !(hi_r > 0.0)))
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: a composite LRF needs 1 <= n_int_r <= 256, hi_r > 0");
    if (type == ANTS_LRF_SLICED && (n_planes < 2 || n_planes > 64 || !(lo[2] < hi[2])))
        return fail(ANTS_E_ARG, "ants_lrf_fit_scheme: a sliced LRF needs 2..64 planes and lo[2] < hi[2]");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = ctx->stream[0];
    const int d = type == ANTS_LRF_COMPOSITE ? 2 : 3, n_s = det->n_s;
    SBuf d_pts, d_vals;
    SC_TRY(smalloc<double>(d_pts, (size_t)n_pts * d, "points"));
    SC_TRY(smalloc<double>(d_vals, (size_t)n_pts * n_s, "values"));
    if (n_pts > 0) {
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_pts.p, pts_host, (size_t)n_pts * d * sizeof(double), cudaMemcpyHostToDevice,
                                      st), "fit_scheme: upload points");
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_vals.p, vals_host, (size_t)n_pts * n_s * sizeof(double),
                                      cudaMemcpyHostToDevice, st), "fit_scheme: upload values");
    }
    std::vector<double> coef;
    const double *P = (const double *)d_pts.p, *V = (const double *)d_vals.p;
    int rc = type == ANTS_LRF_COMPOSITE ? fit_composite(ctx, det, n_int, lo, hi, n_int_r, hi_r, n_pts, P, V, ridge,
                                                        coef, st)
             : type == ANTS_LRF_AXIAL_Z ? fit_axial_z(ctx, det, n_int, lo, hi, n_pts, P, V, ridge, coef, st)
                                        : fit_sliced(ctx, det, n_int, lo, hi, n_planes, n_pts, P, V, ridge, coef, st);
    if (rc != ANTS_OK) return rc;
    return lrf_create_impl(ctx, det, type, n_int, lo, hi, 0, coef.data(), nullptr, n_int_r, hi_r, n_planes, out);
}
