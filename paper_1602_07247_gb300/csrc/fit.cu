// FP64 least-squares fit of B-spline LRFs (Sec. 6: LRFs are computed from
// datasets of positions and signals), on the GPU.
//
// Minimise sum_p (f(p) - v_p)^2 for a tensor-product cubic B-spline f with
// n_coef coefficients, for n_sets value columns at once:
//   (B^T B + lambda I) c = B^T v,   solved by a square-root-free Cholesky
//   factorisation (A = L D L^T) of the banded normal matrix.
// Every sum is taken in a fixed order, so the result is bitwise
// reproducible:
//   1. per sample: knot span and the 4 weights per axis, cell id
//   2. samples bucketed per cell (counting sort; each bucket then sorted by
//      sample index)
//   3. A(u, v) = sum over the cells both basis functions cover, over the
//      samples of each cell, of B_u B_v  (one thread per band entry)
//      r(u, s) = sum over u's cells and their samples of B_u v_s
//   4. right-looking elimination on the band, one launch per column
//   5. forward / diagonal / backward substitution, one block per value set
#include <cmath>

#include "internal.cuh"

namespace ants {

namespace {

struct FitGrid {
    int dims;
    int n[3];        // intervals per axis (1 for unused axes)
    int nb[3];       // basis functions per axis: n + 3 (1 for unused axes)
    double lo[3], hi[3], h[3];
    int n_coef, n_cells, bw;
};

__device__ __forceinline__ void seg_weights(double t, double w[4])
{
    const double k = 1.0 / 6.0;
    double t2 = t * t, t3 = t2 * t, u = 1.0 - t;
    w[0] = k * u * u * u;
    w[1] = k * (3.0 * t3 - 6.0 * t2 + 4.0);
    w[2] = k * (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0);
    w[3] = k * t3;
}

__global__ void fit_point_basis(FitGrid g, const double *pts, long n_pts, int *cell, int *span,
                                double *wts)
{
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pts) return;
    int c = 0, mult = 1;
    bool ok = true;
    for (int a = 0; a < 3; ++a) {
        double w[4] = {1.0, 0.0, 0.0, 0.0};
        int j = 0;
        if (a < g.dims) {
            double x = pts[p * g.dims + a];
            ok = ok && x >= g.lo[a] && x <= g.hi[a];
            double u = (x - g.lo[a]) / g.h[a];
            j = (int)floor(u);
            j = j < 0 ? 0 : (j > g.n[a] - 1 ? g.n[a] - 1 : j);
            if (ok) seg_weights(u - (double)j, w);
        }
        span[p * 3 + a] = j;
        for (int q = 0; q < 4; ++q) wts[(p * 3 + a) * 4 + q] = w[q];
        c += j * mult;
        mult *= g.n[a];
    }
    cell[p] = ok ? c : -1;
}

__global__ void fit_count(const int *cell, long n_pts, int *count)
{
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pts && cell[p] >= 0) atomicAdd(&count[cell[p]], 1);
}

// exclusive scan of n_cells counts (small: one block, serial chunks)
__global__ void fit_scan(const int *count, int n_cells, int *offset)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int acc = 0;
        for (int c = 0; c < n_cells; ++c) {
            offset[c] = acc;
            acc += count[c];
        }
        offset[n_cells] = acc;
    }
}

__global__ void fit_scatter(const int *cell, long n_pts, const int *offset, int *cursor, int *list)
{
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pts && cell[p] >= 0) {
        int pos = atomicAdd(&cursor[cell[p]], 1);
        list[offset[cell[p]] + pos] = (int)p;
    }
}

// order every bucket by sample index (insertion sort; buckets are small)
__global__ void fit_sort_buckets(const int *offset, int n_cells, int *list)
{
    int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n_cells) return;
    int b = offset[c], e = offset[c + 1];
    for (int i = b + 1; i < e; ++i) {
        int v = list[i], k = i - 1;
        while (k >= b && list[k] > v) {
            list[k + 1] = list[k];
            --k;
        }
        list[k + 1] = v;
    }
}

__device__ __forceinline__ void decode(const FitGrid &g, int u, int q[3])
{
    q[0] = u % g.nb[0];
    q[1] = (u / g.nb[0]) % g.nb[1];
    q[2] = u / (g.nb[0] * g.nb[1]);
}

// B_u at sample p (given u's per-axis index q)
__device__ __forceinline__ double basis_at(const int *span, const double *wts, long p, const int q[3])
{
    double b = 1.0;
    for (int a = 0; a < 3; ++a) {
        int r = q[a] - span[p * 3 + a];
        if (r < 0 || r > 3) return 0.0;
        b *= wts[(p * 3 + a) * 4 + r];
    }
    return b;
}

// band storage of the lower triangle: A(i, k), 0 <= i - k <= bw, at i*(bw+1) + (i-k)
__global__ void fit_assemble_band(FitGrid g, const int *offset, const int *list, const int *span,
                                  const double *wts, double lambda, double *band)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)g.n_coef * (g.bw + 1);
    if (t >= total) return;
    int u = (int)(t / (g.bw + 1)), d = (int)(t % (g.bw + 1)), v = u - d;
    double acc = 0.0;
    if (v >= 0) {
        int qu[3], qv[3], lo[3], hi[3];
        decode(g, u, qu);
        decode(g, v, qv);
        bool near = true;
        for (int a = 0; a < 3; ++a) {
            // cells (spans) whose 4 basis functions include both indices
            lo[a] = max(max(qu[a], qv[a]) - 3, 0);
            hi[a] = min(min(qu[a], qv[a]), g.n[a] - 1);
            near = near && lo[a] <= hi[a];
        }
        if (near) {
            for (int cz = lo[2]; cz <= hi[2]; ++cz)
                for (int cy = lo[1]; cy <= hi[1]; ++cy)
                    for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                        int c = (cz * g.n[1] + cy) * g.n[0] + cx;
                        for (int k = offset[c]; k < offset[c + 1]; ++k) {
                            long p = list[k];
                            acc += basis_at(span, wts, p, qu) * basis_at(span, wts, p, qv);
                        }
                    }
        }
        if (d == 0) acc += lambda;
    }
    band[t] = acc;
}

// r[u][s] = sum over u's cells and their samples of B_u(p) v[p][s]
__global__ void fit_rhs(FitGrid g, int n_sets, const int *offset, const int *list, const int *span,
                        const double *wts, const double *vals, double *rhs)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)g.n_coef * n_sets;
    if (t >= total) return;
    int u = (int)(t / n_sets), s = (int)(t % n_sets);
    int q[3], lo[3], hi[3];
    decode(g, u, q);
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(q[a] - 3, 0);
        hi[a] = min(q[a], g.n[a] - 1);
    }
    double acc = 0.0;
    for (int cz = lo[2]; cz <= hi[2]; ++cz)
        for (int cy = lo[1]; cy <= hi[1]; ++cy)
            for (int cx = lo[0]; cx <= hi[0]; ++cx) {
                int c = (cz * g.n[1] + cy) * g.n[0] + cx;
                for (int k = offset[c]; k < offset[c + 1]; ++k) {
                    long p = list[k];
                    acc += basis_at(span, wts, p, q) * vals[p * n_sets + s];
                }
            }
    rhs[t] = acc;
}

// one elimination step on column j: A(i,k) -= A(i,j) A(k,j) / A(j,j) for
// j < k <= i <= j + bw.  Column j itself is kept (it holds L D).
__global__ void fit_elim_step(int n, int bw, int j, double *band, int *not_pd)
{
    const int W = bw + 1;
    double djj = band[(long)j * W];
    if (blockIdx.x == 0 && threadIdx.x == 0 && !(djj > 0.0)) *not_pd = 1;
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int di = (int)(t / bw) + 1, dk = (int)(t % bw) + 1;  // i = j + di, k = j + dk
    if (di > bw || dk > di) return;
    int i = j + di, k = j + dk;
    if (i >= n) return;
    double aij = band[(long)i * W + di];
    double akj = band[(long)k * W + dk];
    if (aij == 0.0 || akj == 0.0) return;
    band[(long)i * W + (i - k)] -= aij * akj / djj;
}

// solve L D L^T x = r for value set s; L(i,k) = A(i,k)/A(k,k), D = diag(A)
__global__ void fit_solve(int n, int bw, int n_sets, const double *band, const double *rhs, double *x)
{
    extern __shared__ double red[];
    const int s = blockIdx.x, W = bw + 1;
    double *xs = x + (long)s * n;
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = rhs[(long)i * n_sets + s];
    __syncthreads();
    // forward: y_i = r_i - sum_{k<i} L(i,k) y_k
    for (int i = 0; i < n; ++i) {
        double part = 0.0;
        for (int d = 1 + threadIdx.x; d <= bw && d <= i; d += blockDim.x) {
            int k = i - d;
            part += band[(long)i * W + d] / band[(long)k * W] * xs[k];
        }
        red[threadIdx.x] = part;
        __syncthreads();
        for (int o = blockDim.x / 2; o; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) xs[i] -= red[0];
        __syncthreads();
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] /= band[(long)i * W];
    __syncthreads();
    // backward: x_i = z_i - sum_{k>i} L(k,i) x_k
    for (int i = n - 1; i >= 0; --i) {
        double part = 0.0;
        for (int d = 1 + threadIdx.x; d <= bw && i + d < n; d += blockDim.x) {
            int k = i + d;
            part += band[(long)k * W + d] / band[(long)i * W] * xs[k];
        }
        red[threadIdx.x] = part;
        __syncthreads();
        for (int o = blockDim.x / 2; o; o >>= 1) {
            if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) xs[i] -= red[0];
        __syncthreads();
    }
}

struct DevBuf {
    void *p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

template <class T>
int dalloc(DevBuf &b, size_t count, const char *what)
{
    cudaError_t e = cudaMalloc(&b.p, count * sizeof(T) + 16);
    if (e != cudaSuccess) return fail(ANTS_E_OOM, "ants_lrf_fit: cudaMalloc(%s): %s", what, cudaGetErrorString(e));
    return ANTS_OK;
}

#define FIT_TRY(x)                  \
    do {                            \
        int _rc = (x);              \
        if (_rc != ANTS_OK) return _rc; \
    } while (0)

}  // namespace

// Fit on the device; coef_out[n_sets][n_coef] on the host.
int lrf_fit_device(const ants_ctx *ctx, int dims, const int *n_int, const double *lo, const double *hi,
                   long n_pts, const double *pts_host, int n_sets, const double *vals_host, double ridge,
                   double *coef_out, double *ridge_used)
{
    FitGrid g{};
    g.dims = dims;
    g.n_coef = 1;
    g.n_cells = 1;
    for (int a = 0; a < 3; ++a) {
        bool used = a < dims;
        g.n[a] = used ? n_int[a] : 1;
        g.nb[a] = used ? n_int[a] + 3 : 1;
        g.lo[a] = used ? lo[a] : 0.0;
        g.hi[a] = used ? hi[a] : 1.0;
        g.h[a] = (g.hi[a] - g.lo[a]) / (double)g.n[a];
        g.n_coef *= g.nb[a];
        g.n_cells *= g.n[a];
    }
    // largest flat-index distance between two basis functions sharing a cell
    g.bw = 3 * (1 + (dims > 1 ? g.nb[0] : 0) + (dims > 2 ? g.nb[0] * g.nb[1] : 0));
    if (g.bw > g.n_coef - 1) g.bw = g.n_coef - 1;
    const int nc = g.n_coef, W = g.bw + 1;
    cudaStream_t st = ctx->stream[0];

    DevBuf d_pts, d_vals, d_cell, d_span, d_wts, d_count, d_off, d_cur, d_list, d_band, d_band0, d_rhs, d_x,
        d_flag;
    FIT_TRY(dalloc<double>(d_pts, (size_t)n_pts * dims, "points"));
    FIT_TRY(dalloc<double>(d_vals, (size_t)n_pts * n_sets, "values"));
    FIT_TRY(dalloc<int>(d_cell, (size_t)n_pts, "cells"));
    FIT_TRY(dalloc<int>(d_span, (size_t)n_pts * 3, "spans"));
    FIT_TRY(dalloc<double>(d_wts, (size_t)n_pts * 12, "weights"));
    FIT_TRY(dalloc<int>(d_count, (size_t)g.n_cells, "counts"));
    FIT_TRY(dalloc<int>(d_off, (size_t)g.n_cells + 1, "offsets"));
    FIT_TRY(dalloc<int>(d_cur, (size_t)g.n_cells, "cursors"));
    FIT_TRY(dalloc<int>(d_list, (size_t)n_pts, "buckets"));
    FIT_TRY(dalloc<double>(d_band, (size_t)nc * W, "band"));
    FIT_TRY(dalloc<double>(d_band0, (size_t)nc * W, "band copy"));
    FIT_TRY(dalloc<double>(d_rhs, (size_t)nc * n_sets, "rhs"));
    FIT_TRY(dalloc<double>(d_x, (size_t)nc * n_sets, "solution"));
    FIT_TRY(dalloc<int>(d_flag, 1, "flag"));
    double *pts = (double *)d_pts.p, *vals = (double *)d_vals.p, *wts = (double *)d_wts.p;
    int *cell = (int *)d_cell.p, *span = (int *)d_span.p, *count = (int *)d_count.p, *off = (int *)d_off.p;
    int *cur = (int *)d_cur.p, *list = (int *)d_list.p, *flag = (int *)d_flag.p;
    double *band = (double *)d_band.p, *band0 = (double *)d_band0.p, *rhs = (double *)d_rhs.p, *x = (double *)d_x.p;

    ANTS_CUDA_TRY(cudaMemcpyAsync(pts, pts_host, (size_t)n_pts * dims * sizeof(double), cudaMemcpyHostToDevice, st),
                  "fit: upload points");
    ANTS_CUDA_TRY(cudaMemcpyAsync(vals, vals_host, (size_t)n_pts * n_sets * sizeof(double), cudaMemcpyHostToDevice,
                                  st), "fit: upload values");
    ANTS_CUDA_TRY(cudaMemsetAsync(count, 0, g.n_cells * sizeof(int), st), "fit: memset");
    ANTS_CUDA_TRY(cudaMemsetAsync(cur, 0, g.n_cells * sizeof(int), st), "fit: memset");
    ANTS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "fit: memset");
    const int T = 256;
    unsigned bp = (unsigned)((n_pts + T - 1) / T);
    long launches = 0;
    if (n_pts > 0) {
        fit_point_basis<<<bp, T, 0, st>>>(g, pts, n_pts, cell, span, wts);
        fit_count<<<bp, T, 0, st>>>(cell, n_pts, count);
        launches += 2;
    }
    fit_scan<<<1, 32, 0, st>>>(count, g.n_cells, off);
    ++launches;
    if (n_pts > 0) {
        fit_scatter<<<bp, T, 0, st>>>(cell, n_pts, off, cur, list);
        ++launches;
    }
    fit_sort_buckets<<<(g.n_cells + T - 1) / T, T, 0, st>>>(off, g.n_cells, list);
    fit_assemble_band<<<(unsigned)(((long)nc * W + T - 1) / T), T, 0, st>>>(g, off, list, span, wts, 0.0, band0);
    fit_rhs<<<(unsigned)(((long)nc * n_sets + T - 1) / T), T, 0, st>>>(g, n_sets, off, list, span, wts, vals, rhs);
    launches += 3;
    ANTS_CUDA_TRY(cudaGetLastError(), "fit: assembly launch");
    // trace of B^T B for the ridge fallback
    std::vector<double> band_host((size_t)nc * W);
    ANTS_CUDA_TRY(cudaMemcpyAsync(band_host.data(), band0, band_host.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                  st), "fit: download band");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: assembly");
    double trace = 0.0;
    for (int i = 0; i < nc; ++i) trace += band_host[(size_t)i * W];
    double lam = ridge;
    bool solved = false;
    for (int attempt = 0; attempt < 2 && !solved; ++attempt) {
        for (size_t k = 0; k < band_host.size(); ++k) {
            double v = band_host[k];
            if (k % W == 0) v += lam;
            band_host[k] = v;
        }
        ANTS_CUDA_TRY(cudaMemcpyAsync(band, band_host.data(), band_host.size() * sizeof(double),
                                      cudaMemcpyHostToDevice, st), "fit: upload band");
        for (size_t k = 0; k < band_host.size(); k += W) band_host[k] -= lam;  // back to B^T B
        ANTS_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "fit: memset");
        unsigned be = (unsigned)(((long)g.bw * g.bw + T - 1) / T);
        if (be == 0) be = 1;
        for (int j = 0; j < nc; ++j) fit_elim_step<<<be, T, 0, st>>>(nc, g.bw, j, band, flag);
        launches += nc;
        ANTS_CUDA_TRY(cudaGetLastError(), "fit: elimination launch");
        int h_flag = 0;
        ANTS_CUDA_TRY(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, st), "fit: flag");
        ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: elimination");
        if (!h_flag) {
            solved = true;
            break;
        }
        lam = 1e-10 * trace / (double)nc;
    }
    if (!solved) return fail(ANTS_E_LRF, "ants_lrf_fit: normal matrix not positive definite even with ridge");
    fit_solve<<<n_sets, 128, 128 * sizeof(double), st>>>(nc, g.bw, n_sets, band, rhs, x);
    ++launches;
    ANTS_CUDA_TRY(cudaGetLastError(), "fit: solve launch");
    ANTS_CUDA_TRY(cudaMemcpyAsync(coef_out, x, (size_t)nc * n_sets * sizeof(double), cudaMemcpyDeviceToHost, st),
                  "fit: download coefficients");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: solve");
    count_launch(launches);
    if (ridge_used) *ridge_used = lam;
    return ANTS_OK;
}

}  // namespace ants

extern "C" ANTS_API int ants_lrf_fit(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                     const double *lo, const double *hi, int shared, long n_pts,
                                     const double *pts_host, const double *vals_host, double ridge,
                                     double *ridge_used, ants_lrf **out)
{
    using namespace ants;
    begin_call();
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_fit: out is NULL");
    *out = nullptr;
    if (!ctx || !det || !n_int || !lo || !hi || (n_pts > 0 && (!pts_host || !vals_host)))
        return fail(ANTS_E_ARG, "ants_lrf_fit: NULL argument");
    if (type != ANTS_LRF_RADIAL && type != ANTS_LRF_XY && type != ANTS_LRF_XYZ)
        return fail(ANTS_E_ARG, "ants_lrf_fit: unknown LRF type %d", type);
    if (shared && type != ANTS_LRF_RADIAL)
        return fail(ANTS_E_ARG, "ants_lrf_fit: shared coefficients need a RADIAL LRF");
    if (n_pts < 0 || n_pts > (1L << 30)) return fail(ANTS_E_ARG, "ants_lrf_fit: n_pts out of range");
    if (!(ridge >= 0.0)) return fail(ANTS_E_ARG, "ants_lrf_fit: ridge must be >= 0");
    int dims = lrf_dims(type);
    long nc = 1;
    for (int a = 0; a < dims; ++a) {
        if (n_int[a] < 1 || n_int[a] > 256 || !(lo[a] < hi[a]))
            return fail(ANTS_E_ARG, "ants_lrf_fit: axis %d needs 1 <= n_int <= 256, lo < hi", a);
        nc *= n_int[a] + 3;
    }
    int n_sets = shared ? 1 : det->n_s;
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    std::vector<double> coef((size_t)nc * n_sets);
    double lam = 0.0;
    int rc = lrf_fit_device(ctx, dims, n_int, lo, hi, n_pts, pts_host, n_sets, vals_host, ridge, coef.data(), &lam);
    if (rc != ANTS_OK) return rc;
    long launches = ants_last_launch_count();
    if (ridge_used) *ridge_used = lam;
    rc = ants_lrf_create(ctx, det, type, n_int, lo, hi, shared, coef.data(), nullptr, out);
    count_launch(launches);
    return rc;
}
