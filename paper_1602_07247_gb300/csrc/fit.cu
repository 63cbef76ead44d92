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
//   2. the samples inside the domain sorted by cell with a stable LSD radix
//      sort (8-bit digits; one warp ranks a chunk of 2048 samples in index
//      order), so each cell's samples stay in index order
//   3. each cell's samples cut into work items of a fixed size; per item the
//      local normal matrix of the 4^d basis functions that are non-zero on
//      the cell (upper triangle) and the local right-hand sides, each entry
//      summed by one thread over the item's samples in order
//   4. A(u, v) and r(u, s): over the cells that cover them, in cell order,
//      the entries of their items, in order
//   5. right-looking elimination on the band, one launch per column
//   6. forward / diagonal / backward substitution, one block per value set
#include <algorithm>
#include <cmath>

#include "bspline.cuh"
#include "internal.cuh"

namespace ants {

namespace {

struct FitGrid {
    int dims;
    int n[3];        // intervals per axis (1 for unused axes)
    int nb[3];       // basis functions per axis: n + 3 (1 for unused axes)
    double lo[3], hi[3], h[3];
    int n_coef, n_cells, bw;
    int nloc;        // basis functions non-zero on one cell: 4^dims
};

__global__ void fit_point_basis(FitGrid g, const double *pts, long n_pts, int *cell, int *valid, int *span,
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
            if (ok) bs_weights_f64(u - (double)j, w);
        }
        span[p * 3 + a] = j;
        for (int q = 0; q < 4; ++q) wts[(p * 3 + a) * 4 + q] = w[q];
        c += j * mult;
        mult *= g.n[a];
    }
    cell[p] = ok ? c : -1;
    valid[p] = ok ? 1 : 0;
}

// the samples inside the domain, in index order: key = cell, idx = sample
__global__ void fit_compact(const int *cell, long n_pts, const int *pos, int *key, int *idx)
{
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < n_pts && cell[p] >= 0) {
        key[pos[p]] = cell[p];
        idx[pos[p]] = (int)p;
    }
}

// --- stable LSD radix sort of (key, idx) by key, 8 bits per pass ------------
constexpr int kRadixChunk = 2048;  // keys ranked in order by one warp
constexpr int kRadixWarps = 4;     // chunks per block

// count[d][chunk]: keys of the chunk whose digit is d
__global__ void __launch_bounds__(32 * kRadixWarps) radix_count(const int *key, long n, int shift, long n_chunks,
                                                                 int *count)
{
    __shared__ int s_cnt[kRadixWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long chunk = (long)blockIdx.x * kRadixWarps + w;
    if (chunk >= n_chunks) return;  // warp-uniform; only warp-level synchronisation follows
    for (int d = lane; d < 256; d += 32) s_cnt[w][d] = 0;
    __syncwarp();
    const long b = chunk * kRadixChunk, e = b + kRadixChunk < n ? b + kRadixChunk : n;
    for (long i = b + lane; i < e; i += 32) atomicAdd(&s_cnt[w][(key[i] >> shift) & 255], 1);
    __syncwarp();
    for (int d = lane; d < 256; d += 32) count[(long)d * n_chunks + chunk] = s_cnt[w][d];
}

// offset[d][chunk] = exclusive scan of count in (digit, chunk) order; each
// warp places its chunk's keys in index order (equal digits ranked by lane)
__global__ void __launch_bounds__(32 * kRadixWarps) radix_scatter(const int *key_in, const int *idx_in, long n,
                                                                   int shift, long n_chunks, const int *offset,
                                                                   int *key_out, int *idx_out)
{
    __shared__ int s_cnt[kRadixWarps][256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long chunk = (long)blockIdx.x * kRadixWarps + w;
    if (chunk >= n_chunks) return;  // warp-uniform
    for (int d = lane; d < 256; d += 32) s_cnt[w][d] = offset[(long)d * n_chunks + chunk];
    __syncwarp();
    const long b = chunk * kRadixChunk, e = b + kRadixChunk < n ? b + kRadixChunk : n;
    for (long i0 = b; i0 < e; i0 += 32) {
        const long i = i0 + lane;
        const bool ok = i < e;
        const int k = ok ? key_in[i] : 0;
        const int d = ok ? (k >> shift) & 255 : 256 + lane;  // idle lanes match only themselves
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int base = ok ? s_cnt[w][d] : 0;
        __syncwarp();
        if (ok) {
            const int pos = base + __popc(peers & ((1u << lane) - 1u));
            key_out[pos] = k;
            idx_out[pos] = idx_in[i];
            if ((peers >> lane) == 1u) s_cnt[w][d] = base + __popc(peers);  // the highest lane of the digit
        }
        __syncwarp();
    }
}

// offset[c] = first sorted position whose cell is >= c, c = 0..n_cells
__global__ void fit_cell_offsets(const int *key, long n, int n_cells, int *offset)
{
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > n_cells) return;
    long lo = 0, hi = n;
    while (lo < hi) {
        long mid = (lo + hi) >> 1;
        if (key[mid] < c) lo = mid + 1;
        else hi = mid;
    }
    offset[c] = (int)lo;
}

__global__ void fit_items_per_cell(const int *offset, int n_cells, int per_item, int *items)
{
    long c = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n_cells) items[c] = (offset[c + 1] - offset[c] + per_item - 1) / per_item;
}

// --- per-item local normal matrices and right-hand sides ---------------------
constexpr int kPartThreads = 128;
constexpr int kPartR = 8;     // outputs per thread per pass
constexpr int kPartTile = 32; // samples staged per round

// index of (a, b), a <= b, in the row-major upper triangle of an n x n matrix
__device__ __forceinline__ int tri_index(int a, int b, int n) { return a * n - a * (a - 1) / 2 + (b - a); }

// partial[item][o]: o < n_mat the local matrix entry (a, b) of tri_index;
// o = n_mat + l * n_sets + s the local right-hand side (l, s)
__global__ void __launch_bounds__(kPartThreads) fit_cell_partials(FitGrid g, int n_sets, int per_item,
                                                                   const int *offset, const int *item_off,
                                                                   const int *idx, const double *wts,
                                                                   const double *vals, double *partial)
{
    __shared__ double s_b[kPartTile][64];
    __shared__ long s_p[kPartTile];
    const long item = blockIdx.x;
    // the cell holding this item: the last cell whose first item is <= item
    int lo = 0, hi = g.n_cells - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo;
    const long k0 = offset[c] + (item - item_off[c]) * (long)per_item;
    const long kend = offset[c + 1] < k0 + per_item ? (long)offset[c + 1] : k0 + per_item;
    const int nloc = g.nloc, n_mat = nloc * (nloc + 1) / 2, n_out = n_mat + nloc * n_sets;
    double *out = partial + item * (long)n_out;
    for (int pass = 0; pass < n_out; pass += kPartThreads * kPartR) {
        int la[kPartR], lb[kPartR];  // lb < 0: right-hand side of set -1 - lb
        double acc[kPartR];
#pragma unroll
        for (int r = 0; r < kPartR; ++r) {
            const int o = pass + (int)threadIdx.x + r * kPartThreads;
            acc[r] = 0.0;
            la[r] = 0;
            lb[r] = 0;
            if (o < n_mat) {
                int a = 0, rem = o;
                while (rem >= nloc - a) {
                    rem -= nloc - a;
                    ++a;
                }
                la[r] = a;
                lb[r] = a + rem;
            } else if (o < n_out) {
                la[r] = (o - n_mat) / n_sets;
                lb[r] = -1 - (o - n_mat) % n_sets;
            }
        }
        for (long t0 = k0; t0 < kend; t0 += kPartTile) {
            const int nt = kend - t0 < kPartTile ? (int)(kend - t0) : kPartTile;
            __syncthreads();  // the previous tile is consumed
            for (int q = threadIdx.x; q < nt * nloc; q += kPartThreads) {
                const int ts = q / nloc, l = q - ts * nloc;
                const long p = idx[t0 + ts];
                s_b[ts][l] = wts[(p * 3 + 0) * 4 + (l & 3)] * wts[(p * 3 + 1) * 4 + ((l >> 2) & 3)] *
                             wts[(p * 3 + 2) * 4 + (l >> 4)];
                if (l == 0) s_p[ts] = p;
            }
            __syncthreads();
            for (int ts = 0; ts < nt; ++ts) {
#pragma unroll
                for (int r = 0; r < kPartR; ++r) {
                    const int o = pass + (int)threadIdx.x + r * kPartThreads;
                    if (o < n_out) {
                        const double bb = lb[r] >= 0 ? s_b[ts][lb[r]] : vals[s_p[ts] * n_sets + (-1 - lb[r])];
                        acc[r] += s_b[ts][la[r]] * bb;
                    }
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kPartR; ++r) {
            const int o = pass + (int)threadIdx.x + r * kPartThreads;
            if (o < n_out) out[o] = acc[r];
        }
    }
}

__device__ __forceinline__ void decode(const FitGrid &g, int u, int q[3])
{
    q[0] = u % g.nb[0];
    q[1] = (u / g.nb[0]) % g.nb[1];
    q[2] = u / (g.nb[0] * g.nb[1]);
}

// local index of basis u (per-axis index q) on the cell with spans (cx, cy, cz)
__device__ __forceinline__ int local_index(const int q[3], int cx, int cy, int cz)
{
    return (q[0] - cx) + 4 * ((q[1] - cy) + 4 * (q[2] - cz));
}

// band storage of the lower triangle: A(i, k), 0 <= i - k <= bw, at i*(bw+1) + (i-k)
__global__ void fit_band_from_partials(FitGrid g, int n_sets, const int *item_off, const double *partial,
                                       double *band)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)g.n_coef * (g.bw + 1);
    if (t >= total) return;
    int u = (int)(t / (g.bw + 1)), d = (int)(t % (g.bw + 1)), v = u - d;
    const int n_out = g.nloc * (g.nloc + 1) / 2 + g.nloc * n_sets;
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
                        const int c = (cz * g.n[1] + cy) * g.n[0] + cx;
                        const int lu = local_index(qu, cx, cy, cz), lv = local_index(qv, cx, cy, cz);
                        const int o = tri_index(min(lu, lv), max(lu, lv), g.nloc);
                        for (int it = item_off[c]; it < item_off[c + 1]; ++it) acc += partial[(long)it * n_out + o];
                    }
        }
    }
    band[t] = acc;
}

// r[u][s] = sum over u's cells and their items of the local right-hand side
__global__ void fit_rhs_from_partials(FitGrid g, int n_sets, const int *item_off, const double *partial,
                                      double *rhs)
{
    long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)g.n_coef * n_sets;
    if (t >= total) return;
    int u = (int)(t / n_sets), s = (int)(t % n_sets);
    const int n_mat = g.nloc * (g.nloc + 1) / 2, n_out = n_mat + g.nloc * n_sets;
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
                const int c = (cz * g.n[1] + cy) * g.n[0] + cx;
                const int o = n_mat + local_index(q, cx, cy, cz) * n_sets + s;
                for (int it = item_off[c]; it < item_off[c + 1]; ++it) acc += partial[(long)it * n_out + o];
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

// Fit on the device from device-resident samples: pts [n_pts][dims] and
// vals [n_pts][n_sets] FP64; coef_out[n_sets][n_coef] on the host.
int lrf_fit_samples(const ants_ctx *ctx, int dims, const int *n_int, const double *lo, const double *hi,
                    long n_pts, const double *pts, int n_sets, const double *vals, double ridge, double *coef_out,
                    double *ridge_used, cudaStream_t st)
{
    FitGrid g{};
    g.dims = dims;
    g.n_coef = 1;
    g.n_cells = 1;
    g.nloc = 1;
    for (int a = 0; a < 3; ++a) {
        bool used = a < dims;
        g.n[a] = used ? n_int[a] : 1;
        g.nb[a] = used ? n_int[a] + 3 : 1;
        g.lo[a] = used ? lo[a] : 0.0;
        g.hi[a] = used ? hi[a] : 1.0;
        g.h[a] = (g.hi[a] - g.lo[a]) / (double)g.n[a];
        g.n_coef *= g.nb[a];
        g.n_cells *= g.n[a];
        if (used) g.nloc *= 4;
    }
    // largest flat-index distance between two basis functions sharing a cell
    g.bw = 3 * (1 + (dims > 1 ? g.nb[0] : 0) + (dims > 2 ? g.nb[0] * g.nb[1] : 0));
    if (g.bw > g.n_coef - 1) g.bw = g.n_coef - 1;
    const int nc = g.n_coef, W = g.bw + 1;
    const int n_mat = g.nloc * (g.nloc + 1) / 2;
    const long n_out = n_mat + (long)g.nloc * n_sets;
    const int per_item = n_out <= 64 ? 1024 : 2048;
    const long n_chunks = (n_pts + kRadixChunk - 1) / kRadixChunk;
    int bits = 0;
    while ((1L << bits) < (long)g.n_cells) ++bits;
    const int passes = (bits + 7) / 8;
    const long n_scan = std::max({n_pts, 256L * n_chunks, (long)g.n_cells});

    DevBuf d_cell, d_valid, d_pos, d_span, d_wts, d_key0, d_idx0, d_key1, d_idx1, d_count, d_off, d_items, d_itoff,
        d_tmp, d_tot, d_band, d_band0, d_rhs, d_x, d_flag, d_part;
    FIT_TRY(dalloc<int>(d_cell, (size_t)n_pts, "cells"));
    FIT_TRY(dalloc<int>(d_valid, (size_t)n_pts, "flags"));
    FIT_TRY(dalloc<int>(d_pos, (size_t)n_pts, "positions"));
    FIT_TRY(dalloc<int>(d_span, (size_t)n_pts * 3, "spans"));
    FIT_TRY(dalloc<double>(d_wts, (size_t)n_pts * 12, "weights"));
    FIT_TRY(dalloc<int>(d_key0, (size_t)n_pts, "keys"));
    FIT_TRY(dalloc<int>(d_idx0, (size_t)n_pts, "indices"));
    FIT_TRY(dalloc<int>(d_key1, (size_t)n_pts, "keys"));
    FIT_TRY(dalloc<int>(d_idx1, (size_t)n_pts, "indices"));
    FIT_TRY(dalloc<int>(d_count, (size_t)256 * (n_chunks > 0 ? n_chunks : 1), "digit counts"));
    FIT_TRY(dalloc<int>(d_off, (size_t)g.n_cells + 1, "cell offsets"));
    FIT_TRY(dalloc<int>(d_items, (size_t)g.n_cells, "items"));
    FIT_TRY(dalloc<int>(d_itoff, (size_t)g.n_cells + 1, "item offsets"));
    FIT_TRY(dalloc<char>(d_tmp, exclusive_scan_tmp_bytes(n_scan), "scan scratch"));
    FIT_TRY(dalloc<int>(d_tot, 1, "total"));
    FIT_TRY(dalloc<double>(d_band, (size_t)nc * W, "band"));
    FIT_TRY(dalloc<double>(d_band0, (size_t)nc * W, "band copy"));
    FIT_TRY(dalloc<double>(d_rhs, (size_t)nc * n_sets, "rhs"));
    FIT_TRY(dalloc<double>(d_x, (size_t)nc * n_sets, "solution"));
    FIT_TRY(dalloc<int>(d_flag, 1, "flag"));
    int *cell = (int *)d_cell.p, *valid = (int *)d_valid.p, *pos = (int *)d_pos.p, *span = (int *)d_span.p;
    int *key = (int *)d_key0.p, *idx = (int *)d_idx0.p, *key2 = (int *)d_key1.p, *idx2 = (int *)d_idx1.p;
    int *count = (int *)d_count.p, *off = (int *)d_off.p, *items = (int *)d_items.p, *itoff = (int *)d_itoff.p;
    int *tot = (int *)d_tot.p, *flag = (int *)d_flag.p;
    double *wts = (double *)d_wts.p, *band = (double *)d_band.p, *band0 = (double *)d_band0.p;
    double *rhs = (double *)d_rhs.p, *x = (double *)d_x.p;

    const int T = 256;
    long launches = 0;
    int n_valid = 0;
    if (n_pts > 0) {
        unsigned bp = (unsigned)((n_pts + T - 1) / T);
        fit_point_basis<<<bp, T, 0, st>>>(g, pts, n_pts, cell, valid, span, wts);
        ++launches;
        FIT_TRY(exclusive_scan(valid, pos, n_pts, tot, d_tmp.p, st));
        fit_compact<<<bp, T, 0, st>>>(cell, n_pts, pos, key, idx);
        ++launches;
        ANTS_CUDA_TRY(cudaMemcpyAsync(&n_valid, tot, sizeof(int), cudaMemcpyDeviceToHost, st), "fit: count");
        ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: basis");
    }
    const long nv_chunks = ((long)n_valid + kRadixChunk - 1) / kRadixChunk;
    const unsigned rb = (unsigned)((nv_chunks + kRadixWarps - 1) / kRadixWarps);
    for (int pass = 0; pass < passes && n_valid > 1; ++pass) {
        radix_count<<<rb, 32 * kRadixWarps, 0, st>>>(key, n_valid, 8 * pass, nv_chunks, count);
        FIT_TRY(exclusive_scan(count, count, 256 * nv_chunks, nullptr, d_tmp.p, st));
        radix_scatter<<<rb, 32 * kRadixWarps, 0, st>>>(key, idx, n_valid, 8 * pass, nv_chunks, count, key2, idx2);
        launches += 2;
        std::swap(key, key2);
        std::swap(idx, idx2);
    }
    const unsigned bcell = (unsigned)((g.n_cells + 1 + T - 1) / T);
    fit_cell_offsets<<<bcell, T, 0, st>>>(key, n_valid, g.n_cells, off);
    fit_items_per_cell<<<bcell, T, 0, st>>>(off, g.n_cells, per_item, items);
    launches += 2;
    FIT_TRY(exclusive_scan(items, itoff, g.n_cells, itoff + g.n_cells, d_tmp.p, st));
    int n_items = 0;
    ANTS_CUDA_TRY(cudaMemcpyAsync(&n_items, itoff + g.n_cells, sizeof(int), cudaMemcpyDeviceToHost, st),
                  "fit: items");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: sort");
    FIT_TRY(dalloc<double>(d_part, (size_t)(n_items > 0 ? n_items : 1) * n_out, "partial sums"));
    double *part = (double *)d_part.p;
    if (n_items > 0) {
        fit_cell_partials<<<(unsigned)n_items, kPartThreads, 0, st>>>(g, n_sets, per_item, off, itoff, idx, wts, vals,
                                                                       part);
        ++launches;
    }
    fit_band_from_partials<<<(unsigned)(((long)nc * W + T - 1) / T), T, 0, st>>>(g, n_sets, itoff, part, band0);
    fit_rhs_from_partials<<<(unsigned)(((long)nc * n_sets + T - 1) / T), T, 0, st>>>(g, n_sets, itoff, part, rhs);
    launches += 2;
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
    cudaStream_t st = ctx->stream[0];
    DevBuf d_pts, d_vals;
    FIT_TRY(dalloc<double>(d_pts, (size_t)n_pts * dims, "points"));
    FIT_TRY(dalloc<double>(d_vals, (size_t)n_pts * n_sets, "values"));
    if (n_pts > 0) {
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_pts.p, pts_host, (size_t)n_pts * dims * sizeof(double),
                                      cudaMemcpyHostToDevice, st), "fit: upload points");
        ANTS_CUDA_TRY(cudaMemcpyAsync(d_vals.p, vals_host, (size_t)n_pts * n_sets * sizeof(double),
                                      cudaMemcpyHostToDevice, st), "fit: upload values");
    }
    std::vector<double> coef((size_t)nc * n_sets);
    double lam = 0.0;
    int rc = lrf_fit_samples(ctx, dims, n_int, lo, hi, n_pts, (const double *)d_pts.p, n_sets,
                             (const double *)d_vals.p, ridge, coef.data(), &lam, st);
    if (rc != ANTS_OK) return rc;
    long launches = ants_last_launch_count();
    if (ridge_used) *ridge_used = lam;
    rc = ants_lrf_create(ctx, det, type, n_int, lo, hi, shared, coef.data(), nullptr, out);
    count_launch(launches);
    return rc;
}
