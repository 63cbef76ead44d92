// FP64 least-squares fit of B-spline LRFs (Sec. 6: LRFs are computed from
// datasets of positions and signals), on the GPU.
//
// Minimise sum_p (f(p) - v_p)^2 for a tensor-product cubic B-spline f with
// n_coef coefficients, for n_sets value columns at once:
//   (B^T B + lambda I) c = B^T v,   solved by a square-root-free Cholesky
//   factorisation (A = L D L^T) of the banded normal matrix.
// Every sum is taken in a fixed order, so the result is bitwise
// reproducible:
//   1. per sample: its cell (knot span per axis)
//   2. the samples inside the domain sorted by cell with a stable LSD radix
//      sort (8-bit digits; one warp ranks a chunk of 2048 samples in index
//      order), so each cell's samples stay in index order
//   3. each cell's samples cut into work items of a fixed size; per item the
//      local normal matrix of the 4^d basis functions that are non-zero on
//      the cell (upper triangle) and the local right-hand sides, each entry
//      summed by one thread over the item's samples in order (weights and
//      values staged in shared memory tile by tile); for one-dimensional
//      single-set fits each thread sums all entries over its share of the
//      item's samples and a fixed tree adds the threads' sums
//   4. per cell, the sum of its items' entries (8 interleaved lanes, then
//      the lanes in order)
//   5. A(u, v) and r(u, s): over the cells that cover them, in cell order
//   6. right-looking elimination on the band, one launch per column
//   7. forward / diagonal / backward substitution, one block per value set
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
    double lo[3], hi[3], h[3], inv_h[3];
    int n_coef, n_cells, bw;
    int nloc;        // basis functions non-zero on one cell: 4^dims
};

// the span of axis a at coordinate x (clamped) and its local parameter;
// the cell of a sample and its weights both come from here, so they agree
__device__ __forceinline__ int axis_span(const FitGrid &g, int a, double x, double &t)
{
    double u = (x - g.lo[a]) * g.inv_h[a];
    int j = (int)floor(u);
    j = j < 0 ? 0 : (j > g.n[a] - 1 ? g.n[a] - 1 : j);
    t = u - (double)j;
    return j;
}

__global__ void fit_point_cells(FitGrid g, const double *pts, long n_pts, int *cell, int *valid)
{
    long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pts) return;
    int c = 0, mult = 1;
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (a < g.dims) {
            double x = pts[p * g.dims + a], t;
            ok = ok && x >= g.lo[a] && x <= g.hi[a];
            c += axis_span(g, a, x, t) * mult;
            mult *= g.n[a];
        }
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
constexpr int kPartR = 8;           // outputs per thread per pass
constexpr int kPartMaxTile = 32;    // samples staged per round
constexpr int kPartSmem = 40 * 1024;  // dynamic; plus 4160 B static, under the 48 KB default

// samples per staged tile for nloc local functions and n_sets values
__host__ __device__ inline int part_tile(int nloc, int n_sets)
{
    const int per = 8 * (12 + nloc + n_sets) + 8;
    const int t = kPartSmem / per;
    return t < 1 ? 1 : (t > kPartMaxTile ? kPartMaxTile : t);
}

// index of (a, b), a <= b, in the row-major upper triangle of an n x n matrix
__device__ __forceinline__ int tri_index(int a, int b, int n) { return a * n - a * (a - 1) / 2 + (b - a); }

// partial[item][o]: o < n_mat the local matrix entry (a, b) of tri_index;
// o = n_mat + l * n_sets + s the local right-hand side (l, s).  Each tile of
// samples is staged in shared memory (weights computed from the points,
// values gathered), so the per-output loops read shared memory only.
// Dynamic shared memory: weights [tile][3][4], local basis values
// [tile][nloc], values [tile][n_sets] (FP64), sample indices [tile].
__global__ void __launch_bounds__(kPartThreads) fit_cell_partials(FitGrid g, int n_sets, int per_item, int tile,
                                                                   const int *offset, const int *item_off,
                                                                   const int *idx, const double *pts,
                                                                   const double *vals, double *partial)
{
    extern __shared__ double smem[];
    __shared__ unsigned short s_tri[64 * 65 / 2];  // (a << 8) | b of each upper-triangle entry
    const int nloc = g.nloc, n_mat = nloc * (nloc + 1) / 2, n_out = n_mat + nloc * n_sets;
    for (int q = threadIdx.x; q < nloc; q += kPartThreads)
        for (int b = q; b < nloc; ++b) s_tri[tri_index(q, b, nloc)] = (unsigned short)((q << 8) | b);
    double *s_w = smem;
    double *s_b = s_w + tile * 12;
    double *s_v = s_b + tile * nloc;
    long *s_p = (long *)(s_v + (size_t)tile * n_sets);
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
    double *out = partial + item * (long)n_out;
    __syncthreads();  // s_tri is complete
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
                la[r] = s_tri[o] >> 8;
                lb[r] = s_tri[o] & 255;
            } else if (o < n_out) {
                la[r] = (o - n_mat) / n_sets;
                lb[r] = -1 - (o - n_mat) % n_sets;
            }
        }
        for (long t0 = k0; t0 < kend; t0 += tile) {
            const int nt = kend - t0 < tile ? (int)(kend - t0) : tile;
            __syncthreads();  // the previous tile is consumed
            for (int q = threadIdx.x; q < nt; q += kPartThreads) s_p[q] = idx[t0 + q];
            __syncthreads();
            for (int ts = threadIdx.x; ts < nt; ts += kPartThreads) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {  // static axis index: the grid stays in registers
                    double w[4] = {1.0, 0.0, 0.0, 0.0};
                    if (a < g.dims) {
                        double t;
                        axis_span(g, a, pts[s_p[ts] * g.dims + a], t);
                        bs_weights_f64(t, w);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) s_w[(ts * 3 + a) * 4 + b] = w[b];
                }
            }
            for (int q = threadIdx.x; q < nt * n_sets; q += kPartThreads) {
                const int ts = q / n_sets, sidx = q - ts * n_sets;
                s_v[q] = vals[s_p[ts] * n_sets + sidx];
            }
            __syncthreads();
            for (int q = threadIdx.x; q < nt * nloc; q += kPartThreads) {
                const int ts = q / nloc, l = q - ts * nloc;
                const double *w = s_w + ts * 12;
                // FP64 is scarce: no products with the unit weights of unused axes
                double b = w[l & 3];
                if (g.dims > 1) b *= w[4 + ((l >> 2) & 3)];
                if (g.dims > 2) b *= w[8 + (l >> 4)];
                s_b[q] = b;
            }
            __syncthreads();
            for (int ts = 0; ts < nt; ++ts) {
#pragma unroll
                for (int r = 0; r < kPartR; ++r) {
                    const int o = pass + (int)threadIdx.x + r * kPartThreads;
                    if (o < n_out) {
                        const double bb = lb[r] >= 0 ? s_b[ts * nloc + lb[r]] : s_v[ts * n_sets + (-1 - lb[r])];
                        acc[r] += s_b[ts * nloc + la[r]] * bb;
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

// The same partial sums for one-dimensional fits of one value set (radial
// profiles: 10 matrix entries and 4 right-hand sides), sample-parallel:
// thread t accumulates all 14 entries over the item's samples t, t + T, ...
// in order, then the threads' sums are added by a fixed tree per entry (an
// FP64 instruction costs the same whatever its active lanes, so every lane
// works).
constexpr int kOut1 = 14;
constexpr int kPer1 = 4096;  // samples per work item

__global__ void __launch_bounds__(kPartThreads) fit_cell_partials_1d(FitGrid g, const int *offset,
                                                                      const int *item_off, const int *idx,
                                                                      const double *pts, const double *vals,
                                                                      double *partial)
{
    __shared__ double s_red[kOut1][kPartThreads];
    const long item = blockIdx.x;
    int lo = 0, hi = g.n_cells - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    const int c = lo;
    const long k0 = offset[c] + (item - item_off[c]) * (long)kPer1;
    const long kend = offset[c + 1] < k0 + kPer1 ? (long)offset[c + 1] : k0 + kPer1;
    double acc[kOut1];
#pragma unroll
    for (int o = 0; o < kOut1; ++o) acc[o] = 0.0;
    for (long k = k0 + threadIdx.x; k < kend; k += kPartThreads) {
        const long p = idx[k];
        double t, w[4];
        axis_span(g, 0, pts[p], t);
        bs_weights_f64(t, w);
        const double v = vals[p];
        int o = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a; b < 4; ++b) acc[o++] += w[a] * w[b];  // o = tri_index(a, b, 4)
#pragma unroll
        for (int a = 0; a < 4; ++a) acc[10 + a] += w[a] * v;
    }
#pragma unroll
    for (int o = 0; o < kOut1; ++o) s_red[o][threadIdx.x] = acc[o];
    __syncthreads();
    for (int half = kPartThreads / 2; half > 0; half >>= 1) {
        for (int q = threadIdx.x; q < kOut1 * half; q += kPartThreads) {
            const int o = q / half, j = q - o * half;
            s_red[o][j] += s_red[o][j + half];
        }
        __syncthreads();
    }
    if (threadIdx.x < kOut1) partial[item * kOut1 + threadIdx.x] = s_red[threadIdx.x][0];
}

// cellsum[c][o] = the sum over cell c's items of partial[item][o]: lane l of
// kRedLanes sums the items l, l + kRedLanes, ... in order, then the lanes
// are added in order
constexpr int kRedOut = 32, kRedLanes = 8;

__global__ void __launch_bounds__(kRedOut * kRedLanes) fit_cell_sums(int n_out, const int *item_off,
                                                                      const double *partial, double *cellsum)
{
    __shared__ double s[kRedLanes][kRedOut];
    const int c = blockIdx.x;
    const int ol = threadIdx.x % kRedOut, lane = threadIdx.x / kRedOut;
    const long o = (long)blockIdx.y * kRedOut + ol;
    double acc = 0.0;
    if (o < n_out)
        for (int it = item_off[c] + lane; it < item_off[c + 1]; it += kRedLanes) acc += partial[(long)it * n_out + o];
    s[lane][ol] = acc;
    __syncthreads();
    if (lane == 0 && o < n_out) {
        double t = s[0][ol];
        for (int l = 1; l < kRedLanes; ++l) t += s[l][ol];
        cellsum[(long)c * n_out + o] = t;
    }
}

__global__ void fit_iota(int n, int *v)
{
    long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) v[i] = (int)i;
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
// vals [n_pts][n_sets] FP64; coef_out[n_sets][n_coef] on the host.  Work
// buffers come from the context's scratch slots 8 and 9 (the call is
// synchronous, so nothing else can be using them when it returns).
int lrf_fit_samples(ants_ctx *ctx, int dims, const int *n_int, const double *lo, const double *hi, long n_pts,
                    const double *pts, int n_sets, const double *vals, double ridge, double *coef_out,
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
        g.inv_h[a] = (double)g.n[a] / (g.hi[a] - g.lo[a]);
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
    const bool one_d = dims == 1 && n_sets == 1;  // n_out == kOut1: the sample-parallel kernel
    const int per_item = one_d ? kPer1 : (n_out <= 64 ? 1024 : 2048);
    const int tile = part_tile(g.nloc, n_sets);
    const long n_chunks = (n_pts + kRadixChunk - 1) / kRadixChunk;
    int bits = 0;
    while ((1L << bits) < (long)g.n_cells) ++bits;
    const int passes = (bits + 7) / 8;
    const long n_scan = std::max({n_pts, 256L * n_chunks, (long)g.n_cells});

    Carve cv;
    const size_t o_cell = cv.take<int>(n_pts), o_valid = cv.take<int>(n_pts), o_pos = cv.take<int>(n_pts);
    const size_t o_key0 = cv.take<int>(n_pts), o_idx0 = cv.take<int>(n_pts);
    const size_t o_key1 = cv.take<int>(n_pts), o_idx1 = cv.take<int>(n_pts);
    const size_t o_count = cv.take<int>(256 * (size_t)(n_chunks > 0 ? n_chunks : 1));
    const size_t o_off = cv.take<int>(g.n_cells + 1), o_items = cv.take<int>(g.n_cells);
    const size_t o_itoff = cv.take<int>(g.n_cells + 1), o_iota = cv.take<int>(g.n_cells + 1);
    const size_t o_tmp = cv.take<char>(exclusive_scan_tmp_bytes(n_scan)), o_tot = cv.take<int>(1);
    const size_t o_band = cv.take<double>((size_t)nc * W), o_band0 = cv.take<double>((size_t)nc * W);
    const size_t o_rhs = cv.take<double>((size_t)nc * n_sets), o_x = cv.take<double>((size_t)nc * n_sets);
    const size_t o_flag = cv.take<int>(1);
    char *base = (char *)ctx_scratch(ctx, 8, cv.off);
    if (!base) return ANTS_E_OOM;
    int *cell = (int *)(base + o_cell), *valid = (int *)(base + o_valid), *pos = (int *)(base + o_pos);
    int *key = (int *)(base + o_key0), *idx = (int *)(base + o_idx0);
    int *key2 = (int *)(base + o_key1), *idx2 = (int *)(base + o_idx1);
    int *count = (int *)(base + o_count), *off = (int *)(base + o_off), *items = (int *)(base + o_items);
    int *itoff = (int *)(base + o_itoff), *iota = (int *)(base + o_iota), *tot = (int *)(base + o_tot);
    int *flag = (int *)(base + o_flag);
    void *tmp = base + o_tmp;
    double *band = (double *)(base + o_band), *band0 = (double *)(base + o_band0);
    double *rhs = (double *)(base + o_rhs), *x = (double *)(base + o_x);

    const int T = 256;
    long launches = 0;
    int n_valid = 0;
    if (n_pts > 0) {
        unsigned bp = (unsigned)((n_pts + T - 1) / T);
        fit_point_cells<<<bp, T, 0, st>>>(g, pts, n_pts, cell, valid);
        ++launches;
        FIT_TRY(exclusive_scan(valid, pos, n_pts, tot, tmp, st));
        fit_compact<<<bp, T, 0, st>>>(cell, n_pts, pos, key, idx);
        ++launches;
        ANTS_CUDA_TRY(cudaMemcpyAsync(&n_valid, tot, sizeof(int), cudaMemcpyDeviceToHost, st), "fit: count");
        ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: cells");
    }
    const long nv_chunks = ((long)n_valid + kRadixChunk - 1) / kRadixChunk;
    const unsigned rb = (unsigned)((nv_chunks + kRadixWarps - 1) / kRadixWarps);
    for (int pass = 0; pass < passes && n_valid > 1; ++pass) {
        radix_count<<<rb, 32 * kRadixWarps, 0, st>>>(key, n_valid, 8 * pass, nv_chunks, count);
        FIT_TRY(exclusive_scan(count, count, 256 * nv_chunks, nullptr, tmp, st));
        radix_scatter<<<rb, 32 * kRadixWarps, 0, st>>>(key, idx, n_valid, 8 * pass, nv_chunks, count, key2, idx2);
        launches += 2;
        std::swap(key, key2);
        std::swap(idx, idx2);
    }
    const unsigned bcell = (unsigned)((g.n_cells + 1 + T - 1) / T);
    fit_cell_offsets<<<bcell, T, 0, st>>>(key, n_valid, g.n_cells, off);
    fit_items_per_cell<<<bcell, T, 0, st>>>(off, g.n_cells, per_item, items);
    launches += 2;
    FIT_TRY(exclusive_scan(items, itoff, g.n_cells, itoff + g.n_cells, tmp, st));
    int n_items = 0;
    ANTS_CUDA_TRY(cudaMemcpyAsync(&n_items, itoff + g.n_cells, sizeof(int), cudaMemcpyDeviceToHost, st),
                  "fit: items");
    ANTS_CUDA_TRY(cudaStreamSynchronize(st), "fit: sort");
    // per-cell sums of the items unless that table would be large (huge
    // grids): then the band sums the items directly
    const bool by_cell = (double)g.n_cells * (double)n_out <= (double)(1L << 27);
    Carve cp;
    const size_t o_part = cp.take<double>((size_t)(n_items > 0 ? n_items : 1) * n_out);
    const size_t o_csum = by_cell ? cp.take<double>((size_t)g.n_cells * n_out) : 0;
    char *pbase = (char *)ctx_scratch(ctx, 9, cp.off);
    if (!pbase) return ANTS_E_OOM;
    double *part = (double *)(pbase + o_part);
    if (n_items > 0 && one_d) {
        fit_cell_partials_1d<<<(unsigned)n_items, kPartThreads, 0, st>>>(g, off, itoff, idx, pts, vals, part);
        ++launches;
    } else if (n_items > 0) {
        const size_t smem = (size_t)tile * (12 + g.nloc + n_sets) * sizeof(double) + (size_t)tile * sizeof(long);
        fit_cell_partials<<<(unsigned)n_items, kPartThreads, smem, st>>>(g, n_sets, per_item, tile, off, itoff, idx,
                                                                         pts, vals, part);
        ++launches;
    }
    const int *sum_off = itoff;
    const double *sums = part;
    if (by_cell) {
        double *csum = (double *)(pbase + o_csum);
        dim3 grid((unsigned)g.n_cells, (unsigned)((n_out + kRedOut - 1) / kRedOut));
        fit_cell_sums<<<grid, kRedOut * kRedLanes, 0, st>>>((int)n_out, itoff, part, csum);
        fit_iota<<<bcell, T, 0, st>>>(g.n_cells, iota);
        launches += 2;
        sum_off = iota;  // one "item" per cell
        sums = csum;
    }
    fit_band_from_partials<<<(unsigned)(((long)nc * W + T - 1) / T), T, 0, st>>>(g, n_sets, sum_off, sums, band0);
    fit_rhs_from_partials<<<(unsigned)(((long)nc * n_sets + T - 1) / T), T, 0, st>>>(g, n_sets, sum_off, sums, rhs);
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

extern "C" ANTS_API int ants_lrf_fit_symmetric(ants_ctx *ctx, const ants_detector *det, const int *n_int,
                                               const double *lo, const double *hi, int n_classes,
                                               const int *class_host, const int *op_host, const double *centre,
                                               long n_pts, const double *pts_host, const double *vals_host,
                                               const double *gain_host, double ridge, ants_lrf **out)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_lrf_fit_symmetric");
    if (!out) return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: out is NULL");
    *out = nullptr;
    if (!ctx || !det || !n_int || !lo || !hi || !class_host || !op_host || !centre ||
        (n_pts > 0 && (!pts_host || !vals_host)))
        return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: NULL argument");
    if (n_pts < 0 || n_pts > (1L << 30) / (det->n_s > 0 ? det->n_s : 1))
        return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: n_pts out of range");
    if (!(ridge >= 0.0)) return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: ridge must be >= 0");
    if (n_classes < 1 || n_classes > det->n_s) return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: n_classes");
    const int n_s = det->n_s;
    for (int i = 0; i < n_s; ++i) {
        if (class_host[i] < 0 || class_host[i] >= n_classes || op_host[i] < 0 || op_host[i] > 23)
            return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: sensor %d class or operation out of range", i);
        if (gain_host && !(gain_host[i] > 0.0)) return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: gains must be > 0");
    }
    for (int a = 0; a < 2; ++a)
        if (n_int[a] < 1 || n_int[a] > 256 || !(lo[a] < hi[a]))
            return fail(ANTS_E_ARG, "ants_lrf_fit_symmetric: axis %d needs 1 <= n_int <= 256, lo < hi", a);
    const long nc = (long)(n_int[0] + 3) * (n_int[1] + 3);
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    cudaStream_t st = ctx->stream[0];
    std::vector<double> coef((size_t)nc * n_classes);
    for (int j = 0; j < n_classes; ++j) {
        // the members' samples mapped into the representative's frame,
        // M^T (p - c) + c, values over the gains; points outside the box left out
        std::vector<double> P, V;
        for (int i = 0; i < n_s; ++i) {
            if (class_host[i] != j) continue;
            const int k = op_host[i];
            const double t = (double)(k % 12) * (3.14159265358979323846 / 6.0);
            double c = std::cos(t), sn = std::sin(t);
            if (k % 3 == 0) {
                const int q = (k % 12) / 3;
                c = q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
                sn = q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
            }
            const double f = k >= 12 ? -1.0 : 1.0;
            const double m00 = c, m01 = -sn * f, m10 = sn, m11 = c * f;
            const double g = gain_host ? gain_host[i] : 1.0;
            for (long e = 0; e < n_pts; ++e) {
                const double dx = pts_host[2 * e] - centre[0], dy = pts_host[2 * e + 1] - centre[1];
                const double x = m00 * dx + m10 * dy + centre[0], y = m01 * dx + m11 * dy + centre[1];
                if (!(x >= lo[0] && x <= hi[0] && y >= lo[1] && y <= hi[1])) continue;
                P.push_back(x);
                P.push_back(y);
                V.push_back(vals_host[e * n_s + i] / g);
            }
        }
        const long np = (long)V.size();
        DevBuf d_pts, d_vals;
        FIT_TRY(dalloc<double>(d_pts, (size_t)np * 2, "points"));
        FIT_TRY(dalloc<double>(d_vals, (size_t)np, "values"));
        if (np > 0) {
            ANTS_CUDA_TRY(cudaMemcpyAsync(d_pts.p, P.data(), P.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                          "fit: upload points");
            ANTS_CUDA_TRY(cudaMemcpyAsync(d_vals.p, V.data(), V.size() * sizeof(double), cudaMemcpyHostToDevice, st),
                          "fit: upload values");
        }
        int rc = lrf_fit_samples(ctx, 2, n_int, lo, hi, np, (const double *)d_pts.p, 1, (const double *)d_vals.p,
                                 ridge, coef.data() + (size_t)j * nc, nullptr, st);
        if (rc != ANTS_OK) return rc;
    }
    long launches = ants_last_launch_count();
    int rc = ants_lrf_create_symmetric(ctx, det, n_int, lo, hi, n_classes, class_host, op_host, centre, coef.data(),
                                       gain_host, out);
    count_launch(launches);
    return rc;
}

extern "C" ANTS_API int ants_lrf_fit(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int,
                                     const double *lo, const double *hi, int shared, long n_pts,
                                     const double *pts_host, const double *vals_host, double ridge,
                                     double *ridge_used, ants_lrf **out)
{
    using namespace ants;
    begin_call();
    ANTS_NVTX("ants_lrf_fit");
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
