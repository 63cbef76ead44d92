// Precision form: score every event on a shared global grid with one tensor-
// core product, then refine the best few grid points.
//
// p1  table    T[g][i] = ln p_i(g) - m_i,  p_i = eta_i / sum_j eta_j at the
//              grid-cell centres g, m_i = mean_g ln p_i(g); BF16, [G][n_s]
//              (sensor index contiguous).  Substituting E = S/H into the
//              Poisson log-likelihood (Sec. 5.1.2.2) gives
//              logL(g) = sum_i s_i ln p_i(g) + const(event), and subtracting
//              m_i only adds - sum_i s_i m_i to every score of an event.
// p2  scores   L[e][g] = sum_i s_i T[g][i] for all events and grid points
//              (BF16 x BF16 -> FP32 tensor-core product), keeping the top-K
//              grid points per event without storing L.
// p3  refine   a local contracting-grid search (Sec. 5.1.2.2) from each
//              candidate not within `nms_cells` cells of a better one (only
//              those are launched); the result with the largest
//              log-likelihood wins (ties: better candidate rank).
#include <cuda_bf16.h>

#include <new>
#include <utility>
#include <vector>

#include "bspline.cuh"
#include "internal.cuh"

struct ants_logtable {
    ants_ctx *ctx = nullptr;
    int device = 0;
    const ants_lrf *lrf = nullptr;
    int nx = 0, ny = 0, n_s = 0;
    float x0 = 0, y0 = 0, dx = 0, dy = 0;  // centre of cell (0, 0) and spacing
    __nv_bfloat16 *d_T = nullptr;          // [nx*ny][n_s]
    float *d_m = nullptr;                  // [n_s]
    // the table the tensor-core scan reads: row r is grid point d_order[r],
    // a fixed pseudo-random order (the running top-K threshold then rises
    // after a few hundred points instead of tracking the raster order)
    __nv_bfloat16 *d_Tp = nullptr;         // [nx*ny][n_s]
    int *d_order = nullptr;                // [nx*ny]
};

namespace ants {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kEtaFloor = 1e-30f;

// one warp per grid point: lnp[g][i] = ln eta_i - ln H
__global__ void table_lnp(LrfDev L, int nx, int ny, float x0, float y0, float dx, float dy, float *lnp)
{
    const long g = (long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (g >= (long)nx * ny) return;
    const float x = x0 + dx * (float)(g % nx), y = y0 + dy * (float)(g / nx);
    float H = 0.0f;
    for (int i = lane; i < L.n_s; i += 32) {
        bool ok;
        const float v = fmaxf(lrf_eta_point(L, i, x, y, 0.0f, ok), kEtaFloor);
        lnp[g * L.n_s + i] = logf(v);
        H += v;
    }
    for (int o = 16; o; o >>= 1) H += __shfl_xor_sync(kFull, H, o);
    const float lh = logf(H);
    for (int i = lane; i < L.n_s; i += 32) lnp[g * L.n_s + i] -= lh;
}

// m_i = mean over grid points (fixed order), T = bf16(lnp - m)
__global__ void table_center(const float *lnp, long G, int n_s, float *m, __nv_bfloat16 *T)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_s) return;
    double acc = 0.0;
    for (long g = 0; g < G; ++g) acc += lnp[g * n_s + i];
    const float mi = (float)(acc / (double)G);
    m[i] = mi;
    for (long g = 0; g < G; ++g) T[g * n_s + i] = __float2bfloat16_rn(lnp[g * n_s + i] - mi);
}

// candidate starts: non-maximum suppression in rank order; suppressed -> NaN
__global__ void candidate_starts(const int *idx, long n, int K, int nx, float x0, float y0, float dx, float dy,
                                 float nms, float *starts)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float qnan = __int_as_float(0x7fc00000);
    int kept[8];
    int nk = 0;
    for (int j = 0; j < K; ++j) {
        const int g = idx[e * K + j];
        float *st = starts + (e * K + j) * 3;
        bool ok = g >= 0 && g < 0x7fffffff;
        for (int q = 0; q < nk && ok; ++q) {
            const int h = kept[q];
            const float cx = fabsf((float)(g % nx - h % nx)), cy = fabsf((float)(g / nx - h / nx));
            if (fmaxf(cx, cy) <= nms) ok = false;
        }
        if (ok) {
            kept[nk++] = g;
            st[0] = x0 + dx * (float)(g % nx);
            st[1] = y0 + dy * (float)(g / nx);
            st[2] = 0.0f;
        } else {
            st[0] = st[1] = st[2] = qnan;
        }
    }
}

// best of the K refines of each event (largest logL; ties to the better rank)
__global__ void pick_best(long n, int K, const float *xyz_c, const float *E_c, const float *logL_c,
                          const int32_t *st_c, float *xyz, float *E, float *logL, int32_t *status, int32_t *cand)
{
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    int best = -1;
    float bl = -INFINITY;
    for (int j = 0; j < K; ++j) {
        const long v = e * K + j;
        if (st_c[v] != ANTS_EVT_OK) continue;
        if (best < 0 || logL_c[v] > bl) {
            best = j;
            bl = logL_c[v];
        }
    }
    const long v = e * K + (best < 0 ? 0 : best);
    xyz[3 * e] = xyz_c[3 * v];
    xyz[3 * e + 1] = xyz_c[3 * v + 1];
    xyz[3 * e + 2] = xyz_c[3 * v + 2];
    E[e] = E_c[v];
    logL[e] = logL_c[v];
    status[e] = st_c[v];
    if (cand) cand[e] = best;
}

unsigned nb(long n, int per) { return (unsigned)((n + per - 1) / per); }

// Candidates that survived the suppression (and every event's first, whose
// search also reports the event's signal status) are listed for the refine;
// the others are marked as not searched.  The order of the list does not
// matter: results go back to each candidate's own slot.
__global__ void compact_candidates(const float *starts, long nv, int K, int *count, int *cidx, int *crow,
                                   float *cstart, float *xyz_c, float *E_c, float *logL_c, int32_t *st_c)
{
    const long v = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    const bool kept = (v % K) == 0 || !isnan(starts[3 * v]);
    if (kept) {
        const int r = atomicAdd(count, 1);
        cidx[r] = (int)v;
        crow[r] = (int)(v / K);
        cstart[3 * r] = starts[3 * v];
        cstart[3 * r + 1] = starts[3 * v + 1];
        cstart[3 * r + 2] = starts[3 * v + 2];
    } else {
        const float qnan = __int_as_float(0x7fc00000);
        xyz_c[3 * v] = xyz_c[3 * v + 1] = xyz_c[3 * v + 2] = qnan;
        E_c[v] = logL_c[v] = qnan;
        st_c[v] = ANTS_EVT_OUT_OF_DOMAIN;
    }
}

__global__ void scatter_candidates(const int *count, const int *cidx, const float *o_xyz, const float *o_E,
                                   const float *o_logL, const int32_t *o_st, float *xyz_c, float *E_c, float *logL_c,
                                   int32_t *st_c)
{
    const long r = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= *count) return;
    const long v = cidx[r];
    xyz_c[3 * v] = o_xyz[3 * r];
    xyz_c[3 * v + 1] = o_xyz[3 * r + 1];
    xyz_c[3 * v + 2] = o_xyz[3 * r + 2];
    E_c[v] = o_E[r];
    logL_c[v] = o_logL[r];
    st_c[v] = o_st[r];
}

// Tp[r] = T[order[r]]
__global__ void permute_rows(const __nv_bfloat16 *T, const int *order, long G, int n_s, __nv_bfloat16 *Tp)
{
    const long t = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G * n_s) return;
    const long r = t / n_s;
    Tp[t] = T[(long)order[r] * n_s + (t - r * n_s)];
}

// Fisher-Yates shuffle driven by splitmix64 (Steele, Lea and Flood 2014), fixed seed
std::vector<int> scan_order(long G)
{
    std::vector<int> o((size_t)G);
    for (long g = 0; g < G; ++g) o[(size_t)g] = (int)g;
    uint64_t x = 0x414E545332ull;
    for (long i = G - 1; i > 0; --i) {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const long j = (long)(z % (uint64_t)(i + 1));
        std::swap(o[(size_t)i], o[(size_t)j]);
    }
    return o;
}

}  // namespace

int check_gemm_params(const ants_lrf *lrf, const ants_gemm_params *P)
{
    if (!P || !P->table) return fail(ANTS_E_ARG, "precision form: NULL params or table");
    if (P->table->lrf != lrf) return fail(ANTS_E_ARG, "precision form: the table belongs to another LRF set");
    if (P->top_k < 1 || P->top_k > 8) return fail(ANTS_E_ARG, "precision form: top_k must be in [1, 8]");
    if (!(P->nms_cells >= 0.0f)) return fail(ANTS_E_ARG, "precision form: nms_cells must be >= 0");
    return check_cgs_params(lrf, &P->refine);
}

int reconstruct_gemm_topk(ants_ctx *ctx, const ants_lrf *lrf, const ants_gemm_params &P, const float *sig, long n,
                          float *xyz, float *E, float *logL, int32_t *status, cudaStream_t s)
{
    const ants_logtable *T = P.table;
    const int K = P.top_k, n_s = lrf->n_s;
    const long G = (long)T->nx * T->ny;
    const long nv = n * K;
    float *val = (float *)ctx_scratch(ctx, 1, (size_t)nv * sizeof(float));
    int *idx = (int *)ctx_scratch(ctx, 2, (size_t)nv * sizeof(int));
    float *starts = (float *)ctx_scratch(ctx, 3, (size_t)nv * 3 * sizeof(float));
    unsigned char *outc = (unsigned char *)ctx_scratch(ctx, 4, (size_t)nv * 6 * sizeof(float) + 1024);
    if (!val || !idx || !starts || !outc) return ANTS_E_OOM;
    float *xyz_c = (float *)outc, *E_c = xyz_c + 3 * nv, *logL_c = E_c + nv;
    int32_t *st_c = (int32_t *)(logL_c + nv);
    // chunks keep the M dimension of one product in int range
    const long chunk = 1L << 24;
    for (long off = 0; off < n; off += chunk) {
        const long m = n - off < chunk ? n - off : chunk;
        int rc = mma_topk(ctx, sig + off * n_s, true, T->d_Tp, T->d_order, (int)m, (int)G, n_s, K, val + off * K,
                          idx + off * K, s);
        if (rc != ANTS_OK) return rc;
    }
    candidate_starts<<<nb(n, 256), 256, 0, s>>>(idx, n, K, T->nx, T->x0, T->y0, T->dx, T->dy, P.nms_cells, starts);
    count_launch();
    int rc = ANTS_OK;
    if (!cgs_xy_supported(lrf, P.refine) || nv > 0x7fffffffL) {
        // every candidate searched (suppressed ones stop at their NaN start)
        rc = launch_cgs_rows(ctx, lrf, P.refine, sig, K, nv, starts, xyz_c, E_c, logL_c, st_c, nullptr, s);
        if (rc != ANTS_OK) return rc;
    } else {
        // only the kept candidates are searched
        unsigned char *lst = (unsigned char *)ctx_scratch(ctx, 5, 256 + (size_t)nv * 5 * sizeof(float));
        unsigned char *res = (unsigned char *)ctx_scratch(ctx, 6, (size_t)nv * 6 * sizeof(float) + 1024);
        if (!lst || !res) return ANTS_E_OOM;
        int *d_count = (int *)lst;
        int *cidx = (int *)(lst + 256), *crow = cidx + nv;
        float *cstart = (float *)(crow + nv);
        float *o_xyz = (float *)res, *o_E = o_xyz + 3 * nv, *o_logL = o_E + nv;
        int32_t *o_st = (int32_t *)(o_logL + nv);
        ANTS_CUDA_TRY(cudaMemsetAsync(d_count, 0, sizeof(int), s), "candidate count");
        compact_candidates<<<nb(nv, 256), 256, 0, s>>>(starts, nv, K, d_count, cidx, crow, cstart, xyz_c, E_c, logL_c,
                                                       st_c);
        count_launch();
        int h_count = 0;
        ANTS_CUDA_TRY(cudaMemcpyAsync(&h_count, d_count, sizeof(int), cudaMemcpyDeviceToHost, s), "candidate count");
        ANTS_CUDA_TRY(cudaStreamSynchronize(s), "candidate count");
        if (h_count > 0) {
            rc = launch_cgs_xy(ctx, lrf, P.refine, sig, 1, crow, h_count, cstart, o_xyz, o_E, o_logL, o_st, nullptr,
                               s);
            if (rc != ANTS_OK) return rc;
            scatter_candidates<<<nb(h_count, 256), 256, 0, s>>>(d_count, cidx, o_xyz, o_E, o_logL, o_st, xyz_c, E_c,
                                                                logL_c, st_c);
            count_launch();
        }
    }
    pick_best<<<nb(n, 256), 256, 0, s>>>(n, K, xyz_c, E_c, logL_c, st_c, xyz, E, logL, status, nullptr);
    count_launch();
    ANTS_CUDA_TRY(cudaGetLastError(), "precision form launch");
    return ANTS_OK;
}

}  // namespace ants

using namespace ants;

extern "C" {

ANTS_API int ants_logtable_create(ants_ctx *ctx, const ants_lrf *lrf, int nx, int ny, ants_logtable **out)
{
    begin_call();
    ANTS_NVTX("ants_logtable_create");
    if (!out) return fail(ANTS_E_ARG, "ants_logtable_create: out is NULL");
    *out = nullptr;
    if (!ctx || !lrf || lrf->ctx != ctx) return fail(ANTS_E_ARG, "ants_logtable_create: bad ctx or lrf");
    if (lrf->type != ANTS_LRF_XY) return fail(ANTS_E_UNIMPLEMENTED, "ants_logtable_create: XY LRFs only");
    if (nx < 2 || ny < 2 || (long)nx * ny > (1L << 20)) return fail(ANTS_E_ARG, "ants_logtable_create: bad grid");
    if (lrf->n_s % 8 != 0) return fail(ANTS_E_SHAPE, "ants_logtable_create: n_sensors must be a multiple of 8");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    ants_logtable *T = new (std::nothrow) ants_logtable();
    if (!T) return fail(ANTS_E_OOM, "ants_logtable_create: out of host memory");
    T->ctx = ctx;
    T->device = ctx->device;
    T->lrf = lrf;
    T->nx = nx;
    T->ny = ny;
    T->n_s = lrf->n_s;
    T->dx = (float)((lrf->hi[0] - lrf->lo[0]) / nx);
    T->dy = (float)((lrf->hi[1] - lrf->lo[1]) / ny);
    T->x0 = (float)(lrf->lo[0] + 0.5 * (lrf->hi[0] - lrf->lo[0]) / nx);
    T->y0 = (float)(lrf->lo[1] + 0.5 * (lrf->hi[1] - lrf->lo[1]) / ny);
    const long G = (long)nx * ny;
    float *lnp = nullptr;
    cudaError_t e = cudaMalloc(&lnp, (size_t)G * T->n_s * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&T->d_T, (size_t)G * T->n_s * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&T->d_m, (size_t)T->n_s * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&T->d_Tp, (size_t)G * T->n_s * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&T->d_order, (size_t)G * sizeof(int));
    if (e == cudaSuccess) {
        const std::vector<int> order = scan_order(G);
        e = cudaMemcpy(T->d_order, order.data(), (size_t)G * sizeof(int), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) {
        table_lnp<<<nb(G, 8), 256>>>(lrf->dev, nx, ny, T->x0, T->y0, T->dx, T->dy, lnp);
        table_center<<<nb(T->n_s, 128), 128>>>(lnp, G, T->n_s, T->d_m, T->d_T);
        permute_rows<<<nb(G * T->n_s, 256), 256>>>(T->d_T, T->d_order, G, T->n_s, T->d_Tp);
        count_launch(3);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    cudaFree(lnp);
    if (e != cudaSuccess) {
        ants_logtable_free(T);
        return cuda_fail(e, "ants_logtable_create");
    }
    *out = T;
    return ANTS_OK;
}

ANTS_API int ants_logtable_values(const ants_logtable *T, float *table_host, float *mean_host)
{
    begin_call();
    if (!T) return fail(ANTS_E_ARG, "ants_logtable_values: NULL table");
    const long G = (long)T->nx * T->ny;
    ANTS_CUDA_TRY(cudaSetDevice(T->ctx->device), "cudaSetDevice");
    if (table_host) {
        std::vector<__nv_bfloat16> h((size_t)G * T->n_s);
        ANTS_CUDA_TRY(cudaMemcpy(h.data(), T->d_T, h.size() * sizeof(__nv_bfloat16), cudaMemcpyDeviceToHost), "copy");
        for (size_t k = 0; k < h.size(); ++k) table_host[k] = __bfloat162float(h[k]);
    }
    if (mean_host)
        ANTS_CUDA_TRY(cudaMemcpy(mean_host, T->d_m, T->n_s * sizeof(float), cudaMemcpyDeviceToHost), "copy");
    return ANTS_OK;
}

ANTS_API int ants_logtable_topk(ants_ctx *ctx, const ants_logtable *T, const float *signals_dev, long n_events,
                                int n_sensors, int top_k, float *score_dev, int32_t *index_dev, void *stream)
{
    begin_call();
    ANTS_NVTX("ants_logtable_topk");
    if (!ctx || !T || T->ctx != ctx) return fail(ANTS_E_ARG, "ants_logtable_topk: bad ctx or table");
    if (n_sensors != T->n_s) return fail(ANTS_E_SHAPE, "ants_logtable_topk: n_sensors %d", n_sensors);
    if (n_events < 0 || n_events > (1L << 30)) return fail(ANTS_E_ARG, "ants_logtable_topk: n_events out of range");
    if (n_events == 0) return ANTS_OK;
    if (!signals_dev || !score_dev || !index_dev) return fail(ANTS_E_ARG, "ants_logtable_topk: NULL buffer");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    int rc = mma_topk(ctx, signals_dev, true, T->d_Tp, T->d_order, (int)n_events, T->nx * T->ny, T->n_s, top_k,
                      score_dev, index_dev, (cudaStream_t)stream);
    if (rc == ANTS_OK) rc = check_bounds(ctx, (cudaStream_t)stream);
    return rc;
}

ANTS_API void ants_logtable_free(ants_logtable *T)
{
    if (!T) return;
    cudaSetDevice(T->device);
    cudaFree(T->d_T);
    cudaFree(T->d_m);
    cudaFree(T->d_Tp);
    cudaFree(T->d_order);
    delete T;
    (void)cudaGetLastError();
}

}  // extern "C"
