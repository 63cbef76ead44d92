// Internal declarations shared by the libants translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <string>
#include <vector>

#include "ants.h"

namespace ants {

// ---------------------------------------------------------------------------
// errors and launch accounting (thread-local, reported through the C ABI)
// ---------------------------------------------------------------------------
int fail(int code, const char *fmt, ...);          // records a message, returns code
int cuda_fail(cudaError_t e, const char *what);    // ANTS_E_CUDA with the CUDA message
void begin_call();                                 // clears the error, zeroes the launch count
void count_launch(long n = 1);

#define ANTS_CUDA_TRY(expr, what)                           \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ::ants::cuda_fail(_e, what); \
    } while (0)

// ---------------------------------------------------------------------------
// index checks of the ANTS_DEBUG_BOUNDS build: ANTS_IN_RANGE(word, i, n, site)
// is true when 0 <= i < n; in that build an index outside the range records
// `site` in *word (the first one wins) and the caller skips the access, so a
// wrong index is reported instead of touching memory.  In the normal build the
// macro is the constant true and every check compiles away.
// ---------------------------------------------------------------------------
#ifdef ANTS_DEBUG_BOUNDS
__device__ __forceinline__ bool dbg_in_range(int *word, long long i, long long n, int site)
{
    if (i >= 0 && i < n) return true;
    if (word) atomicCAS(word, 0, site);
    return false;
}
#define ANTS_IN_RANGE(word, i, n, site) ::ants::dbg_in_range((word), (long long)(i), (long long)(n), (site))
#else
#define ANTS_IN_RANGE(word, i, n, site) true
#endif

// a named NVTX range over one library call (seen by profilers that record NVTX)
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};
#define ANTS_NVTX(name) ::ants::NvtxScope ants_nvtx_scope_(name)

// ---------------------------------------------------------------------------
// device view of an LRF set, passed by value to kernels
// ---------------------------------------------------------------------------
struct LrfDev {
    int type;          // ANTS_LRF_*
    int n_s;           // sensors
    int shared;        // RADIAL: one coefficient set for all sensors
    int n_coef;        // coefficients per set
    int n_int[3];      // intervals per axis
    int stride_y;      // n_int[0] + 3
    int stride_z;      // (n_int[0] + 3) * (n_int[1] + 3)
    int positive;      // every coefficient > 0 and max <= 2^100 min (eta > 0, ratios normal)
    float lo[3], hi[3], inv_h[3];
    const float *coef; // [n_sets][n_coef] FP32
    const float *sxy;  // [n_s][2]
    const float *gain; // [n_s] factor on a RADIAL LRF
    const float *cog_w;// [n_s] 1 / relative gain (centroid weights)
    int *dbg;          // the context's index-check word (written only by the ANTS_DEBUG_BOUNDS build)
    // XY LRFs: sensors interleaved in pairs, [n_pairs][n_int[1]+3][n_int[0]+3]
    // float2 = (sensor 2p, sensor 2p+1); an odd count is padded with zeros
    const float2 *coef2;
    // XY LRFs: the same pairs with the pair index fastest, [n_int[1]+3][n_int[0]+3][n_pairs]
    // float2 (a warp whose lanes take consecutive pairs reads one contiguous run)
    const float2 *coef2_pf;
    const float *coef_t;   // XY: the coefficients sensor-minor, [k][n_s] (per-point loops over sensors)
    const int *set_of;     // RADIAL grouped / XY symmetry classes (Sec. 6.2): the coefficient set of each sensor; nullable
    int n_sets;            // coefficient sets
    const int *op_of;      // XY symmetry classes: the operation of each sensor (sym_op)
    float sym_c[2];        // XY symmetry classes: the centre of the operations
    // RADIAL LRFs: each interval's cubic in the power basis of its local
    // parameter t, (p0, p1, p2, p3) with f = p0 + t (p1 + t (p2 + t p3)),
    // [n_sets][n_int[0]]
    const float4 *rpoly;
    int n_pairs;
    int pair_stride;   // (n_int[1]+3) * (n_int[0]+3)
    // COMPOSITE: the axial part's intervals on [0, hi_r] (its cubics in
    // rpoly, [n_s][n_int_r]); the XY part follows n_int_r + 3 coefficients
    // of each sensor's set in coef.  SLICED: planes over lo[2]..hi[2],
    // inv_h[2] = (n_planes - 1) / (hi[2] - lo[2]).
    int n_int_r;
    float hi_r, inv_h_r;
    int n_planes, n_coef_xy;
};

}  // namespace ants

constexpr int kScratchSlots = 13;

struct ants_ctx {
    int device = 0;
    int n_sm = 0;
    size_t smem_optin = 0;
    cudaStream_t stream[2] = {nullptr, nullptr};
    // chunk buffers of ants_reconstruct_host (grown on demand)
    size_t host_cap_events = 0;
    int host_cap_sensors = 0;
    void *d_sig[2] = {nullptr, nullptr};
    float *d_start[2] = {nullptr, nullptr};
    float *d_out[2] = {nullptr, nullptr};   // xyz(3) E logL per event
    int32_t *d_status[2] = {nullptr, nullptr};
    // general device scratch slots (grown on demand by ants::ctx_scratch):
    // 0 network activations, 1-6 precision and learned forms, 7 FP16
    // widening, 8-9 LRF fit, 10 refit samples, 11 event filter, 12 mapped
    // samples of symmetry classes
    void *scratch[kScratchSlots] = {};
    size_t scratch_cap[kScratchSlots] = {};
    // device word set by a kernel whose bounded wait ran out (ants_ctx_fault)
    int *d_fault = nullptr;
    // device word of the ANTS_DEBUG_BOUNDS build: the site of the first index
    // a checked kernel found out of range (ants_debug_bounds_site)
    int *d_bounds = nullptr;
};

struct ants_detector {
    int n_s = 0;
    std::vector<double> xy;    // [n_s][2]
    std::vector<double> gain;  // [n_s] relative gains (1 when not given)
};

struct ants_lrf {
    ants_ctx *ctx = nullptr;
    int device = 0;  // the context's device (freeing does not read the context)
    int type = 0, n_s = 0, shared = 0, n_sets = 0, n_coef = 0;
    int n_int[3] = {0, 0, 0};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    std::vector<double> coef;      // FP64 master [n_sets][n_coef]
    std::vector<double> gain;      // [n_s] (RADIAL factor; 1 otherwise)
    std::vector<double> sxy;       // [n_s][2]
    std::vector<double> rel_gain;  // [n_s] detector relative gains
    int n_int_r = 0;               // COMPOSITE axial part
    double hi_r = 0.0;
    int n_planes = 0;              // SLICED
    float *d_coef = nullptr, *d_sxy = nullptr, *d_gain = nullptr, *d_cogw = nullptr;
    float2 *d_coef2 = nullptr;
    float2 *d_coef2_pf = nullptr;
    float *d_coeft = nullptr;
    int *d_set_of = nullptr;
    std::vector<int> groups;       // RADIAL grouped / XY classes: the group of each sensor (empty otherwise)
    std::vector<int> ops;          // XY classes: the symmetry operation of each sensor
    double sym_c[2] = {0.0, 0.0};
    int *d_op_of = nullptr;
    float4 *d_rpoly = nullptr;
    ants::LrfDev dev{};
};

namespace ants {
int lrf_dims(int type);
// the LRF types with a z coordinate / with an XY box as (part of) their domain
// kernel template argument for XY sets with symmetry classes (their API type
// stays ANTS_LRF_XY; the kernels that read them are instantiated apart so the
// plain XY code carries no symmetry branch)
constexpr int kLrfXYSym = 100;

// the 2 x 2 matrix of symmetry operation k (row-major): the rotation by
// (k mod 12) x 30 degrees, preceded for k >= 12 by the reflection y -> -y
__host__ __device__ inline void sym_op(int k, float m[4])
{
    // cos and sin of (k mod 12) x 30 degrees, rounded to float (no table, so
    // no local memory in the kernels)
    const float h = 0.8660254037844386f;
    float c = 1.0f, s = 0.0f;
    switch (k % 12) {
    case 1: c = h; s = 0.5f; break;
    case 2: c = 0.5f; s = h; break;
    case 3: c = 0.0f; s = 1.0f; break;
    case 4: c = -0.5f; s = h; break;
    case 5: c = -h; s = 0.5f; break;
    case 6: c = -1.0f; s = 0.0f; break;
    case 7: c = -h; s = -0.5f; break;
    case 8: c = -0.5f; s = -h; break;
    case 9: c = 0.0f; s = -1.0f; break;
    case 10: c = 0.5f; s = -h; break;
    case 11: c = h; s = -0.5f; break;
    default: break;
    }
    const float f = k >= 12 ? -1.0f : 1.0f;
    m[0] = c;
    m[1] = -s * f;
    m[2] = s;
    m[3] = c * f;
}

__host__ __device__ inline bool lrf_is_3d(int type)
{
    return type == ANTS_LRF_XYZ || type == ANTS_LRF_AXIAL_Z || type == ANTS_LRF_SLICED;
}
__host__ __device__ inline bool lrf_has_box(int type)
{
    return type == ANTS_LRF_XY || type == ANTS_LRF_XYZ || type == ANTS_LRF_COMPOSITE || type == ANTS_LRF_SLICED ||
           type == kLrfXYSym;
}
// any LRF type: create from coefficients (api.cu)
int lrf_create_impl(ants_ctx *ctx, const ants_detector *det, int type, const int *n_int, const double *lo,
                    const double *hi, int shared, const double *coef_host, const double *gain_host, int n_int_r,
                    double hi_r, int n_planes, ants_lrf **out, int n_groups = 0,
                    const int *group = nullptr, const int *op = nullptr, const double *centre = nullptr);
// launches of the reconstruction kernels (cgs.cu)
int launch_cgs_plain(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p,
                     const float *sig, long n_e, const float *start, float *xyz, float *E,
                     float *logL, int32_t *status, int16_t *trace, cudaStream_t stream);
int check_cgs_params(const ants_lrf *lrf, const ants_cgs_params *p);
// offsets of consecutive 256-byte aligned pieces of one scratch arena
struct Carve {
    size_t off = 0;
    template <class T>
    size_t take(size_t count)
    {
        const size_t at = off;
        off += (count * sizeof(T) + 255) & ~(size_t)255;
        return at;
    }
};
// device scratch slot `slot` (0..12) of at least `bytes`; NULL (error recorded) on failure.
// Growing a slot frees the old buffer, so the caller must not have work in
// flight that uses it.
void *ctx_scratch(ants_ctx *ctx, int slot, size_t bytes);
// exclusive prefix sum of n int32 values (in == out allowed); *total_dev
// (nullable) receives the sum; tmp holds exclusive_scan_tmp_bytes(n) bytes
size_t exclusive_scan_tmp_bytes(long n);
int exclusive_scan(const int *in, int *out, long n, int *total_dev, void *tmp, cudaStream_t s);
// FP64 least-squares B-spline fit from device samples pts [n_pts][dims],
// vals [n_pts][n_sets]; coefficients [n_sets][n_coef] to the host (fit.cu)
int lrf_fit_samples(ants_ctx *ctx, int dims, const int *n_int, const double *lo, const double *hi,
                    long n_pts, const double *pts, int n_sets, const double *vals, double ridge, double *coef_out,
                    double *ridge_used, cudaStream_t st);
// f[i] = h[i] for n FP16 values (exact widening), on stream s
int widen_half(const __half *h, size_t n, float *f, cudaStream_t s);
// learned proposal (mlp.cu)
int mlp_forward(ants_ctx *ctx, const ants_mlp *M, const float *sig, long n, bool bf, float *O, cudaStream_t s);
int mlp_decode(const ants_mlp *M, const float *O, long n, float *xyz, float *E, cudaStream_t s);
int mlp_n_in(const ants_mlp *M);
// ANTS_DEBUG_BOUNDS build: wait for stream s and fail with ANTS_E_INTERNAL when
// a checked kernel recorded an index out of range (a no-op otherwise)
int check_bounds(const ants_ctx *ctx, cudaStream_t s);
// tcgen05 products with fused epilogues (umma.cu); B [N][K] BF16, K <= 256
// top-K: columns ranked by value, ties by order[n] (the grid index of column n)
int mma_topk(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *B, const int *order, int M, int N,
             int K, int topk, float *val, int *idx, cudaStream_t s);
int mma_bias_gelu(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *B, const float *bias, int M,
                  int N, int K, __nv_bfloat16 *out, cudaStream_t s);
// training products of the network with BF16 operands (umma.cu):
// z = A W^T + b (FP32), h = GELU(z) (BF16), hT = h transposed [N][ldT] (nullable)
int mma_train_forward(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *W, const float *bias,
                      int M, int N, int K, float *z, __nv_bfloat16 *h, __nv_bfloat16 *hT, int ldT, cudaStream_t s);
// dz = (dY Wt^T) GELU'(z) (FP32) and dzT = dz transposed in BF16 [N][ldT] (nullable)
int mma_gelu_backward(const ants_ctx *ctx, const float *dY, const __nv_bfloat16 *Wt, const float *z, int M, int N,
                      int K, float *dz, __nv_bfloat16 *dzT, int ldT, cudaStream_t s);
// C = A B^T in FP32, A [M][K] and B [N][K] BF16 (any K with N <= 256)
int mma_f32(const ants_ctx *ctx, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, float *C,
            cudaStream_t s);
// precision form (precision.cu)
int check_gemm_params(const ants_lrf *lrf, const ants_gemm_params *P);
int reconstruct_gemm_topk(ants_ctx *ctx, const ants_lrf *lrf, const ants_gemm_params &P, const float *sig, long n,
                          float *xyz, float *E, float *logL, int32_t *status, cudaStream_t s);
// learned-proposal reconstruction (seeded.cu)
int check_seeded_params(const ants_lrf *lrf, const ants_mlp_seeded_params *P);
int reconstruct_mlp_seeded(ants_ctx *ctx, const ants_lrf *lrf, const ants_mlp_seeded_params &P, const float *sig,
                           long n, float *xyz, float *E, float *logL, int32_t *status, int16_t *trace,
                           cudaStream_t s);
bool cgs_xy_supported(const ants_lrf *lrf, const ants_cgs_params &p);
// search variants (variant.cu)
int check_minimize_params(const ants_lrf *lrf, const ants_minimize_params *P);
int reconstruct_minimize(const ants_ctx *ctx, const ants_lrf *lrf, const ants_minimize_params &P, const float *sig,
                         long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                         int16_t *n_iter, cudaStream_t s);
int check_variant_params(const ants_lrf *lrf, const ants_cgs_variant_params *P);
// start (nullable): given starts [n_e][3] instead of the variant's own
int reconstruct_variant(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_variant_params &P, const float *sig,
                        long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                        int16_t *trace, cudaStream_t s);
// event e reads signal row rows[e] when rows is given, else row e / row_div
int launch_cgs_xy(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig, int row_div,
                  const int *rows,
                  long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status, int16_t *trace,
                  cudaStream_t stream);
// as launch_cgs_plain, with event e reading signal row e / row_div
int launch_cgs_rows(const ants_ctx *ctx, const ants_lrf *lrf, const ants_cgs_params &p, const float *sig,
                    int row_div, long n_e, const float *start, float *xyz, float *E, float *logL, int32_t *status,
                    int16_t *trace, cudaStream_t stream);
}  // namespace ants
