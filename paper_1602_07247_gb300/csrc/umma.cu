// BF16 products on the fifth-generation tensor cores (tcgen05) with fused row
// epilogues:
//
//   C[m][n] = sum_k A[m][k] B[n][k]     A [M][K]: FP32 (rounded to BF16 while
//                                       it is staged) or BF16;  B [N][K] BF16
//
// K a multiple of 8, at most 256 unless N fits one 256-column n-tile (then
// the band's A is streamed through its four 64-wide chunk slots, any K); A
// rows 16-byte aligned.  Persistent CTAs (one per SM) take 128-row bands of C
// ("m-tiles") in a fixed stride; every band walks all of N in 256-column
// n-tiles.  Warp roles (22 warps):
//   warp 0      TMA producer: B as 256 x 64 boxes (128-byte swizzle) through
//               a 3-stage ring, re-read from L2 for every band;
//   warp 1      allocates 512 TMEM columns; one thread issues
//               tcgen05.mma.kind::f16 (M = 128, N = 256, K = 16) into one of
//               two 128 x 256 FP32 accumulators;
//   warps 2-5   stage the band's A in shared memory in the same swizzled
//               K-major layout, one 64-wide K chunk at a time; a chunk is
//               refilled for the next band as soon as the last MMA reading it
//               has completed (its own full/empty mbarrier pair);
//   warps 6-21  epilogue: tcgen05.ld of the finished accumulator while the
//               other one fills (warp w reads TMEM lanes 32(w%4)..+31, i.e. C
//               rows; four groups of four warps take 64 columns each).
// Epilogues:
//   EPI_TOPK       running top-K per row over all N (value desc, column asc),
//                  written as K (score, column) pairs per row;
//   EPI_BIAS_GELU  GELU(C + bias[n]) stored as BF16 (N a multiple of 8);
// and for training the network (Sec. 5.1.3) with BF16 operands (N a multiple
// of 8; the transposed BF16 copies [N][ldT] are the K-major operands of the
// weight gradients, rows M..ldT-1 written as zeros):
//   EPI_SAVE       z = C + bias[n] kept in FP32, GELU(z) stored as BF16, and
//                  optionally transposed;
//   EPI_GELU_BWD   dz = C GELU'(z[m][n]) stored in FP32 and transposed BF16;
//   EPI_F32        C stored in FP32 (weight gradients, K = batch).
// Every mbarrier wait is bounded in time.  A wait that runs out sets a shared
// abort flag and the context's fault word; every role then stops, waits
// (bounded) for its own copies and products in flight, and the block frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <vector>

#include "internal.cuh"

namespace ants {

namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 2, kMaxK = 256, kMaxTop = 8;
constexpr int kAChunks = kMaxK / kBK;
constexpr int kLoaderWarp0 = 2, kEpiWarp0 = 6, kEpiWarps = 16;
constexpr int kEpiGroups = kEpiWarps / 4, kGroupCols = kBN / kEpiGroups;  // 4 groups of 64 columns
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kThreads = (kEpiWarp0 + kEpiWarps) * 32;
constexpr uint32_t kAChunkBytes = kBM * kBK * 2;  // 16 KiB
constexpr uint32_t kBStageBytes = kBN * kBK * 2;  // 32 KiB
constexpr uint64_t kWaitNs = 1000000000ull;       // 1 s per wait

enum { EPI_TOPK = 0, EPI_BIAS_GELU = 1, EPI_SAVE = 2, EPI_GELU_BWD = 3, EPI_F32 = 4 };

// shared-memory map (offsets from a 1024-byte aligned base)
constexpr uint32_t kOffA = 0;
constexpr uint32_t kOffB = kOffA + kAChunks * kAChunkBytes;
constexpr int kChunk = 32;                                                // columns staged per candidate pass
constexpr uint32_t kOffCand = kOffB + kStages * kBStageBytes;             // staged values [kChunk][kEpiThreads]
constexpr uint32_t kOffThr = kOffCand + kChunk * kEpiThreads * 4;          // top-K thresholds [kEpiGroups][kBM]
constexpr uint32_t kOffBar = kOffThr + kEpiGroups * kBM * 4;
constexpr int kNumBars = 2 * kStages + 2 * kAChunks + 4 + 1 + 2;
constexpr uint32_t kOffMisc = kOffBar + kNumBars * 8;                     // tmem base, abort flag
constexpr uint32_t kSmemBytes = kOffMisc + 16 + 1024;                     // + alignment slack

struct UmmaArgs {
    int M, N, K;
    const void *A;
    int topk;
    const int *order;  // grid index of column n (top-K ranks ties by it)
    float *top_val;
    int *top_idx;
    const float *bias;
    __nv_bfloat16 *out;
    float *zbuf;               // EPI_SAVE: z written; EPI_GELU_BWD: z read ([M][N] FP32)
    float *out_f;              // EPI_GELU_BWD, EPI_F32: [M][N] FP32
    __nv_bfloat16 *out_t;      // transposed BF16 copy [N][ldT] (nullable)
    int ldT;
    int *fault;
    int *dbg;                  // index-check word (ANTS_DEBUG_BOUNDS build)
    int hold_producer;  // self-test only: the TMA producer issues nothing
};

// ---- PTX wrappers -----------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint32_t b, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(count) : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void bar_arrive(uint32_t b)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint32_t b, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
}

__device__ __forceinline__ uint64_t now_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// the same test, the thread suspended until the phase completes or about
// kSuspendNs have passed (a waiting role then takes no issue slots from the
// roles that work)
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool bar_try_suspend(uint32_t b, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok)
        : "r"(b), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// bounded wait; false once this or another role has given up
__device__ __forceinline__ bool bar_wait(uint32_t b, uint32_t parity, volatile int *abort, int *fault)
{
    if (bar_try(b, parity)) return true;
    const uint64_t t0 = now_ns();
    while (true) {
        if (bar_try_suspend(b, parity)) return true;
        if (*abort) return false;
        if (now_ns() - t0 > kWaitNs) {
            *abort = 1;
            atomicExch(fault, 1);
            return false;
        }
    }
}

// bounded wait used while draining (ignores the abort flag)
__device__ __forceinline__ void bar_drain(uint32_t b, uint32_t parity, int *fault)
{
    const uint64_t t0 = now_ns();
    while (!bar_try_suspend(b, parity))
        if (now_ns() - t0 > kWaitNs) {
            atomicExch(fault, 1);
            return;
        }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t b)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(b)
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (leading offset unused for this layout; set to 16 bytes)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t accumulate)
{
    asm volatile(
        "{ .reg .pred p; setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(tmem),
        "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint32_t b)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(b) : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }

// d GELU / dx = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.3989422804014327f * expf(-0.5f * x * x);
}

// grid index of column n; the empty-entry marker -1 ranks last
__device__ __forceinline__ int gidx(const int *order, int n) { return n >= 0 ? __ldg(order + n) : 0x7fffffff; }

// (x, grid index ox) ranks before list entry (w, column d)
__device__ __forceinline__ bool ahead_of(float x, int ox, float w, int d, const int *order)
{
    return x > w || (x == w && ox < gidx(order, d));
}

// The running top-K of a row is an unsorted list: slots j < K hold entries
// (value tv, column tn; empty: -inf, -1), slots j >= K hold +inf and are never
// the worst.  Only the worst entry is tracked (slot wj, value thr, column
// thr_n); a candidate that ranks ahead of it replaces it.  The list is sorted
// once, when the row is written.

// replace slot wj by (x, n)
__device__ __forceinline__ void list_replace(float (&tv)[kMaxTop], int (&tn)[kMaxTop], int wj, float x, int n)
{
#pragma unroll
    for (int j = 0; j < kMaxTop; ++j) {
        const bool h = j == wj;
        tv[j] = h ? x : tv[j];
        tn[j] = h ? n : tn[j];
    }
}

// the worst entry: the smallest value, among equal values the largest grid
// index (the empty marker -1 ranks last); grid indices are loaded only when
// several entries share the smallest value
__device__ __forceinline__ void list_worst(const float (&tv)[kMaxTop], const int (&tn)[kMaxTop], const int *order,
                                           int &wj, float &thr, int &thr_n)
{
    float wv = tv[0];
#pragma unroll
    for (int j = 1; j < kMaxTop; ++j) wv = fminf(wv, tv[j]);
    int w = 0, wn = tn[0];
    bool found = false, tie = false;
#pragma unroll
    for (int j = 0; j < kMaxTop; ++j) {
        const bool eq = tv[j] == wv;
        tie = tie || (eq && found);
        w = (eq && !found) ? j : w;
        wn = (eq && !found) ? tn[j] : wn;
        found = found || eq;
    }
    if (tie) {
        int wg = -1;
#pragma unroll
        for (int j = 0; j < kMaxTop; ++j)
            if (tv[j] == wv) {
                const int g = gidx(order, tn[j]);
                if (g > wg) {
                    wg = g;
                    w = j;
                    wn = tn[j];
                }
            }
    }
    wj = w;
    thr = wv;
    thr_n = wn;
}

// sort the list for output: value descending, grid index ascending; slots
// j >= k (unused) go last; g receives the grid indices (empty: 0x7fffffff)
__device__ __forceinline__ void list_sort(float (&tv)[kMaxTop], int (&g)[kMaxTop], const int (&tn)[kMaxTop], int k,
                                          const int *order)
{
#pragma unroll
    for (int j = 0; j < kMaxTop; ++j) {
        g[j] = j < k ? gidx(order, tn[j]) : 0x7fffffff;
        if (j >= k) tv[j] = -INFINITY;
    }
#pragma unroll
    for (int r = 0; r < kMaxTop; ++r)
#pragma unroll
        for (int j = r & 1; j + 1 < kMaxTop; j += 2) {
            const bool sw = tv[j + 1] > tv[j] || (tv[j + 1] == tv[j] && g[j + 1] < g[j]);
            const float v0 = tv[j], v1 = tv[j + 1];
            const int g0 = g[j], g1 = g[j + 1];
            tv[j] = sw ? v1 : v0;
            tv[j + 1] = sw ? v0 : v1;
            g[j] = sw ? g1 : g0;
            g[j + 1] = sw ? g0 : g1;
        }
}

// ---- the kernel -------------------------------------------------------------
template <int EPI, bool A_F32>
__global__ void __launch_bounds__(kThreads, 1) umma_tn_kernel(const __grid_constant__ CUtensorMap tmB, UmmaArgs a)
{
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                            ~static_cast<uintptr_t>(1023));
    const uint32_t sbase = su32(smem);
    const uint32_t sA = sbase + kOffA, sB = sbase + kOffB;
    const uint32_t bars = sbase + kOffBar;
    auto b_full = [&](int s) { return bars + 8u * s; };
    auto b_empty = [&](int s) { return bars + 8u * (kStages + s); };
    auto a_full = [&](int c) { return bars + 8u * (2 * kStages + c); };
    auto a_empty = [&](int c) { return bars + 8u * (2 * kStages + kAChunks + c); };
    auto acc_full = [&](int i) { return bars + 8u * (2 * kStages + 2 * kAChunks + i); };
    auto acc_empty = [&](int i) { return bars + 8u * (2 * kStages + 2 * kAChunks + 2 + i); };
    const uint32_t mma_done = bars + 8u * (2 * kStages + 2 * kAChunks + 4);
    const uint32_t mrg_full = mma_done + 8u, mrg_empty = mma_done + 16u;  // top-K merge buffer hand-off
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc);
    volatile int *abort = reinterpret_cast<volatile int *>(smem + kOffMisc + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mt = (a.M + kBM - 1) / kBM, n_nt = (a.N + kBN - 1) / kBN;
    const int n_kc = (a.K + kBK - 1) / kBK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            bar_init(b_full(s), 1);
            bar_init(b_empty(s), 1);
        }
        for (int c = 0; c < kAChunks; ++c) {
            bar_init(a_full(c), 4 * 32);
            bar_init(a_empty(c), 1);
        }
        for (int i = 0; i < 2; ++i) {
            bar_init(acc_full(i), 1);
            bar_init(acc_empty(i), kEpiThreads);
        }
        bar_init(mma_done, 1);
        bar_init(mrg_full, (kEpiGroups - 1) * 128);
        bar_init(mrg_empty, 128);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (EPI == EPI_TOPK && threadIdx.x < kEpiGroups * kBM)
        reinterpret_cast<float *>(smem + kOffThr)[threadIdx.x] = -INFINITY;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(su32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            int s = 0;
            uint32_t ph = 0, issued = 0, issued_ph = 0;
            bool ok = !a.hold_producer;
            for (int mt = blockIdx.x; mt < n_mt && ok; mt += gridDim.x)
                for (int nt = 0; nt < n_nt && ok; ++nt)
                    for (int kc = 0; kc < n_kc && ok; ++kc) {
                        ok = bar_wait(b_empty(s), ph ^ 1, abort, a.fault);
                        if (!ok) break;
                        bar_expect_tx(b_full(s), kBStageBytes);
                        if (ANTS_IN_RANGE(a.dbg, s, kStages, 302))
                            tma_load_2d(sB + s * kBStageBytes, &tmB, kc * kBK, nt * kBN, b_full(s));
                        issued |= 1u << s;
                        issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
                        if (++s == kStages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
            // every copy issued has landed before the block may exit
            for (int t = 0; t < kStages; ++t)
                if (issued & (1u << t)) bar_drain(b_full(t), (issued_ph >> t) & 1, a.fault);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            int s = 0, j = 0;
            uint32_t ph = 0;
            uint32_t apar = 0;  // parity of each A chunk slot's next fill
            bool ok = true;
            for (int mt = blockIdx.x; mt < n_mt && ok; mt += gridDim.x) {
                for (int nt = 0; nt < n_nt && ok; ++nt, ++j) {
                    const int ab = j & 1;
                    const uint32_t use = (uint32_t)(j >> 1);
                    ok = bar_wait(acc_empty(ab), (use & 1) ^ 1, abort, a.fault);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(ab * kBN);
                    for (int kc = 0; kc < n_kc; ++kc) {
                        const int c = kc % kAChunks;  // A chunk slot (K > 256 only with one n-tile)
                        if (nt == 0) {
                            ok = bar_wait(a_full(c), (apar >> c) & 1u, abort, a.fault);
                            if (!ok) break;
                            apar ^= 1u << c;
                        }
                        ok = bar_wait(b_full(s), ph, abort, a.fault);
                        if (!ok) break;
                        tc_fence_after();
                        const int ksteps = min(kBK / 16, (a.K - kc * kBK + 15) / 16);
                        for (int ks = 0; ks < ksteps; ++ks)
                            if (ANTS_IN_RANGE(a.dbg, c * kAChunkBytes + ks * 32, kAChunks * kAChunkBytes, 303) &&
                                ANTS_IN_RANGE(a.dbg, ab * kBN + kBN - 1, 512, 304))
                                umma(d, sdesc(sA + c * kAChunkBytes + ks * 32), sdesc(sB + s * kBStageBytes + ks * 32),
                                     (kc | ks) != 0);
                        umma_commit(b_empty(s));
                        if (nt == n_nt - 1) umma_commit(a_empty(c));
                        if (++s == kStages) {
                            s = 0;
                            ph ^= 1;
                        }
                    }
                    if (!ok) break;
                    umma_commit(acc_full(ab));
                }
            }
            // every product issued has completed before the block may exit
            umma_commit(mma_done);
            bar_drain(mma_done, 0, a.fault);
        }
        __syncwarp();
    } else if (warp < kEpiWarp0) {
        // ---------------- A loaders (FP32 -> BF16, or BF16) ----------------
        const int lt = threadIdx.x - kLoaderWarp0 * 32;  // 0..127
        uint32_t apar = 0;  // parity of each chunk slot's next fill
        bool ok = true;
        for (int mt = blockIdx.x; mt < n_mt && ok; mt += gridDim.x) {
            const long m0 = (long)mt * kBM;
            for (int kc = 0; kc < n_kc && ok; ++kc) {
                const int c = kc % kAChunks;
                ok = bar_wait(a_empty(c), ((apar >> c) & 1u) ^ 1u, abort, a.fault);
                if (!ok) break;
                apar ^= 1u << c;
#pragma unroll 1
                for (int half = 0; half < 2; ++half) {
                    uint4 packed[4];
                    if (A_F32) {
                        float4 lo[4], hi[4];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int item = lt + 128 * (4 * half + q), r = item >> 3, c8 = item & 7;
                            const long m = m0 + r;
                            const int k = kc * kBK + c8 * 8;
                            if (m < a.M && k < a.K) {
                                const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(a.A) +
                                                                                   (size_t)m * a.K + k);
                                lo[q] = __ldcs(p);
                                hi[q] = __ldcs(p + 1);
                            } else {
                                lo[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                                hi[q] = lo[q];
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            __nv_bfloat162 h0 = __floats2bfloat162_rn(lo[q].x, lo[q].y);
                            __nv_bfloat162 h1 = __floats2bfloat162_rn(lo[q].z, lo[q].w);
                            __nv_bfloat162 h2 = __floats2bfloat162_rn(hi[q].x, hi[q].y);
                            __nv_bfloat162 h3 = __floats2bfloat162_rn(hi[q].z, hi[q].w);
                            packed[q] = make_uint4(*reinterpret_cast<uint32_t *>(&h0), *reinterpret_cast<uint32_t *>(&h1),
                                                   *reinterpret_cast<uint32_t *>(&h2), *reinterpret_cast<uint32_t *>(&h3));
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int item = lt + 128 * (4 * half + q), r = item >> 3, c8 = item & 7;
                            const long m = m0 + r;
                            const int k = kc * kBK + c8 * 8;
                            packed[q] = make_uint4(0u, 0u, 0u, 0u);
                            if (m < a.M && k < a.K)
                                packed[q] = __ldcs(reinterpret_cast<const uint4 *>(
                                    static_cast<const __nv_bfloat16 *>(a.A) + (size_t)m * a.K + k));
                        }
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int item = lt + 128 * (4 * half + q), r = item >> 3, c8 = item & 7;
                        const uint32_t dst = sA + c * kAChunkBytes + r * 128 + ((c8 ^ (r & 7)) << 4);
                        if (ANTS_IN_RANGE(a.dbg, dst - sA + 15, kAChunks * kAChunkBytes, 301))
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(dst), "r"(packed[q].x),
                                         "r"(packed[q].y), "r"(packed[q].z), "r"(packed[q].w)
                                         : "memory");
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_arrive(a_full(c));
            }
        }
    } else {
        // ---------------- epilogue ----------------
        const int ew = warp - kEpiWarp0, grp = ew >> 2, quarter = warp & 3;
        const int row = quarter * 32 + lane, et = ew * 32 + lane;  // et mod 128 names the row's slot
        const uint32_t tl = tmem + ((uint32_t)(quarter * 32) << 16);
        // staged values [kChunk][kEpiThreads]; at the end of a band the threads
        // of groups 1-3 leave their lists in their own slots (entry q: value in
        // row q, column in row kMaxTop + q) for the group-0 thread on that row
        float *cand = reinterpret_cast<float *>(smem + kOffCand);
        // each row's four groups publish the value of their list's worst entry:
        // a score below another group's is not in the row's top-K (that group
        // holds K entries above it); stale values are lower, so still safe
        volatile float *s_thr = reinterpret_cast<volatile float *>(smem + kOffThr);
        const int my_thr = grp * kBM + row;
        int j = 0, it = 0;
        bool ok = true;
        for (int mt = blockIdx.x; mt < n_mt && ok; mt += gridDim.x, ++it) {
            const long m = (long)mt * kBM + row;
            const uint32_t par = (uint32_t)(it & 1);
            float tv[kMaxTop];
            int tn[kMaxTop];
#pragma unroll
            for (int q = 0; q < kMaxTop; ++q) {
                tv[q] = q < a.topk ? -INFINITY : INFINITY;
                tn[q] = -1;
            }
            float thr = -INFINITY;  // the worst entry's value (the k-th so far) ...
            int thr_n = -1, wj = 0;  // ... its column and slot
            if (EPI == EPI_TOPK && grp > 0) {
                // group 0 has read this thread's list of the previous band
                if (!(ok = bar_wait(mrg_empty, par ^ 1, abort, a.fault))) break;
            }
            for (int nt = 0; nt < n_nt; ++nt, ++j) {
                const int ab = j & 1;
                const uint32_t use = (uint32_t)(j >> 1);
                ok = bar_wait(acc_full(ab), use & 1, abort, a.fault);
                if (!ok) break;
                tc_fence_after();
#pragma unroll 1
                for (int h = 0; h < kGroupCols / 32; ++h) {
                    const int col0 = grp * kGroupCols + h * 32;
                    uint32_t v[32];
                    if (ANTS_IN_RANGE(a.dbg, ab * kBN + col0 + 31, 512, 305)) {
                        tmem_ld32(tl + (uint32_t)(ab * kBN + col0), v);
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q) v[q] = 0u;
                    }
                    if (h == kGroupCols / 32 - 1) {
                        tc_fence_before();
                        bar_arrive(acc_empty(ab));
                    }
                    const int n0 = nt * kBN + col0;
                    if (EPI == EPI_TOPK) {
                        // a band's first chunk fills the empty list with its first K
                        // values directly; the others are candidates as usual
                        uint32_t skip = 0;
                        if (nt == 0 && h == 0 && n0 + 32 <= a.N) {
#pragma unroll
                            for (int q = 0; q < kMaxTop; ++q)
                                if (q < a.topk) {
                                    tv[q] = __uint_as_float(v[q]);
                                    tn[q] = n0 + q;
                                }
                            list_worst(tv, tn, a.order, wj, thr, thr_n);
                            s_thr[my_thr] = thr;
                            skip = (1u << a.topk) - 1u;
                        }
                        // candidates: values not below the k-th (ties are ranked
                        // by grid index below) nor below another group's k-th
                        float tsh = thr;
#pragma unroll
                        for (int g2 = 0; g2 < kEpiGroups; ++g2)
                            if (g2 != grp) tsh = fmaxf(tsh, s_thr[g2 * kBM + row]);
                        uint32_t mask = 0;
                        if (n0 + 32 <= a.N) {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                asm("{ .reg .pred p; setp.ge.f32 p, %1, %2; @p or.b32 %0, %0, %3; }"
                                    : "+r"(mask)
                                    : "f"(__uint_as_float(v[q])), "f"(tsh), "r"(1u << q));
                        } else {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                mask |= (n0 + q < a.N && __uint_as_float(v[q]) >= tsh) ? (1u << q) : 0u;
                        }
                        mask &= ~skip;
                        if (__any_sync(0xffffffffu, mask != 0)) {
#pragma unroll
                            for (int q = 0; q < 32; ++q)
                                if (ANTS_IN_RANGE(a.dbg, q * kEpiThreads + et, kChunk * kEpiThreads, 306))
                                    cand[q * kEpiThreads + et] = __uint_as_float(v[q]);
                            // the warp drains its lanes' candidates together
                            while (__any_sync(0xffffffffu, mask != 0)) {
                                if (mask) {
                                    const int q = __ffs(mask) - 1;
                                    mask &= mask - 1;
                                    const float x = cand[q * kEpiThreads + et];
                                    const int n = n0 + q;
                                    if (x > thr || (x == thr && gidx(a.order, n) < gidx(a.order, thr_n))) {
                                        list_replace(tv, tn, wj, x, n);
                                        list_worst(tv, tn, a.order, wj, thr, thr_n);
                                        s_thr[my_thr] = thr;
                                    }
                                }
                            }
                        }
                    } else if (EPI != EPI_BIAS_GELU) {
                        // training epilogues; the transposed copy gets each value as it is made
                        const bool in_row = m < a.M;
                        const bool tr = EPI != EPI_F32 && a.out_t != nullptr && m < a.ldT;
                        uint32_t pk[16];  // EPI_SAVE: GELU values of the row as BF16 pairs
                        float prev = 0.0f;
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const int n = n0 + q;
                            const float c = __uint_as_float(v[q]);
                            float o = 0.0f;
                            if (in_row && n < a.N && ANTS_IN_RANGE(a.dbg, (long)m * a.N + n, (long)a.M * a.N, 309)) {
                                const size_t at = (size_t)m * a.N + n;
                                if (EPI == EPI_SAVE) {
                                    const float z = c + __ldg(a.bias + n);
                                    a.zbuf[at] = z;
                                    o = gelu_f(z);
                                } else if (EPI == EPI_GELU_BWD) {
                                    o = c * gelu_grad_f(a.zbuf[at]);
                                    a.out_f[at] = o;
                                } else {
                                    o = c;
                                    a.out_f[at] = o;
                                }
                            }
                            if (tr && n < a.N && ANTS_IN_RANGE(a.dbg, (long)n * a.ldT + m, (long)a.N * a.ldT, 310))
                                a.out_t[(size_t)n * a.ldT + m] = __float2bfloat16_rn(o);
                            if (EPI == EPI_SAVE) {
                                if (q & 1) {
                                    __nv_bfloat162 hh = __floats2bfloat162_rn(prev, o);
                                    pk[q >> 1] = *reinterpret_cast<uint32_t *>(&hh);
                                } else {
                                    prev = o;
                                }
                            }
                        }
                        if (EPI == EPI_SAVE && in_row) {
                            __nv_bfloat16 *o = a.out + (size_t)m * a.N + n0;
                            for (int q = 0; q < 4 && 8 * q < a.N - n0 &&
                                            ANTS_IN_RANGE(a.dbg, (long)m * a.N + n0 + 8 * q + 7, (long)a.M * a.N, 311);
                                 ++q)
                                reinterpret_cast<uint4 *>(o)[q] =
                                    make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                        }
                    } else if (m < a.M) {
                        uint32_t pk[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const int n = n0 + 2 * q;
                            const float y0 = n < a.N ? gelu_f(__uint_as_float(v[2 * q]) + __ldg(a.bias + n)) : 0.f;
                            const float y1 =
                                n + 1 < a.N ? gelu_f(__uint_as_float(v[2 * q + 1]) + __ldg(a.bias + n + 1)) : 0.f;
                            __nv_bfloat162 hh = __floats2bfloat162_rn(y0, y1);
                            pk[q] = *reinterpret_cast<uint32_t *>(&hh);
                        }
                        __nv_bfloat16 *o = a.out + (size_t)m * a.N + n0;
                        for (int q = 0; q < 4 && 8 * q < a.N - n0 &&
                                        ANTS_IN_RANGE(a.dbg, (long)m * a.N + n0 + 8 * q + 7, (long)a.M * a.N, 308);
                             ++q)
                            reinterpret_cast<uint4 *>(o)[q] =
                                make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
                    }
                }
            }
            if (!ok) break;
            if (EPI == EPI_TOPK) {
                // the row's thresholds start the next band at -inf: each group
                // resets its own before the merge hand-off (which orders the
                // groups' bands)
                s_thr[my_thr] = -INFINITY;
                // group 0 merges the lists of the other groups' threads on its row
                if (grp > 0) {
#pragma unroll
                    for (int q = 0; q < kMaxTop; ++q)
                        if (q < a.topk) {
                            cand[q * kEpiThreads + et] = tv[q];
                            cand[(kMaxTop + q) * kEpiThreads + et] = __int_as_float(tn[q]);
                        }
                    bar_arrive(mrg_full);
                } else {
                    ok = bar_wait(mrg_full, par, abort, a.fault);
                    if (!ok) break;
                    for (int g = 1; g < kEpiGroups; ++g)
                        for (int q = 0; q < a.topk; ++q) {
                            const float x = cand[q * kEpiThreads + et + 128 * g];
                            const int n = __float_as_int(cand[(kMaxTop + q) * kEpiThreads + et + 128 * g]);
                            if (n >= 0 && ahead_of(x, gidx(a.order, n), thr, thr_n, a.order)) {
                                list_replace(tv, tn, wj, x, n);
                                list_worst(tv, tn, a.order, wj, thr, thr_n);
                            }
                        }
                    bar_arrive(mrg_empty);
                    int gi[kMaxTop];
                    list_sort(tv, gi, tn, a.topk, a.order);
                    if (m < a.M && ANTS_IN_RANGE(a.dbg, (long)m * a.topk + a.topk - 1, (long)a.M * a.topk, 307))
#pragma unroll
                        for (int q = 0; q < kMaxTop; ++q)
                            if (q < a.topk) {
                                a.top_val[(size_t)m * a.topk + q] = tv[q];
                                a.top_idx[(size_t)m * a.topk + q] = gi[q];
                            }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ---- host side --------------------------------------------------------------
typedef CUresult (*EncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

// B [N][K] BF16 row-major as 256-row x 64-column boxes, 128-byte swizzle,
// zeros outside the matrix
int encode_b(CUtensorMap *map, const __nv_bfloat16 *B, int N, int K)
{
    EncodeTiled enc = encoder();
    if (!enc) return fail(ANTS_E_CUDA, "tensor core product: cuTensorMapEncodeTiled is not available");
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)K * sizeof(__nv_bfloat16)};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBN};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(B), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(ANTS_E_INTERNAL, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ANTS_OK;
}

int check_shape(const void *A, const __nv_bfloat16 *B, int M, int N, int K)
{
    if (M < 0 || N < 1 || K < 8 || K % 8 != 0 || (K > kMaxK && N > kBN))
        return fail(ANTS_E_SHAPE,
                    "tensor core product: need K >= 8, K %% 8 == 0 and K <= %d unless N <= %d (K = %d, N = %d)", kMaxK,
                    kBN, K, N);
    if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        return fail(ANTS_E_ARG, "tensor core product: operands must be 16-byte aligned");
    return ANTS_OK;
}

template <int EPI, bool AF>
int launch(const ants_ctx *ctx, const CUtensorMap &map, const UmmaArgs &a, cudaStream_t s)
{
    static bool attr = false;  // per process; the attribute is per function
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(umma_tn_kernel<EPI, AF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBytes);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(tensor core product)");
        attr = true;
    }
    const int n_mt = (a.M + kBM - 1) / kBM;
    const int grid = n_mt < ctx->n_sm ? n_mt : ctx->n_sm;
    umma_tn_kernel<EPI, AF><<<grid, kThreads, kSmemBytes, s>>>(map, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "tensor core product launch");
    count_launch();
    return ANTS_OK;
}

}  // namespace

int mma_topk(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *B, const int *order, int M, int N,
             int K, int topk, float *val, int *idx, cudaStream_t s)
{
    if (topk < 1 || topk > kMaxTop) return fail(ANTS_E_ARG, "top-K: K must be in [1, %d]", kMaxTop);
    int rc = check_shape(A, B, M, N, K);
    if (rc != ANTS_OK || M == 0) return rc;
    CUtensorMap map;
    rc = encode_b(&map, B, N, K);
    if (rc != ANTS_OK) return rc;
    UmmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.topk = topk;
    a.order = order;
    a.top_val = val;
    a.top_idx = idx;
    a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
    return a_f32 ? launch<EPI_TOPK, true>(ctx, map, a, s) : launch<EPI_TOPK, false>(ctx, map, a, s);
}

int mma_bias_gelu(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *B, const float *bias, int M,
                  int N, int K, __nv_bfloat16 *out, cudaStream_t s)
{
    int rc = check_shape(A, B, M, N, K);
    if (rc != ANTS_OK || M == 0) return rc;
    if (N % 8 != 0 || (reinterpret_cast<uintptr_t>(out) & 15))
        return fail(ANTS_E_SHAPE, "tensor core product: GELU output needs N %% 8 == 0 and 16-byte alignment");
    CUtensorMap map;
    rc = encode_b(&map, B, N, K);
    if (rc != ANTS_OK) return rc;
    UmmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.bias = bias;
    a.out = out;
    a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
    return a_f32 ? launch<EPI_BIAS_GELU, true>(ctx, map, a, s) : launch<EPI_BIAS_GELU, false>(ctx, map, a, s);
}

int mma_train_forward(const ants_ctx *ctx, const void *A, bool a_f32, const __nv_bfloat16 *W, const float *bias,
                      int M, int N, int K, float *z, __nv_bfloat16 *h, __nv_bfloat16 *hT, int ldT, cudaStream_t s)
{
    int rc = check_shape(A, W, M, N, K);
    if (rc != ANTS_OK || M == 0) return rc;
    if (N % 8 != 0 || K > kMaxK || (hT && ldT < M) || (reinterpret_cast<uintptr_t>(h) & 15) ||
        (reinterpret_cast<uintptr_t>(z) & 15))
        return fail(ANTS_E_SHAPE, "tensor core training forward: N %% 8, K <= %d, ldT >= M, aligned outputs", kMaxK);
    CUtensorMap map;
    rc = encode_b(&map, W, N, K);
    if (rc != ANTS_OK) return rc;
    UmmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.bias = bias;
    a.out = h;
    a.zbuf = z;
    a.out_t = hT;
    a.ldT = ldT;
    a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
    return a_f32 ? launch<EPI_SAVE, true>(ctx, map, a, s) : launch<EPI_SAVE, false>(ctx, map, a, s);
}

int mma_gelu_backward(const ants_ctx *ctx, const float *dY, const __nv_bfloat16 *Wt, const float *z, int M, int N,
                      int K, float *dz, __nv_bfloat16 *dzT, int ldT, cudaStream_t s)
{
    int rc = check_shape(dY, Wt, M, N, K);
    if (rc != ANTS_OK || M == 0) return rc;
    if (N % 8 != 0 || K > kMaxK || (dzT && ldT < M))
        return fail(ANTS_E_SHAPE, "tensor core GELU backward: N %% 8, K <= %d, ldT >= M", kMaxK);
    CUtensorMap map;
    rc = encode_b(&map, Wt, N, K);
    if (rc != ANTS_OK) return rc;
    UmmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = dY;
    a.zbuf = const_cast<float *>(z);
    a.out_f = dz;
    a.out_t = dzT;
    a.ldT = ldT;
    a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
    return launch<EPI_GELU_BWD, true>(ctx, map, a, s);
}

int mma_f32(const ants_ctx *ctx, const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, float *C,
            cudaStream_t s)
{
    int rc = check_shape(A, B, M, N, K);
    if (rc != ANTS_OK || M == 0) return rc;
    if (N % 8 != 0) return fail(ANTS_E_SHAPE, "tensor core product: FP32 output needs N %% 8 == 0");
    CUtensorMap map;
    rc = encode_b(&map, B, N, K);
    if (rc != ANTS_OK) return rc;
    UmmaArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.A = A;
    a.out_f = C;
    a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
    return launch<EPI_F32, false>(ctx, map, a, s);
}

}  // namespace ants

using namespace ants;

// Self-test of the bounded waits (no counterpart in the paper): a top-K
// product whose producer is held back must give up after its 1 s wait limit,
// report through the fault word, and leave the context usable.
extern "C" ANTS_API int ants_selftest_stalled_product(ants_ctx *ctx)
{
    begin_call();
    if (!ctx) return fail(ANTS_E_ARG, "ants_selftest_stalled_product: NULL context");
    ANTS_CUDA_TRY(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int M = 256, N = 256, K = 64;
    float *A = nullptr, *val = nullptr;
    __nv_bfloat16 *B = nullptr;
    int *order = nullptr, *idx = nullptr;
    cudaError_t e = cudaMalloc(&A, (size_t)M * K * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&B, (size_t)N * K * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMalloc(&order, N * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&val, (size_t)M * 8 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&idx, (size_t)M * 8 * sizeof(int));
    int rc = ANTS_OK;
    if (e != cudaSuccess) rc = cuda_fail(e, "self-test buffers");
    std::vector<int> ho(N);
    for (int i = 0; i < N; ++i) ho[i] = i;
    // A = 1, B = 0 except B[n][0] = n/256: every row's best column is N-1
    std::vector<float> hA((size_t)M * K, 1.0f);
    std::vector<__nv_bfloat16> hB((size_t)N * K, __float2bfloat16_rn(0.0f));
    for (int n = 0; n < N; ++n) hB[(size_t)n * K] = __float2bfloat16_rn((float)n / 256.0f);
    if (rc == ANTS_OK) {
        e = cudaMemcpy(A, hA.data(), hA.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(B, hB.data(), hB.size() * sizeof(__nv_bfloat16), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(order, ho.data(), N * sizeof(int), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(ctx->d_fault, 0, sizeof(int));
        if (e != cudaSuccess) rc = cuda_fail(e, "self-test upload");
    }
    CUtensorMap map;
    if (rc == ANTS_OK) rc = encode_b(&map, B, N, K);
    int fault_stalled = 0, fault_after = 0;
    if (rc == ANTS_OK) {
        UmmaArgs a{};
        a.M = M;
        a.N = N;
        a.K = K;
        a.A = A;
        a.topk = 8;
        a.order = order;
        a.top_val = val;
        a.top_idx = idx;
        a.fault = ctx->d_fault;
    a.dbg = ctx->d_bounds;
        a.hold_producer = 1;
        rc = launch<EPI_TOPK, true>(ctx, map, a, nullptr);
        if (rc == ANTS_OK) {
            e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaMemcpy(&fault_stalled, ctx->d_fault, sizeof(int), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess) e = cudaMemset(ctx->d_fault, 0, sizeof(int));
            if (e != cudaSuccess) rc = cuda_fail(e, "self-test (stalled launch)");
        }
        if (rc == ANTS_OK) {
            a.hold_producer = 0;
            rc = launch<EPI_TOPK, true>(ctx, map, a, nullptr);
        }
        if (rc == ANTS_OK) {
            e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaMemcpy(&fault_after, ctx->d_fault, sizeof(int), cudaMemcpyDeviceToHost);
            int best = -1;
            if (e == cudaSuccess) e = cudaMemcpy(&best, idx, sizeof(int), cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) rc = cuda_fail(e, "self-test (normal launch)");
            else if (!fault_stalled) rc = fail(ANTS_E_INTERNAL, "self-test: the stalled product did not report");
            else if (fault_after || best != N - 1)
                rc = fail(ANTS_E_INTERNAL, "self-test: the context is not usable after the timeout (%d, %d)",
                          fault_after, best);
        }
    }
    cudaFree(A);
    cudaFree(B);
    cudaFree(order);
    cudaFree(val);
    cudaFree(idx);
    return rc;
}
