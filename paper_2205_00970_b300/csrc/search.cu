// LIDER batched search (Sec. 3.3.2, Sec. 6.2) on one GPU.
//
// Steps and kernels, in order, for nq queries probing c clusters each
// (tensor score modes; SIMT mode in brackets):
//   1. hash     split_tf32 + qnorm_kernel + front_tc_kernel (3xTF32 tiles of
//               queries x [projections; centroids]: the hash values and the
//               routing scores in one launch) [dot2_tile_kernel<hash>]
//   2. route    topc_exact_kernel: the c best centroids by x.mu - |mu|^2/2,
//               ties -> lower index, exact despite approximate scores
//               [dot2_tile_kernel<score> + topc_kernel]; with the Layer-1
//               centroids retriever, route_core_kernel then routes instead;
//               hash_recheck_kernel (hash values near a bucket edge
//               recomputed exactly) + pack_kernel: packed query hashkeys for
//               the L arrays, p-stable or hyperplane (Sec. 4.1, 4.2)
//   3. group    group_*_kernel: (query, probe) pairs bucketed by cluster;
//               primary_order_kernel: queries grouped by best cluster (the
//               re-score's order)
//   4. locate   locate_kernel, one thread per (pair, array): re-scale the key
//               (Sec. 5.1), two-stage RMI prediction (Sec. 5.2), clamp
//               (Sec. 7.4, counted as OOR/LE), lower bound searched inside
//               the leaf's recorded error window (with a counted fallback
//               outside it), then the bi-directional expansion window of
//               Sec. 4 by co-rank search
//   5. gather   qgather_*_kernel (the queries in pair order, in the mode's
//               operand format) + mark_kernel (each pair's candidate union as
//               a bitmap over its cluster's positions)
//   6. score    tc_units_kernel + tc_score_kernel: dense 128 x 256 tiles on
//               tcgen05 written as per-pair score rows, with per-32-position
//               candidate maxima [score_group_kernel: union, exact FP32
//               scores and per-pair top-k in one persistent kernel]
//   7. select   select_hist_kernel (per query: a threshold from a histogram
//               of the chunk maxima, the chunks that clear it read, the ks-th
//               best collected score by a radix select, the guard band below
//               it kept) and select_query_kernel (fallback for massive ties)
//   8. merge    rescore_kernel: exact FP32 scores of each query's list, sorted
//               [merge_kernel: k-way merge of the c per-pair lists]

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lider_internal.cuh"
#include "tc.cuh"

namespace lider {

namespace {

constexpr int kScoreThreads = 256;

// counters[] slots
enum {
    CNT_QBOUNDARY = 0,
    CNT_QCLAMPED,
    CNT_FALLBACK,
    CNT_CANDIDATES,
    CNT_EMPTY,
    CNT_ITEM,       // persistent-kernel work counter
    CNT_ROUTE_FALLBACK,
    CNT_BOUNDS,     // accesses skipped by a failed bounds check (must stay 0)
    CNT_SEL_OVERFLOW,  // queries whose guarded candidate band did not fit (result may be inexact)
    CNT_OOR,        // RMI predictions at either end of the array (Sec. 7.4)
    CNT_LE,         // RMI predictions more than k from the lower bound
    CNT_OOR_LE,     // both
    CNT_QORDER,     // queries placed by primary_order_kernel
    CNT_SLOTS = 13
};

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) once per (kernel, device,
// size): a search repeated under stream capture then makes no such call.
std::mutex g_attr_mutex;
std::map<std::pair<const void*, int>, int> g_attr_set;

int smem_attr(const void* fn, int bytes) {
    int dev = 0;
    LIDER_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    int& have = g_attr_set[{fn, dev}];
    if (have >= bytes) return LIDER_OK;
    LIDER_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    have = bytes;
    return LIDER_OK;
}

inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ------------------------------------------------------------------ route --
// Warp per query: the c best (score desc, index asc) of ncl FP64 scores.
__global__ void topc_kernel(const double* __restrict__ S, int64_t nq, int ncl, int c,
                            int32_t* __restrict__ route, int32_t* __restrict__ trace_route) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const double* s = S + q * ncl;
    double ps = INFINITY;
    int pj = -1;
    for (int r = 0; r < c; ++r) {
        double best = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < ncl; j += 32) {
            double v = s[j];
            if (v != v) v = -INFINITY;                            // NaN ranks last
            const bool after = (v < ps) || (v == ps && j > pj);   // strictly after the last pick
            if (after && (v > best || (v == best && j < bj))) { best = v; bj = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
        }
        if (bj >= ncl) bj = 0;                                    // unreachable: c <= ncl
        ps = best;
        pj = bj;
        if (lane == 0) {
            route[q * c + r] = bj;
            if (trace_route) trace_route[q * c + r] = bj;
        }
    }
}

// Tensor-core routing (tensor score modes).  Approximate scores
// q.mu - |mu|^2/2 of every (query, centroid) come from 128 x 256 tiles of the
// tcgen05 engine (three TF32 products per FP32 product); a warp per query then
// takes the c + kRouteExtra best, scores them again exactly (Dot2, finished in
// FP64) and keeps the c best by exact score (ties -> lower index).  If the
// best approximate score left out of the shortlist is within the tensor-core
// error guard of the c-th exact score, every centroid of that query is scored
// exactly instead.
constexpr int kRouteExtra = 8;
// topc_exact_kernel stages a query's routing scores in shared memory when the
// row has at most this many centroids (8 warps x 4 KB per block)
constexpr int kTopcStageCols = 1024;
// Bound on the error of one 3xTF32 tensor-core score, relative to |q| |x|
// (the product of the two norms).  The dropped lo*lo term and the TF32
// rounding of the tails contribute about 3 * 2^-22 of sum |q_i x_i| <= |q| |x|;
// with the tensor cores' FP32 accumulation the engine tests measure less than
// 2e-6 of sum |q_i x_i| up to d = 784, so 3e-5 leaves a wide margin.  The
// route and candidate guards use it.
constexpr float kTcGuard = 3e-5f;

// ----------------------------------------------------------- hash + route --
// Both the hash values t = (a_h . q + b_h) / W and the routing scores
// q.mu - |mu|^2/2 are contractions of the queries with a fixed matrix, so one
// launch of the tcgen05 engine (three TF32 products per FP32 product) runs
// them together over the front operand F: rows [0, H) are the projections,
// rows [Hp, Hp + ncl) the centroids (Hp = H rounded up to 256; the rows
// between are zero), and every 256-row tile of F is either a hash tile or a
// route tile.  The tiles of one query tile are adjacent in the schedule, so
// its queries are read from L2 by the CTAs that share them.
//
// Hash tiles: where floor(t) could depend on the tile's error (t within its
// bound, or within 1e-6 for the boundary count, of an integer; of zero for
// hyperplane hashes, whose b is 0 and W 1) the (query, projection) goes to a
// list, and hash_recheck_kernel recomputes t with exactly the arithmetic of
// the SIMT hashing kernel (sequential Dot2 over k, finished in FP64), so the
// query keys are the same bit for bit on every score path.
// Route tiles: approximate scores for topc_exact_kernel.
struct FrontSched {
    int nq;
    int nth, ntr;               // hash tiles (Hp / 256) and route tiles per query tile
    int Hp;
    __device__ int count() const { return ((nq + 127) / 128) * (nth + ntr); }
    __device__ void coords(int u, int& arow, int& brow) const {
        const int nt = nth + ntr, t = u % nt;
        arow = (u / nt) * 128;
        brow = t < nth ? t * 256 : Hp + (t - nth) * 256;
    }
};

struct FrontEpi {
    // hash tiles
    double* t;                  // nq x H
    const float* b;             // offsets b_h
    const float* a_norm;        // |a_h|
    const float* qnorm;         // |q| (rounded up)
    int32_t* recheck;           // ((q0 + q) * H + h) of the undecided values
    int32_t* n_recheck;
    float W, guard;             // guard: kTcGuard
    int H;
    int q0;                     // index of this launch's first query in the whole batch
    bool hyper;                 // hyperplane hashes: only the sign of t decides
    // route tiles
    float* S;                   // nq x ncl approximate scores
    const double* half_norm;
    int ncl;
    int nq, nth, ntr;
    // this tile and row
    int q, n0;
    bool hash;
    float qn;
    __device__ void begin(int u, int row) {
        const int nt = nth + ntr, tt = u % nt;
        q = (u / nt) * 128 + row;
        hash = tt < nth;
        n0 = (hash ? tt : tt - nth) * 256;
        qn = (hash && q < nq) ? qnorm[q] : 0.f;
    }
    __device__ void operator()(int, int, int col0, const uint32_t (&v)[32]) {
        if (q >= nq) return;
        if (hash) {
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
                const int h = n0 + col0 + i;
                if (h >= H) break;
                const float acc = __uint_as_float(v[i]);
                const float bh = b[h];
                const float tf = __fdiv_rn(__fadd_rn(acc, bh), W);
                // |tf - t| <= (tile error + FP32 rounding of acc + b) / W + rounding of the division
                const float eps = __fdiv_rn(guard * qn * a_norm[h] + 4.f * 0x1p-24f * (fabsf(acc) + fabsf(bh)), W) +
                                  0x1p-22f * fabsf(tf);
                const float dist = hyper ? fabsf(tf) : fabsf(tf - rintf(tf));
                t[(int64_t)q * H + h] = (double)tf;
                if (!(dist > 1.01f * eps + 1.1e-6f)) recheck[atomicAdd(n_recheck, 1)] = (q0 + q) * H + h;
            }
        } else {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int j = n0 + col0 + i;
                if (j < ncl) S[(int64_t)q * ncl + j] = __uint_as_float(v[i]) - (float)half_norm[j];
            }
        }
    }
    __device__ void done(int, int) {}
};

__global__ void __launch_bounds__(tc::kThreads, 1)
    front_tc_kernel(const __grid_constant__ CUtensorMap mQhi, const __grid_constant__ CUtensorMap mQlo,
                    const __grid_constant__ CUtensorMap mFhi, const __grid_constant__ CUtensorMap mFlo, int kchunks,
                    FrontSched sched, FrontEpi epi, int* err) {
    extern __shared__ unsigned char smem[];
    __shared__ tc::Ctl ctl;
    tc::gemm_tiles<tc::KindTf32x3>(&mQhi, &mQlo, &mFhi, &mFlo, kchunks, sched, epi, err, smem, ctl);
}

// t of the listed (query, projection) values, with the SIMT hashing kernel's
// arithmetic: Dot2 steps over k = 0..d-1 in order, FP64 finish.  One warp
// per value: the warp stages both rows in shared memory (2 d floats, dynamic)
// and lane 0 runs the sequential Dot2 from there.
__global__ void __launch_bounds__(32) hash_recheck_kernel(const float* __restrict__ Q, const float* __restrict__ A,
                                                          const float* __restrict__ b, double W, int d, int H,
                                                          const int32_t* __restrict__ recheck,
                                                          const int32_t* __restrict__ n_recheck,
                                                          double* __restrict__ t) {
    extern __shared__ float rows[];        // x[0..d), a[0..d)
    const int n = *n_recheck;
    const int lane = threadIdx.x;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int idx = recheck[i];
        const int64_t q = idx / H;
        const int h = idx - (int)q * H;
        const float* x = Q + q * d;
        const float* a = A + (int64_t)h * d;
        for (int k = lane; k < d; k += 32) {
            rows[k] = x[k];
            rows[d + k] = a[k];
        }
        __syncwarp();
        if (lane == 0) {
            Dot2 acc{0.f, 0.f};
            for (int k = 0; k < d; ++k) dot2_step(acc, rows[k], rows[d + k]);
            t[idx] = __ddiv_rn(__dadd_rn(dot2_value(acc), (double)b[h]), W);
        }
        __syncwarp();
    }
}

// |q| per query, rounded up (warp per query).
__global__ void qnorm_kernel(const float* __restrict__ Q, int64_t nq, int d, float* __restrict__ out) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    // every step rounds up and every term is non-negative, so the FP32 sum
    // bounds the exact sum of squares from above (no FP64: its rate is low here)
    float s = 0.f;
    for (int i = lane; i < d; i += 32) {
        const float v = Q[q * d + i];
        s = __fmaf_ru(v, v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s = __fadd_ru(s, __shfl_xor_sync(0xffffffffu, s, o));
    if (lane == 0) out[q] = __fsqrt_ru(s);
}

// Merge the 32 lanes' Dot2 accumulators (s, c) by TwoSum in a fixed
// butterfly order; every lane ends with the same pair.  FP32 throughout: the
// FP64 rate of this GPU is a small fraction of its FP32 rate.
__device__ __forceinline__ void warp_merge_dot2(Dot2& a) {
    for (int o = 16; o > 0; o >>= 1) {
        const float os = __shfl_xor_sync(0xffffffffu, a.s, o);
        const float oc = __shfl_xor_sync(0xffffffffu, a.c, o);
        const float t = __fadd_rn(a.s, os);
        const float z = __fadd_rn(t, -a.s);
        const float e = __fadd_rn(__fadd_rn(a.s, -__fadd_rn(t, -z)), __fadd_rn(os, -z));   // a.s + os = t + e
        a.s = t;
        a.c = __fadd_rn(__fadd_rn(a.c, oc), e);
    }
}

// Order-preserving 64-bit key of an FP64 score (ascending in the score;
// NaN as -inf), compared with integer instructions.
__device__ __forceinline__ uint64_t score_key(double v) {
    uint64_t u = (uint64_t)__double_as_longlong(v);
    if ((u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) u = 0xfff0000000000000ull;   // NaN -> -inf
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// q.mu - |mu|^2/2 by one warp in compensated arithmetic: per-lane Dot2 over
// elements lane, lane + 32, ..., lanes merged by TwoSum, FP64 finish.
__device__ __forceinline__ double warp_exact_score(const float* __restrict__ q, const float* __restrict__ mu, int d,
                                                   double half_norm) {
    const int lane = threadIdx.x & 31;
    Dot2 acc{0.f, 0.f};
#pragma unroll 8
    for (int i = lane; i < d; i += 32) dot2_step(acc, __ldg(q + i), __ldg(mu + i));
    warp_merge_dot2(acc);
    return __dadd_rn(dot2_value(acc), -half_norm);
}

// warp_exact_score of four centroids at once (the same arithmetic per
// centroid, so the same values; their loads overlap).  Centroid t is
// C + rows[t] * d.
__device__ __forceinline__ void warp_exact_scores4(const float* __restrict__ q, const float* __restrict__ C,
                                                   const int (&rows)[4], int d, const double* __restrict__ half_norm,
                                                   double (&out)[4]) {
    const int lane = threadIdx.x & 31;
    Dot2 acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const float* mu[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) mu[t] = C + (int64_t)rows[t] * d;
#pragma unroll 2
    for (int i = lane; i < d; i += 32) {
        const float qi = __ldg(q + i);
        float m[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) m[t] = __ldg(mu[t] + i);
#pragma unroll
        for (int t = 0; t < 4; ++t) dot2_step(acc[t], qi, m[t]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        warp_merge_dot2(acc[t]);
        out[t] = __dadd_rn(dot2_value(acc[t]), -half_norm[rows[t]]);
    }
}

// Guard formula of a score mode (see candidate_guard).
inline int guard_mode(int score_mode) {
    return score_mode == LIDER_SCORE_TENSOR ? 1 : score_mode == LIDER_SCORE_F16 ? 2
                                                : score_mode == LIDER_SCORE_FP8 ? 3 : 0;
}

// Power of two sq with sq * amax in [2^13, 2^14) (1 for amax == 0): the
// FP16 path's query scale.
__device__ __forceinline__ float f16_query_scale(float amax) {
    if (!(amax > 0.f) || !(amax <= 3.0e38f)) return 1.f;
    int e = 0;
    frexpf(amax, &e);
    e = max(-100, min(e, 127));
    return ldexpf(1.f, 14 - e);
}

// Per-query scale and error bound of the approximate candidate scores.
// qn: |q| as computed in FP32 (inflated here to bound the true norm).
// gmode 1 (3xTF32): guard = kTcGuard |q| |x|max.
// gmode 2 (FP16): q and x are scaled by powers of two sq, sx and rounded to
// FP16; with e_q = fp16(sq q) - sq q and e_x = fp16(sx x) - sx x (their norms
// measured exactly: eq for this query, xres for the worst row), and the
// products exact in FP32,
//   fp16(sq q) . fp16(sx x) - sq sx q.x = e_q . fp16(sx x) + sq q . e_x,
// bounded by eq |x^|max + sq |q| xres; the tensor cores sum the d products
// with an error below d 2^-23 of their absolute sum <= (sq |q| + eq) |x^|max.
// gmode 0 (served BF16 form): no guard.  qbound bounds |approximate score|
// (it sets the select histogram's range).
// FP32 throughout, every rounding upward (products by powers of two are
// exact), so each result bounds its exact expression from above; this GPU's
// FP64 rate is a small fraction of its FP32 rate.
__device__ void candidate_guard(int gmode, float qn, float sq, float eq, int d, float xmax, float sx,
                                float xres, float xhat, float* qscale, float* qguard, float* qbound) {
    const float q = __fmul_ru(qn, 1.00001f);
    float g = 0.f, s = 1.f;
    if (gmode == 1) {
        g = __fmul_ru(__fmul_ru(kTcGuard, q), xmax);
    } else if (gmode == 0) {
        g = __fmul_ru(0x1p-6f * q, xmax);              // BF16: only bounds the scores below
    } else if (gmode == 3) {
        g = __fmul_ru(__fmul_ru(0.3f, q), xmax);       // FP8: only bounds the scores below
    } else if (gmode == 2) {
        const float acc = (float)d * 0x1p-23f;
        const float qs = sq * q;
        g = __fadd_ru(__fadd_ru(__fmul_ru(eq, xhat), __fmul_ru(qs, xres)),
                      __fmul_ru(__fmul_ru(acc, __fadd_ru(qs, eq)), xhat));
        s = sq * sx;
    }
    // |approximate score| <= s |q| |x|max + its error (s = 1 unless FP16)
    const float B = __fmul_ru(__fadd_ru(__fmul_ru(s * q, xmax), g), 1.f + 0x1p-20f);
    *qscale = gmode == 2 ? sq : 1.f;
    // the select reads scores as 16-bit codes over [-B, B] (score_code), each
    // within 0.51 of a step 2B/65535 of the score: one step joins the guard
    *qguard = (gmode == 0 || gmode == 3) ? 0.f
                                         : __fmul_ru(__fadd_ru(g, __fdiv_ru(2.f * B, 65535.f)), 1.f + 0x1p-20f);
    *qbound = B;
}

// 16-bit score codes of the tensor paths: code = rint((B - s) * 65535 / 2B),
// saturated to [0, 65535], for |s| <= B (B = qbound of the query; the score
// kernel's score_code_sat); code_score maps a code back (B - code * 2B/65535).
// Every kernel maps codes back with code_score, so a code means the same
// float everywhere, and the float decreases as the code grows.
__device__ __forceinline__ float code_step(float B) { return __fdiv_rn(__fmul_rn(2.f, B), 65535.f); }
__device__ __forceinline__ float code_score(uint32_t code, float B, float step) {
    return __fsub_rn(B, __fmul_rn((float)code, step));
}

__global__ void topc_exact_kernel(const float* __restrict__ S, const float* __restrict__ Q,
                                  const float* __restrict__ C, const double* __restrict__ half_norm, int64_t nq,
                                  int ncl, int d, int c, float guard_scale, int32_t* __restrict__ route,
                                  int32_t* __restrict__ trace_route, int gmode, float max_xnorm, float x_scale,
                                  float xres_max, float xhat_max,
                                  float* __restrict__ qscale, float* __restrict__ qguard, float* __restrict__ qbound,
                                  unsigned long long* fallbacks) {
    constexpr unsigned kFull = 0xffffffffu;
    extern __shared__ float s_rows[];      // per warp: its query's ncl scores (when staged)
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const float* srow = S + q * ncl;
    if (ncl <= kTopcStageCols) {
        // every round below scans the row: stage it once (same values, same order)
        float* own = s_rows + (threadIdx.x >> 5) * ncl;
        for (int j = lane; j < ncl; j += 32) own[j] = srow[j];
        __syncwarp();
        srow = own;
    }
    const float* qv = Q + q * d;
    const int nsl = min(c + kRouteExtra, ncl);
    // shortlist: the nsl best approximate scores (ties -> lower index), built
    // in rounds; the first c + 1 usually settle the route (see below).
    // Entry e (e < nsl <= 40) is held by lane e % 32 in register slot e / 32.
    int sl0 = 0, sl1 = 0;
    float av0 = -INFINITY, av1 = -INFINITY;
    float ps = INFINITY;
    int pj = -1;
    auto next_best = [&](int r) {
        float best = -INFINITY;
        int bj = 0x7fffffff;
        for (int j = lane; j < ncl; j += 32) {
            float v = srow[j];
            if (v != v) v = -INFINITY;
            const bool after = (v < ps) || (v == ps && j > pj);
            if (after && (v > best || (v == best && j < bj))) { best = v; bj = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(kFull, best, o);
            const int oj = __shfl_xor_sync(kFull, bj, o);
            if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
        }
        if (bj >= ncl) bj = 0;
        ps = best;
        pj = bj;
        if ((r & 31) == lane) {
            if (r < 32) { sl0 = bj; av0 = best; } else { sl1 = bj; av1 = best; }
        }
    };
    auto entry_sl = [&](int e) { return __shfl_sync(kFull, e < 32 ? sl0 : sl1, e & 31); };
    const int n_first = min(c + 1, nsl);
#pragma unroll 1
    for (int r = 0; r < n_first; ++r) next_best(r);
    float qn2 = 0.f, amax = 0.f;
    for (int i = lane; i < d; i += 32) {
        const float v = qv[i];
        qn2 = fmaf(v, v, qn2);
        amax = fmaxf(amax, fabsf(v));
    }
    for (int o = 16; o > 0; o >>= 1) {
        qn2 += __shfl_xor_sync(kFull, qn2, o);
        amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, o));
    }
    const float guard = guard_scale * sqrtf(qn2);
    // FP16 path: the query's scale and the norm of its rounding residual
    const float sq = gmode == 2 ? f16_query_scale(amax) : 1.f;
    // (r = fp16(v) - v is exact in FP32; the FP32 sum of the d squares is
    // inflated by (1 + (d + 32) 2^-23) to bound the exact one)
    float eq2 = 0.f;
    if (gmode == 2) {
        for (int i = lane; i < d; i += 32) {
            const float v = qv[i] * sq;
            const float r = __half2float(__float2half_rn(v)) - v;
            eq2 = fmaf(r, r, eq2);
        }
        for (int o = 16; o > 0; o >>= 1) eq2 += __shfl_xor_sync(kFull, eq2, o);
    }
    const float eq = __fsqrt_ru(__fmul_ru(eq2, __fadd_ru(1.f, (float)(d + 32) * 0x1p-23f)));
    if (lane == 0)
        candidate_guard(gmode, sqrtf(qn2), sq, eq, d, max_xnorm, x_scale, xres_max, xhat_max, qscale + q,
                        qguard + q, qbound + q);
    // Entries e and e + 1 are "separated" when the approximate score of e leads
    // that of e + 1 by more than twice the error bound: then every exact score
    // of an entry up to e exceeds every exact score after it (the gap is
    // rounded down and twice the guard is exact, so a gap that passes also
    // passes in exact arithmetic).  Maximal runs of unseparated entries keep
    // their place in the order; only their members' order is open.  So: find
    // E, the first separated entry at or after c - 1 (the top-c set is then
    // entries 0..E), score exactly the members of runs of two or more up to
    // E, and order each such run by exact score (ties -> lower index).  When
    // the shortlist ends before such an E, every centroid is scored exactly.
    int n_cur = n_first;
    int E = -1;
    uint64_t sep = 0ull;                      // bit e: entries e and e + 1 separated
    for (;;) {
        // entry e + 1's score, or the end of the row (nothing after: separated)
        float next0 = __shfl_down_sync(kFull, av0, 1);
        const float a32 = __shfl_sync(kFull, av1, 0);
        if (lane == 31) next0 = a32;
        const float next1 = __shfl_down_sync(kFull, av1, 1);
        const auto separated = [&](int e, float a, float nx) {
            if (e >= n_cur) return false;
            if (e + 1 >= n_cur) return n_cur == ncl;
            return __fsub_rd(a, nx) > 2.f * guard;
        };
        const unsigned m0 = __ballot_sync(kFull, separated(lane, av0, next0));
        const unsigned m1 = __ballot_sync(kFull, separated(lane + 32, av1, next1));
        sep = (uint64_t)m0 | ((uint64_t)m1 << 32);
        const uint64_t cand = sep & (~0ull << (c - 1));
        if (cand) {
            E = __ffsll((long long)cand) - 1;
            break;
        }
        if (n_cur >= nsl) break;
        next_best(n_cur++);
    }
    // No separation at or after c - 1 within the shortlist: the run holding
    // entry c - 1 reaches the shortlist's end.  Its members are scored
    // exactly as well, and the result stands when the best approximate score
    // outside the shortlist, plus the guard, stays below the exact c-th score;
    // otherwise every centroid is scored exactly.
    const bool open_tail = E < 0;
    if (open_tail) E = nsl - 1;
    int outv = 0;                             // lane r < c: the route's r-th centroid
    uint64_t kc = 0ull;                       // open tail: the exact key of the route's c-th
    {
        const uint64_t upto = (2ull << E) - 1;        // entries 0..E (E < 40)
        const uint64_t open = ~sep;                   // bit e: e and e + 1 not separated
        // members of runs of two or more: e with e - 1 or e + 1 in its run
        // (the open tail's last entry counts as unseparated from what follows)
        const uint64_t need = ((open << 1) | open) & upto;
        if (!need) {
            outv = sl0;                               // the approximate order is the exact one
        } else {
            // exact scores of the open runs' members, four at a time
            uint64_t ek0 = 0ull, ek1 = 0ull;
            uint64_t rest = need;
            while (rest) {
                int rows[4], ent[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    ent[t] = rest ? __ffsll((long long)rest) - 1 : -1;
                    if (rest) rest &= rest - 1;
                    rows[t] = entry_sl(ent[t] >= 0 ? ent[t] : ent[0]);
                }
                double e4[4];
                warp_exact_scores4(qv, C, rows, d, half_norm, e4);
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int e = ent[t];
                    if (e >= 0 && (e & 31) == lane) {
                        if (e < 32) ek0 = score_key(e4[t]); else ek1 = score_key(e4[t]);
                    }
                }
            }
            // runs end at a separated entry or at E
            const uint64_t ends = sep | (1ull << E);
            // the longest open run (warp-uniform loop bound below)
            int run_len = 0;
            for (uint64_t r = need; r;) {
                const int a = __ffsll((long long)r) - 1;
                const int b = __ffsll((long long)(ends & (~0ull << a))) - 1;    // run [a, b], b <= E
                run_len = max(run_len, b - a + 1);
                r &= (b >= 63) ? 0ull : (~0ull << (b + 1));
            }
            const uint64_t starts = (sep << 1) | 1ull;  // bit e: a run starts at e
#pragma unroll
            for (int slot = 0; slot < 2; ++slot) {
                // final place of entry e = lane + 32 slot: its run's start plus its
                // rank in the run by (exact score descending, index ascending)
                const int e = lane + 32 * slot;
                const bool mine = e <= E;
                const int a = mine ? 63 - __clzll((long long)(starts & ((2ull << e) - 1))) : 0;
                const int b = mine ? __ffsll((long long)(ends & (~0ull << e))) - 1 : -1;
                const uint64_t my_key = slot ? ek1 : ek0;
                const int my_j = slot ? sl1 : sl0;
                const bool open_e = mine && b > a;
                int rank = 0;
                for (int t = 0; t < run_len; ++t) {
                    const int f = min(a + t, 63);
                    const uint64_t k0 = __shfl_sync(kFull, ek0, f & 31), k1 = __shfl_sync(kFull, ek1, f & 31);
                    const int j0 = __shfl_sync(kFull, sl0, f & 31), j1 = __shfl_sync(kFull, sl1, f & 31);
                    const uint64_t fk = f < 32 ? k0 : k1;
                    const int fj = f < 32 ? j0 : j1;
                    if (open_e && f != e && a + t <= b && (fk > my_key || (fk == my_key && fj < my_j))) ++rank;
                }
                const int pos = mine ? a + rank : -1;
                const unsigned at_c = __ballot_sync(kFull, pos == c - 1);
                if (at_c) kc = __shfl_sync(kFull, my_key, __ffs(at_c) - 1);
                // the lane of place pos (< c) takes entry e's centroid
                const int hi = slot ? E - 32 : min(E, 31);
                for (int src = 0; src <= hi; ++src) {
                    const int p = __shfl_sync(kFull, pos, src);
                    const int jv = __shfl_sync(kFull, my_j, src);
                    if (p == lane && p < c) outv = jv;
                }
            }
        }
    }
    bool rescan = false;
    if (open_tail) {
        // the best approximate score outside the shortlist
        float best = -INFINITY;
        for (int j = lane; j < ncl; j += 32) {
            float v = srow[j];
            if (v != v) v = -INFINITY;
            const bool after = (v < ps) || (v == ps && j > pj);
            if (after && v > best) best = v;
        }
        for (int o = 16; o > 0; o >>= 1) best = fmaxf(best, __shfl_xor_sync(kFull, best, o));
        rescan = score_key((double)best + (double)guard) >= kc;
    }
    if (rescan) {
        // a centroid outside the shortlist may beat the c-th: score them all exactly
        if (lane == 0) atomicAdd(fallbacks, 1ull);
        double pe = INFINITY;
        int pjj = -1;
        for (int r = 0; r < c; ++r) {
            double best = -INFINITY;
            int bj = 0x7fffffff;
            for (int j = 0; j < ncl; ++j) {
                const double v = warp_exact_score(qv, C + (int64_t)j * d, d, half_norm[j]);
                const bool after = (v < pe) || (v == pe && j > pjj);
                if (after && (v > best || (v == best && j < bj))) { best = v; bj = j; }
            }
            if (lane == r) outv = bj < ncl ? bj : 0;
            pe = best;
            pjj = bj;
        }
    }
    if (lane < c) {
        route[q * c + lane] = outv;
        if (trace_route) trace_route[q * c + lane] = outv;
    }
}

// ------------------------------------------------------------------ group --
__global__ void group_count_kernel(const int32_t* __restrict__ route, int64_t npairs, int32_t* __restrict__ cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npairs) atomicAdd(&cnt[route[i]], 1);
}

// Single block: off = exclusive scan of cnt, item_off = exclusive scan of
// ceil(cnt / G), cursor = off.
// Tensor-core units of cluster j: ceil(cnt/128) query tiles x ceil(n_c/256) row tiles.
__device__ __forceinline__ int32_t tc_units(int32_t cnt, int64_t n_c) {
    return n_c > 0 ? ((cnt + tc::kBM - 1) / tc::kBM) * (int32_t)((n_c + tc::kBN - 1) / tc::kBN) : 0;
}

// Words of one pair's candidate bitmap over its cluster's positions.
__device__ __forceinline__ int64_t bitmap_words(int64_t n_c) { return (n_c + 31) >> 5; }

__global__ void group_scan_kernel(const int32_t* __restrict__ cnt, int ncl, int G, const int64_t* __restrict__ cl_off,
                                  int32_t* __restrict__ off, int32_t* __restrict__ cursor,
                                  int32_t* __restrict__ item_off, int32_t* __restrict__ unit_off,
                                  int64_t* __restrict__ bm_off) {
    __shared__ int32_t s_a[1024], s_b[1024], s_c[1024];
    __shared__ int64_t s_d[1024];
    __shared__ int32_t carry_a, carry_b, carry_c;
    __shared__ int64_t carry_d;
    if (threadIdx.x == 0) { carry_a = 0; carry_b = 0; carry_c = 0; carry_d = 0; }
    __syncthreads();
    for (int base = 0; base < ncl; base += 1024) {
        const int j = base + threadIdx.x;
        const int32_t v = (j < ncl) ? cnt[j] : 0;
        const int32_t vb = (v + G - 1) / G;
        const int64_t n_c = (j < ncl) ? cl_off[j + 1] - cl_off[j] : 0;
        const int32_t vc = (j < ncl) ? tc_units(v, n_c) : 0;
        const int64_t vd = (int64_t)v * bitmap_words(n_c);
        s_a[threadIdx.x] = v;
        s_b[threadIdx.x] = vb;
        s_c[threadIdx.x] = vc;
        s_d[threadIdx.x] = vd;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {          // inclusive Hillis-Steele scans
            const int32_t ta = threadIdx.x >= o ? s_a[threadIdx.x - o] : 0;
            const int32_t tb = threadIdx.x >= o ? s_b[threadIdx.x - o] : 0;
            const int32_t tcv = threadIdx.x >= o ? s_c[threadIdx.x - o] : 0;
            const int64_t td = threadIdx.x >= o ? s_d[threadIdx.x - o] : 0;
            __syncthreads();
            s_a[threadIdx.x] += ta;
            s_b[threadIdx.x] += tb;
            s_c[threadIdx.x] += tcv;
            s_d[threadIdx.x] += td;
            __syncthreads();
        }
        if (j < ncl) {
            const int32_t ea = carry_a + s_a[threadIdx.x] - v;
            off[j] = ea;
            cursor[j] = ea;
            item_off[j] = carry_b + s_b[threadIdx.x] - vb;
            unit_off[j] = carry_c + s_c[threadIdx.x] - vc;
            bm_off[j] = carry_d + s_d[threadIdx.x] - vd;
        }
        __syncthreads();
        if (threadIdx.x == 1023) {
            carry_a += s_a[1023]; carry_b += s_b[1023]; carry_c += s_c[1023]; carry_d += s_d[1023];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        off[ncl] = carry_a; item_off[ncl] = carry_b; unit_off[ncl] = carry_c; bm_off[ncl] = carry_d;
    }
}

__global__ void group_fill_kernel(const int32_t* __restrict__ route, int64_t npairs, int32_t* __restrict__ cursor,
                                  int32_t* __restrict__ pairs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < npairs) pairs[atomicAdd(&cursor[route[i]], 1)] = (int32_t)i;
}

// The queries grouped by their best cluster (probe 0), one block per
// cluster: block j reserves a contiguous range for the queries whose first
// probe is cluster j and fills it (order inside the range is free).  The
// re-score runs its blocks in this order, so queries with neighbouring
// candidates gather their rows close together in time and share them
// through L2.  Every query has exactly one probe 0, so the ranges cover
// 0..nq-1.
__global__ void primary_order_kernel(const int32_t* __restrict__ pairs, const int32_t* __restrict__ off, int c,
                                     int32_t* __restrict__ qorder, unsigned long long* __restrict__ counter) {
    __shared__ int s_cnt, s_base, s_pos;
    const int j = blockIdx.x;
    const int lo = off[j], hi = off[j + 1];
    if (threadIdx.x == 0) { s_cnt = 0; s_pos = 0; }
    __syncthreads();
    int mine = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) mine += (pairs[i] % c) == 0;
    if (mine) atomicAdd(&s_cnt, mine);
    __syncthreads();
    if (threadIdx.x == 0) s_base = s_cnt ? (int)atomicAdd(counter, (unsigned long long)s_cnt) : 0;
    __syncthreads();
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int p = pairs[i];
        if (p % c == 0) qorder[s_base + atomicAdd(&s_pos, 1)] = p / c;
    }
}

// The grouping of a small batch in one launch (one block of kGroupThreads):
// the same outputs as group_count_kernel + group_scan_kernel +
// group_fill_kernel + primary_order_kernel, with the per-cluster counters in
// shared memory.  Pairs inside a cluster, and queries inside a first-probe
// cluster, are in no particular order (as there).
constexpr int kGroupThreads = 1024;
constexpr int kGroupMaxCl = 4096;           // clusters (two shared counters each)
constexpr int64_t kGroupMaxPairs = 131072;  // larger batches take the multi-block kernels (faster there)
constexpr int kGroupLoads = 4;              // int4 loads of route in flight per thread

// Exclusive scan of one value per thread over the block (all threads call
// it); *total receives the sum.  s_w holds kGroupThreads / 32 entries.
template <class T>
__device__ T block_excl_scan(T v, T* s_w, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_w[wid] = x;
    __syncthreads();
    if (wid == 0) {
        T y = lane < nw ? s_w[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        if (lane < nw) s_w[lane] = y;               // inclusive over warps
    }
    __syncthreads();
    const T before = (wid > 0 ? s_w[wid - 1] : T(0)) + x - v;
    *total = s_w[nw - 1];
    __syncthreads();                               // s_w is free again
    return before;
}

__global__ void __launch_bounds__(kGroupThreads) group_kernel(
        const int32_t* __restrict__ route, int64_t npairs, int c, int ncl, int G, const int64_t* __restrict__ cl_off,
        int32_t* __restrict__ cnt_out, int32_t* __restrict__ off, int32_t* __restrict__ item_off,
        int32_t* __restrict__ unit_off, int64_t* __restrict__ bm_off, int32_t* __restrict__ pairs,
        int32_t* __restrict__ qorder) {
    __shared__ int32_t s_cnt[kGroupMaxCl], s_cnt0[kGroupMaxCl];   // counts, then cursors
    __shared__ int32_t s_w32[kGroupThreads / 32];
    __shared__ int64_t s_w64[kGroupThreads / 32];
    const int tid = threadIdx.x;
    for (int j = tid; j < ncl; j += kGroupThreads) {
        s_cnt[j] = 0;
        s_cnt0[j] = 0;
    }
    __syncthreads();
    // the pairs four at a time (route is 16-byte aligned), kGroupLoads loads
    // of a thread in flight; then the tail
    const int64_t n4 = npairs / 4;
    const int4* r4 = reinterpret_cast<const int4*>(route);
    auto for_pairs = [&](auto&& f) {
        for (int64_t v0 = tid; v0 < n4; v0 += (int64_t)kGroupThreads * kGroupLoads) {
            int4 x[kGroupLoads];
#pragma unroll
            for (int u = 0; u < kGroupLoads; ++u) {
                const int64_t v = v0 + (int64_t)u * kGroupThreads;
                if (v < n4) x[u] = __ldg(r4 + v);
            }
#pragma unroll
            for (int u = 0; u < kGroupLoads; ++u) {
                const int64_t v = v0 + (int64_t)u * kGroupThreads;
                if (v < n4) {
                    f(4 * v, x[u].x);
                    f(4 * v + 1, x[u].y);
                    f(4 * v + 2, x[u].z);
                    f(4 * v + 3, x[u].w);
                }
            }
        }
        for (int64_t i = 4 * n4 + tid; i < npairs; i += kGroupThreads) f(i, __ldg(route + i));
    };
    for_pairs([&](int64_t i, int j) {
        atomicAdd(&s_cnt[j], 1);
        if (qorder && i % c == 0) atomicAdd(&s_cnt0[j], 1);   // the query's first probe
    });
    __syncthreads();
    // each thread a run of consecutive clusters; scans of the runs' sums
    const int per = (ncl + kGroupThreads - 1) / kGroupThreads;
    const int j0 = min(ncl, tid * per), j1 = min(ncl, j0 + per);
    int32_t sa = 0, sb = 0, sc = 0, s0 = 0;
    int64_t sd = 0;
    for (int j = j0; j < j1; ++j) {
        const int32_t v = s_cnt[j];
        const int64_t n_c = cl_off[j + 1] - cl_off[j];
        sa += v;
        sb += (v + G - 1) / G;
        sc += tc_units(v, n_c);
        sd += (int64_t)v * bitmap_words(n_c);
        s0 += s_cnt0[j];
    }
    int32_t ta, tb, tcn, t0;
    int64_t td;
    int32_t ea = block_excl_scan(sa, s_w32, &ta);
    int32_t eb = block_excl_scan(sb, s_w32, &tb);
    int32_t ec = block_excl_scan(sc, s_w32, &tcn);
    int32_t e0 = block_excl_scan(s0, s_w32, &t0);
    int64_t ed = block_excl_scan(sd, s_w64, &td);
    for (int j = j0; j < j1; ++j) {
        const int32_t v = s_cnt[j];
        const int64_t n_c = cl_off[j + 1] - cl_off[j];
        cnt_out[j] = v;
        off[j] = ea;
        item_off[j] = eb;
        unit_off[j] = ec;
        bm_off[j] = ed;
        const int32_t v0 = s_cnt0[j];
        s_cnt[j] = ea;                             // cursors
        s_cnt0[j] = e0;
        ea += v;
        eb += (v + G - 1) / G;
        ec += tc_units(v, n_c);
        ed += (int64_t)v * bitmap_words(n_c);
        e0 += v0;
    }
    if (tid == 0) {
        off[ncl] = ta;
        item_off[ncl] = tb;
        unit_off[ncl] = tcn;
        bm_off[ncl] = td;
    }
    __syncthreads();
    for_pairs([&](int64_t i, int j) {
        pairs[atomicAdd(&s_cnt[j], 1)] = (int32_t)i;
        if (qorder && i % c == 0) qorder[atomicAdd(&s_cnt0[j], 1)] = (int32_t)(i / c);
    });
}

// ----------------------------------------------------------------- locate --
// One thread per (pair, array l).  pair = q * c + probe.  Also counts the RMI
// diagnostics of Sec. 7.4: predictions at either end of the array (OOR) and
// predictions more than k from the lower bound (LE).
__global__ void locate_kernel(Geometry g, int64_t npairs, int c, int R, int k,
                              const int32_t* __restrict__ route, const uint64_t* __restrict__ qkeys,
                              int32_t* __restrict__ wstart, int32_t* __restrict__ wlen,
                              int32_t* __restrict__ trace_pstar, int32_t* __restrict__ trace_wstart,
                              int32_t* __restrict__ trace_wlen, unsigned long long* __restrict__ counters) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned fb = 0, empty = 0, oor = 0, le = 0, both = 0;
    if (gid < npairs * g.L) {
        const int64_t pair = gid / g.L;
        const int l = (int)(gid % g.L);
        const int64_t q = pair / c;
        const int j = route[pair];
        const int64_t base = g.cl_off[j];
        const int64_t n_c = g.cl_off[j + 1] - base;
        const uint64_t x = qkeys[q * g.L + l];
        Located o{0, 0, 0, 0};
        if (n_c == 0) {
            empty = (l == 0);
        } else {
            o = locate_window(g.keys + (int64_t)l * g.n + base, n_c, g.root[(int64_t)j * g.L + l],
                              g.leaf + ((int64_t)j * g.L + l) * g.F, g.F, x, R, g.m, g.beta, g.B, g.raw_keys != 0,
                              fb);
            oor = (o.ph == 0 || o.ph == n_c - 1);
            le = (o.ph - o.p > k || o.p - o.ph > k);
            both = oor & le;
        }
        wstart[gid] = (int32_t)o.s;
        wlen[gid] = (int32_t)o.T;
        if (trace_pstar) trace_pstar[gid] = (int32_t)o.p;
        if (trace_wstart) trace_wstart[gid] = (int32_t)o.s;
        if (trace_wlen) trace_wlen[gid] = (int32_t)o.T;
    }
    for (int s = 16; s > 0; s >>= 1) {
        fb += __shfl_xor_sync(0xffffffffu, fb, s);
        empty += __shfl_xor_sync(0xffffffffu, empty, s);
        oor += __shfl_xor_sync(0xffffffffu, oor, s);
        le += __shfl_xor_sync(0xffffffffu, le, s);
        both += __shfl_xor_sync(0xffffffffu, both, s);
    }
    if ((threadIdx.x & 31) == 0) {
        if (fb) atomicAdd(&counters[CNT_FALLBACK], (unsigned long long)fb);
        if (empty) atomicAdd(&counters[CNT_EMPTY], (unsigned long long)empty);
        if (oor) atomicAdd(&counters[CNT_OOR], (unsigned long long)oor);
        if (le) atomicAdd(&counters[CNT_LE], (unsigned long long)le);
        if (both) atomicAdd(&counters[CNT_OOR_LE], (unsigned long long)both);
    }
}

// ------------------------------------------------- Layer-1 route (core) --
// The centroids retriever of Sec. 3.2 as a core model: the query key of each
// array is located in the sorted centroid keys of that array and expanded by
// Rc = r0 * c positions (locate_window, as in every cluster); the c best of
// the union of the L windows by the routing score, ties to the lower index,
// become the query's route.  Every window holds min(Rc, n_clusters) >= c
// distinct centroids, so the union never has fewer than c.
//
// Scores come from the routing step's score matrix, which this path computes
// for every query anyway (its per-query error bounds serve the tensor score
// modes):
//   - exact FP64 scores (SIMT mode, S_exact): the c best candidates directly;
//   - tensor-core scores within `guard` of the exact ones (S_approx): the c+1
//     best candidates by approximate score; when every gap among them exceeds
//     twice the guard, their order is the exact one; otherwise every candidate
//     within twice the guard of the c-th approximate score (a set that holds
//     the exact c best) is re-scored exactly (warp_exact_score) and the c best
//     taken from those.
// One warp per query; lane l handles array l.  Per warp, shared memory holds
// the union as a bitmap (words), then as an ascending list of up to cap
// centroids, with an FP32 and a 64-bit score key per entry.
__global__ void route_core_kernel(Geometry g, const uint64_t* __restrict__ ckeys, const int32_t* __restrict__ cpos,
                                  const RmiRoot* __restrict__ croot, const RmiLeaf* __restrict__ cleaf,
                                  const uint64_t* __restrict__ qkeys, const float* __restrict__ Q, int64_t nq,
                                  int c, int Rc, int words, int cap, int warp_bytes,
                                  const float* __restrict__ S_approx, float guard_scale,
                                  const double* __restrict__ S_exact, int32_t* __restrict__ route,
                                  int32_t* __restrict__ trace_route) {
    extern __shared__ __align__(16) unsigned char route_smem[];
    const int lane = threadIdx.x & 31;
    const int64_t q = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (q >= nq) return;                                   // whole warps leave together
    unsigned char* base = route_smem + (size_t)(threadIdx.x >> 5) * warp_bytes;
    uint32_t* bm = reinterpret_cast<uint32_t*>(base);
    base += align_up_dev((size_t)words * 4, 16);
    int32_t* list = reinterpret_cast<int32_t*>(base);
    base += align_up_dev((size_t)cap * 4, 16);
    float* av = reinterpret_cast<float*>(base);
    base += align_up_dev((size_t)cap * 4, 16);
    uint64_t* key = reinterpret_cast<uint64_t*>(base);
    const int ncl = g.ncl;
    for (int w = lane; w < words; w += 32) bm[w] = 0u;
    __syncwarp();
    unsigned fb = 0;
    for (int l = lane; l < g.L; l += 32) {
        const Located o = locate_window(ckeys + (int64_t)l * ncl, ncl, croot[l], cleaf + (int64_t)l * g.F, g.F,
                                        qkeys[q * g.L + l], Rc, g.m, g.beta, g.B, g.raw_keys != 0, fb);
        const int32_t* P = cpos + (int64_t)l * ncl;
        for (int64_t i = o.s; i < o.s + o.T; ++i) {
            const int j = P[i];
            atomicOr(&bm[j >> 5], 1u << (j & 31));
        }
    }
    __syncwarp();
    // the union as an ascending list
    int n = 0;
    for (int w0 = 0; w0 < words; w0 += 32) {
        const int w = w0 + lane;
        const uint32_t bits = w < words ? bm[w] : 0u;
        const int cnt = __popc(bits);
        int incl = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int pos = n + incl - cnt;
        for (uint32_t b = bits; b && pos < cap; b &= b - 1) list[pos++] = w * 32 + (__ffs(b) - 1);
        n += __shfl_sync(0xffffffffu, incl, 31);
    }
    n = min(n, cap);
    __syncwarp();
    // rounds of a warp arg-max over the entries after the previous pick
    // (key descending, centroid index ascending); rounds beyond the list give -1
    auto pick = [&](uint64_t& ps, int& pj, auto skip) {
        uint64_t best = 0ull;
        int bj = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const uint64_t v = key[i];
            const int j = list[i];
            if (skip(v)) continue;
            const bool after = (v < ps) || (v == ps && j > pj);
            if (after && (v > best || (v == best && j < bj))) { best = v; bj = j; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const uint64_t ov = __shfl_xor_sync(0xffffffffu, best, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
        }
        ps = best;
        pj = bj;
    };
    auto none = [](uint64_t) { return false; };
    auto absent = [](uint64_t v) { return v == 0ull; };
    int out[LIDER_MAX_C];
    if (S_exact) {
        for (int i = lane; i < n; i += 32) key[i] = score_key(S_exact[q * ncl + list[i]]);
        __syncwarp();
        uint64_t ps = ~0ull;
        int pj = -1;
        for (int r = 0; r < c; ++r) { pick(ps, pj, none); out[r] = pj; }
    } else {
        const float* srow = S_approx + q * ncl;
        for (int i = lane; i < n; i += 32) {
            float v = srow[list[i]];
            if (v != v) v = -INFINITY;
            av[i] = v;
            key[i] = (uint64_t)float_order(v);
        }
        __syncwarp();
        const float* qv = Q + q * g.d;
        float qn2 = 0.f;
        for (int t = lane; t < g.d; t += 32) qn2 = fmaf(qv[t], qv[t], qn2);
        for (int o = 16; o > 0; o >>= 1) qn2 += __shfl_xor_sync(0xffffffffu, qn2, o);
        const float guard = guard_scale * sqrtf(qn2);
        // the c + 1 best approximate scores (the (c+1)-th is -inf when n == c)
        uint64_t ps = ~0ull;
        int pj = -1;
        float a[LIDER_MAX_C + 1];
        for (int r = 0; r < c + 1; ++r) {
            if (r == n) { a[r] = -INFINITY; break; }
            pick(ps, pj, none);
            if (r < c) out[r] = pj;
            a[r] = float_from_order((uint32_t)ps);
        }
        bool clear = true;
        for (int r = 0; r < c; ++r)
            if (!(__fsub_rd(a[r], a[r + 1]) > 2.f * guard)) clear = false;
        if (!clear) {
            // exact scores of the band; entries outside it are left out (key 0)
            const float t = __fsub_rd(a[c - 1], 2.f * guard);
            for (int i = 0; i < n; ++i) {
                const bool in = av[i] >= t;
                double v = 0.0;
                if (in) v = warp_exact_score(qv, g.C + (int64_t)list[i] * g.d, g.d, g.half_norm[list[i]]);
                if (lane == 0) key[i] = in ? score_key(v) : 0ull;
            }
            __syncwarp();
            ps = ~0ull;
            pj = -1;
            for (int r = 0; r < c; ++r) { pick(ps, pj, absent); out[r] = pj; }
        }
    }
    if (lane == 0) {
        for (int r = 0; r < c; ++r) {
            const int j = out[r] < ncl ? out[r] : 0;       // unreachable: the union holds >= c centroids
            route[q * c + r] = j;
            if (trace_route) trace_route[q * c + r] = j;
        }
    }
}

// Launch shape of route_core_kernel: per-warp shared memory for the bitmap,
// the list, its FP32 scores and 64-bit keys, 16 bytes per listed centroid
// (n_clusters <= 8192 keeps one warp under 133 KB), up to 8 warps per block.
struct RouteCoreShape {
    int Rc, words, cap, warp_bytes, wpb;
};

RouteCoreShape route_core_shape(const Geometry& g, int r0, int c) {
    RouteCoreShape s;
    s.Rc = r0 * c;
    const int T = std::min(s.Rc, g.ncl);
    s.words = (int)cdiv(g.ncl, 32);
    s.cap = (int)std::min<int64_t>(g.ncl, (int64_t)T * g.L);
    s.warp_bytes = (int)align_up(align_up((size_t)s.words * 4, 16) + 2 * align_up((size_t)s.cap * 4, 16) +
                                     (size_t)s.cap * 8, 16);
    s.wpb = std::max(1, std::min(8, (216 * 1024) / s.warp_bytes));
    return s;
}

// ------------------------------------------------------------------ score --
// Work item = up to G (query, probe) pairs of one cluster j.  Each pair's
// candidate set is the union of its L expansion windows (Sec. 3.3.1: each
// array is searched, then the results are merged); here it is a bit per
// (cluster-local position, pair) in a shared-memory mask, so duplicates
// across arrays collapse for free.  The cluster's rows are then streamed
// once per item: every marked row is loaded by one warp and dotted with each
// query whose bit is set, so a row shared by several queries of the item is
// read once.  Each pair's (score, position) keys go to its list in global
// scratch; after the item, the block selects each pair's top k (Sec. 6.1:
// the k best of the verified candidates) by bucket selection and a small
// bitonic sort in shared memory.
//
// Score of (q, row): lane l accumulates x[i]*q[i] for float4 chunks
// i = l, l+32, ... in ascending order with FMA, then a butterfly sum over the
// warp.  The order depends only on d, so a query's scores do not depend on
// its batch-mates.
struct ScoreArgs {
    Geometry g;
    const float* Q;
    int c, G, k, T_cap;         // T_cap = L * R, capacity of one pair's score list
    int region_bytes;           // dynamic shared memory before the mask
    const int32_t* off;
    const int32_t* cnt;
    const int32_t* item_off;
    const int32_t* pairs;
    const int32_t* wstart;
    uint64_t* pbuf;             // npairs x T_cap keys: (~order(score) << 32) | position
    float* pscore;              // npairs x k, best first
    int64_t* pid;               // npairs x k corpus ids
    int32_t* trace_ucount;
    unsigned long long* counters;
};

constexpr int kMaxGroup = 16;    // bits of a position's mask
constexpr int kTile = 8192;      // positions per mask tile
constexpr int kChunkNV = 8;      // general path: float4 per lane per row chunk
constexpr int kBins = 256;       // buckets of the top-k selection
constexpr int kCandCap = 1024;   // keys sorted after bucket selection

__device__ __forceinline__ uint32_t mask_bits(const uint32_t* mask, int pl) {
    return (mask[pl >> 1] >> (16 * (pl & 1))) & 0xffffu;
}

__device__ __forceinline__ uint64_t score_key(float sc, uint32_t pos) {
    return ((uint64_t)(~float_order(sc)) << 32) | (uint64_t)pos;
}

// Block-wide ascending bitonic sort of n (a power of two) keys in shared memory.
__device__ void block_bitonic(uint64_t* key, int n) {
    for (int size = 2; size <= n; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
                const int lo_i = 2 * stride * (i / stride) + (i % stride);
                const int hi_i = lo_i + stride;
                const bool up = (lo_i & size) == 0;
                const uint64_t x0 = key[lo_i], x1 = key[hi_i];
                if ((x0 > x1) == up) { key[lo_i] = x1; key[hi_i] = x0; }
            }
            __syncthreads();
        }
    }
}

// The k smallest of U distinct keys at src (global), written best first to
// (ps, pi) with padding.  K: shared buffer of next_pow2(T_cap) keys; cand:
// kCandCap keys.  Bucket selection on the 32-bit score order finds the bucket
// holding the k-th key; only the keys up to that bucket are sorted.
__device__ void block_topk(const uint64_t* __restrict__ src, int U, int k, uint64_t* K, uint64_t* cand,
                           uint32_t* bins, uint32_t* scal, int64_t base, const int64_t* __restrict__ orig_id,
                           float* __restrict__ ps, int64_t* __restrict__ pi) {
    const int tid = threadIdx.x;
    const int kk = min(k, U);
    uint64_t* out = cand;
    if (U <= kCandCap) {
        const int SP = U > 1 ? next_pow2_dev(U) : 1;
        for (int u = tid; u < SP; u += blockDim.x) cand[u] = (u < U) ? src[u] : ~0ull;
        __syncthreads();
        block_bitonic(cand, SP);
    } else {
        if (tid == 0) { scal[0] = 0xffffffffu; scal[1] = 0u; scal[2] = 0u; }
        for (int b = tid; b < kBins; b += blockDim.x) bins[b] = 0u;
        __syncthreads();
        uint32_t lo = 0xffffffffu, hi = 0u;
        for (int u = tid; u < U; u += blockDim.x) {
            const uint64_t v = src[u];
            K[u] = v;
            const uint32_t h = (uint32_t)(v >> 32);
            lo = min(lo, h);
            hi = max(hi, h);
        }
        atomicMin(&scal[0], lo);
        atomicMax(&scal[1], hi);
        __syncthreads();
        // buckets linear in the score between the best and the worst key; the
        // map is monotone (round-to-nearest subtraction and scaling preserve
        // order), so every key of a better bucket beats every key of a worse one
        const float s_best = float_from_order(~scal[0]);
        const float s_worst = float_from_order(~scal[1]);
        const float span = s_best - s_worst;
        const float scale = span > 0.f ? (float)kBins / span : 0.f;
        auto bucket = [&](uint64_t v) -> uint32_t {
            const float sc = float_from_order(~(uint32_t)(v >> 32));
            return (uint32_t)fminf(__fmul_rn(__fadd_rn(s_best, -sc), scale), (float)(kBins - 1));
        };
        for (int u = tid; u < U; u += blockDim.x) atomicAdd(&bins[bucket(K[u])], 1u);
        __syncthreads();
        if (tid == 0) {
            uint32_t cum = 0;
            int bsel = kBins - 1;
            for (int b = 0; b < kBins; ++b) {
                cum += bins[b];
                if (cum >= (uint32_t)kk) { bsel = b; break; }
            }
            scal[2] = (uint32_t)bsel;
            scal[3] = cum;
            scal[4] = 0u;
        }
        __syncthreads();
        const uint32_t bsel = scal[2], sel = scal[3];
        if (sel <= (uint32_t)kCandCap) {
            for (int u = tid; u < U; u += blockDim.x) {
                const uint64_t v = K[u];
                if (bucket(v) <= bsel) cand[atomicAdd(&scal[4], 1u)] = v;
            }
            __syncthreads();
            const int SP = sel > 1 ? next_pow2_dev((int)sel) : 1;
            for (int u = (int)sel + tid; u < SP; u += blockDim.x) cand[u] = ~0ull;
            __syncthreads();
            block_bitonic(cand, SP);
        } else {                                    // many equal scores: sort everything
            const int SP = next_pow2_dev(U);
            for (int u = U + tid; u < SP; u += blockDim.x) K[u] = ~0ull;
            __syncthreads();
            block_bitonic(K, SP);
            out = K;
        }
    }
    for (int r = tid; r < k; r += blockDim.x) {
        if (r < kk) {
            const uint64_t kv = out[r];
            ps[r] = float_from_order(~(uint32_t)(kv >> 32));
            pi[r] = orig_id[base + (int64_t)(uint32_t)kv];
        } else {
            ps[r] = -INFINITY;
            pi[r] = -1;
        }
    }
    __syncthreads();
}

// Score the marked rows of one tile.  NV > 0: d == 128 * NV, a row is NV
// float4 per lane held in registers and the set bits are visited two at a
// time with one shared butterfly; NV == 0: any d, chunks of kChunkNV float4
// with bounds checks.
template <int NV>
__device__ __forceinline__ void score_tile(const ScoreArgs& a, const float4* Qs4, const uint32_t* mask, int tl,
                                           int64_t base, int64_t t0, int* s_cnt, const int64_t* s_pair) {
    const Geometry& g = a.g;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nwarps = kScoreThreads / 32;
    const int d4 = g.d / 4;
    for (int pl = warp; pl < tl; pl += nwarps) {
        uint32_t m = mask_bits(mask, pl);
        if (m == 0u) continue;
        const uint32_t pos = (uint32_t)(t0 + pl);
        const float4* X4 = reinterpret_cast<const float4*>(g.X + (base + pos) * (int64_t)g.d);
        if constexpr (NV > 0) {
            float4 x[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) x[v] = __ldg(X4 + lane + 32 * v);
            while (m) {
                // up to four set bits at a time: four independent FMA chains
                int q[4];
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    if (m) {
                        q[s2] = __ffs(m) - 1;
                        m &= m - 1;
                    } else {
                        q[s2] = -1;
                    }
                }
                float acc[4];
#pragma unroll
                for (int s2 = 0; s2 < 4; ++s2) {
                    acc[s2] = 0.f;
                    const float4* y4 = Qs4 + (q[s2] >= 0 ? q[s2] : q[0]) * d4 + lane;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const float4 y = y4[32 * v];
                        acc[s2] = fmaf(x[v].x, y.x, acc[s2]);
                        acc[s2] = fmaf(x[v].y, y.y, acc[s2]);
                        acc[s2] = fmaf(x[v].z, y.z, acc[s2]);
                        acc[s2] = fmaf(x[v].w, y.w, acc[s2]);
                    }
                }
                // one butterfly for four dots: after the xor-16 and xor-8 halving
                // steps lanes 0-7 hold dot 0, 8-15 dot 1, 16-23 dot 2, 24-31 dot 3;
                // every dot gets the same pairing tree as a plain warp sum
                const bool b16 = (lane & 16) != 0, b8 = (lane & 8) != 0;
                float k0 = b16 ? acc[2] : acc[0], k1 = b16 ? acc[3] : acc[1];
                const float s0 = b16 ? acc[0] : acc[2], s1 = b16 ? acc[1] : acc[3];
                k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
                k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
                float keep = b8 ? k1 : k0;
                const float send = b8 ? k0 : k1;
                keep += __shfl_xor_sync(0xffffffffu, send, 8);
                for (int o = 4; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
                if ((lane & 7) == 0) {
                    const int grp = lane >> 3;
                    const int qs = grp == 0 ? q[0] : grp == 1 ? q[1] : grp == 2 ? q[2] : q[3];
                    if (qs >= 0) {
                        const int slot = atomicAdd(&s_cnt[qs], 1);
                        a.pbuf[s_pair[qs] * a.T_cap + slot] = score_key(keep, pos);
                    }
                }
            }
        } else {
            float part[kMaxGroup];
#pragma unroll
            for (int q = 0; q < kMaxGroup; ++q) part[q] = 0.f;
            for (int c0 = 0; c0 < d4; c0 += 32 * kChunkNV) {
                float4 x[kChunkNV];
#pragma unroll
                for (int v = 0; v < kChunkNV; ++v) {
                    const int i4 = c0 + lane + 32 * v;
                    x[v] = (i4 < d4) ? __ldg(X4 + i4) : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int q = 0; q < kMaxGroup; ++q) {
                    if (!((m >> q) & 1u)) continue;
                    float acc = part[q];
#pragma unroll
                    for (int v = 0; v < kChunkNV; ++v) {
                        const int i4 = c0 + lane + 32 * v;
                        if (i4 < d4) {
                            const float4 y = Qs4[q * d4 + i4];
                            acc = fmaf(x[v].x, y.x, acc);
                            acc = fmaf(x[v].y, y.y, acc);
                            acc = fmaf(x[v].z, y.z, acc);
                            acc = fmaf(x[v].w, y.w, acc);
                        }
                    }
                    part[q] = acc;
                }
            }
#pragma unroll
            for (int q = 0; q < kMaxGroup; ++q) {
                if (!((m >> q) & 1u)) continue;
                float sc = part[q];
                for (int o = 16; o > 0; o >>= 1) sc += __shfl_xor_sync(0xffffffffu, sc, o);
                if (lane == 0) {
                    const int slot = atomicAdd(&s_cnt[q], 1);
                    a.pbuf[s_pair[q] * a.T_cap + slot] = score_key(sc, pos);
                }
            }
        }
    }
}

// Dynamic shared memory: region of region_bytes (queries G x d floats while
// scoring, then the top-k buffers) | mask kTile/2 u32 (16 bits per position).
template <int NV>
__global__ void __launch_bounds__(kScoreThreads) score_group_kernel(ScoreArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const Geometry& g = a.g;
    float* Qs = reinterpret_cast<float*>(smem);
    uint32_t* mask = reinterpret_cast<uint32_t*>(smem + a.region_bytes);
    uint64_t* K = reinterpret_cast<uint64_t*>(smem);
    uint64_t* cand = K + next_pow2_dev(a.T_cap);
    __shared__ int s_item;
    __shared__ int s_cnt[kMaxGroup];
    __shared__ int64_t s_pair[kMaxGroup];
    __shared__ uint32_t s_bins[kBins];
    __shared__ uint32_t s_scal[8];
    const int tid = threadIdx.x;
    const int total_items = a.item_off[g.ncl];
    const int d4 = g.d / 4;
    const float4* Qs4 = reinterpret_cast<const float4*>(Qs);

    for (;;) {
        if (tid == 0) s_item = (int)atomicAdd(&a.counters[CNT_ITEM], 1ull);
        __syncthreads();
        const int item = s_item;
        if (item >= total_items) break;
        int lo = 0, hi = g.ncl - 1;                       // last j with item_off[j] <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.item_off[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int j = lo;
        const int first = a.off[j] + (item - a.item_off[j]) * a.G;
        const int count = min(a.G, a.off[j] + a.cnt[j] - first);
        const int64_t base = g.cl_off[j];
        const int64_t n_c = g.cl_off[j + 1] - base;

        if (tid < count) {
            s_pair[tid] = a.pairs[first + tid];
            s_cnt[tid] = 0;
        }
        __syncthreads();
        for (int i = tid; i < count * d4; i += kScoreThreads) {
            const int gq = i / d4, c4 = i - gq * d4;
            const int64_t q = s_pair[gq] / a.c;
            reinterpret_cast<float4*>(Qs)[i] = reinterpret_cast<const float4*>(a.Q + q * g.d)[c4];
        }
        const int T = (int)min((int64_t)a.T_cap / g.L, n_c);   // window length min(R, n_c)

        for (int64_t t0 = 0; t0 < n_c; t0 += kTile) {
            const int tl = (int)min((int64_t)kTile, n_c - t0);
            for (int i = tid; i < (tl + 1) / 2; i += kScoreThreads) mask[i] = 0u;
            __syncthreads();
            // mark the union of the windows of every pair of the item
            {   // one warp per window, lanes along the window
                const int warp = tid >> 5, lane = tid & 31;
                for (int wi = warp; wi < count * g.L; wi += kScoreThreads / 32) {
                    const int gq = wi / g.L, l = wi - gq * g.L;
                    const int32_t ws = a.wstart[s_pair[gq] * g.L + l];
                    const int32_t* P = g.pos + (int64_t)l * g.n + base + ws;
                    const uint32_t bit = 1u << gq;
                    for (int t = lane; t < T; t += 32) {
                        const int64_t pl = (int64_t)P[t] - t0;
                        if (pl >= 0 && pl < tl) atomicOr(&mask[pl >> 1], bit << (16 * (int)(pl & 1)));
                    }
                }
            }
            __syncthreads();
            score_tile<NV>(a, Qs4, mask, tl, base, t0, s_cnt, s_pair);
            __syncthreads();
        }
        // per-pair top-k (the query rows in shared memory are no longer needed)
        for (int gq = 0; gq < count; ++gq) {
            const int64_t pair = s_pair[gq];
            const int U = s_cnt[gq];
            block_topk(a.pbuf + pair * a.T_cap, U, a.k, K, cand, s_bins, s_scal, base, g.orig_id,
                       a.pscore + pair * a.k, a.pid + pair * a.k);
        }
        if (tid < count) {
            atomicAdd(&a.counters[CNT_CANDIDATES], (unsigned long long)s_cnt[tid]);
            if (a.trace_ucount) a.trace_ucount[s_pair[tid]] = s_cnt[tid];
        }
        __syncthreads();
    }
}

// ----------------------------------------------------- tensor-core score --
// Scoring on the tcgen05 tensor cores (LIDER_SCORE_TENSOR).  The pairs of one
// cluster are cut into query tiles of 128 (their queries gathered, in pair
// order, into Qp, split into TF32 head and tail) and the cluster's rows into
// row tiles of 256; each (query tile, row tile) unit is one dense 128 x 256
// tile computed with three TF32 products per FP32 product (tc.cuh).  The
// epilogue keeps only candidates: mark_kernel first writes, per pair, a
// bitmap over its cluster's positions of the union of its L expansion windows
// (Sec. 3.3.1), and a tile reads 8 words of it per query.  Each candidate's
// key goes to the pair's list; select_query_kernel then picks each query's best.
__global__ void qgather_kernel(const float* __restrict__ Q, const int32_t* __restrict__ pairs, int64_t np, int c,
                               int d, float* __restrict__ qp_hi, float* __restrict__ qp_lo) {
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= np) return;
    const int64_t q = pairs[slot] / c;
    const float4* src = reinterpret_cast<const float4*>(Q + q * d);
    float4* hi = reinterpret_cast<float4*>(qp_hi + slot * d);
    float4* lo = reinterpret_cast<float4*>(qp_lo + slot * d);
    for (int i = lane; i < d / 4; i += 32) {
        const float4 v = src[i];
        float4 h, l;
        h.x = __uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u); l.x = __fsub_rn(v.x, h.x);
        h.y = __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u); l.y = __fsub_rn(v.y, h.y);
        h.z = __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u); l.z = __fsub_rn(v.z, h.z);
        h.w = __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u); l.w = __fsub_rn(v.w, h.w);
        hi[i] = h;
        lo[i] = l;
    }
}

// FP16 path: the queries in pair order, scaled by their power of two and
// rounded to FP16.
__global__ void qgather_f16_kernel(const float* __restrict__ Q, const int32_t* __restrict__ pairs, int64_t np, int c,
                                   int d, const float* __restrict__ qscale, uint16_t* __restrict__ qp) {
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= np) return;
    const int64_t q = pairs[slot] / c;
    const float s = qscale[q];
    const float* src = Q + q * d;
    uint16_t* dst = qp + slot * d;
    for (int i = lane; i < d; i += 32) dst[i] = __half_as_ushort(__float2half_rn(src[i] * s));
}

// Served FP8 form: the queries in pair order as e4m3 with one scale per query
// (max|q| / 448), recorded per slot for the epilogue.
__global__ void qgather_f8_kernel(const float* __restrict__ Q, const int32_t* __restrict__ pairs, int64_t np, int c,
                                  int d, float* __restrict__ slot_scale, uint8_t* __restrict__ qp) {
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= np) return;
    const int64_t q = pairs[slot] / c;
    const float* src = Q + q * d;
    float amax = 0.f;
    for (int i = lane; i < d; i += 32) amax = fmaxf(amax, fabsf(src[i]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float inv = amax > 0.f ? 448.f / amax : 1.f;
    if (lane == 0) slot_scale[slot] = amax > 0.f ? amax / 448.f : 1.f;
    uint8_t* dst = qp + slot * d;
    for (int i = lane; i < d; i += 32) dst[i] = (uint8_t)__nv_cvt_float_to_fp8(src[i] * inv, __NV_SATFINITE, __NV_E4M3);
}

// Served form: the queries in pair order, rounded to BF16.
__global__ void qgather_bf16_kernel(const float* __restrict__ Q, const int32_t* __restrict__ pairs, int64_t np, int c,
                                    int d, uint16_t* __restrict__ qp) {
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (slot >= np) return;
    const int64_t q = pairs[slot] / c;
    const float* src = Q + q * d;
    uint16_t* dst = qp + slot * d;
    for (int i = lane; i < d; i += 32) dst[i] = __bfloat16_as_ushort(__float2bfloat16_rn(src[i]));
}


// One warp per pair slot (pairs in cluster order; blockDim / 32 slots per
// block): the union of the pair's L expansion windows as a bitmap over the
// cluster's positions, at bitmap + bm_off[j] + (slot - off[j]) * words_j; also
// slot_of[pair] = slot and ucount[pair] = the number of candidates (set bits).
// A bitmap of up to smem_words words is built in the warp's shared memory,
// a larger one in place with global atomics.
__global__ void __launch_bounds__(256) mark_kernel(const int32_t* __restrict__ pairs,
                                                   const int32_t* __restrict__ route, const int32_t* __restrict__ off,
                                                   const int64_t* __restrict__ cl_off,
                                                   const int64_t* __restrict__ bm_off,
                                                   const int32_t* __restrict__ wstart, const int32_t* __restrict__ pos,
                                                   int64_t n, int L, int R, uint32_t* __restrict__ bitmap,
                                                   int32_t* __restrict__ slot_of, int32_t* __restrict__ ucount,
                                                   int smem_words, int64_t np) {
    extern __shared__ uint32_t sbits[];         // (blockDim / 32) x smem_words
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    if (slot >= np) return;                     // the whole warp
    const int64_t pair = pairs[slot];
    const int j = route[pair];
    const int64_t base = cl_off[j];
    const int64_t n_c = cl_off[j + 1] - base;
    if (lane == 0) slot_of[pair] = (int32_t)slot;
    if (n_c == 0) return;                       // ucount stays 0 (cleared)
    const int64_t words = bitmap_words(n_c);
    uint32_t* dst = bitmap + bm_off[j] + (slot - off[j]) * words;
    const int T = (int)min((int64_t)R, n_c);
    const bool in_smem = words <= smem_words;
    uint32_t* bits = in_smem ? sbits + (size_t)warp * smem_words : dst;
    for (int64_t i = lane; i < words; i += 32) bits[i] = 0u;
    __syncwarp();
    // window starts of the L arrays loaded at once (L <= 32), then each
    // window's positions in rounds of up to kMarkBatch loads per lane, all
    // issued before their shared-memory atomics
    constexpr int kMarkBatch = 12;
    const int ws_lane = lane < L ? wstart[pair * L + lane] : 0;
    for (int l = 0; l < L; ++l) {
        const int32_t* P = pos + (int64_t)l * n + base + __shfl_sync(0xffffffffu, ws_lane, l);
        for (int t0 = lane; t0 < T; t0 += 32 * kMarkBatch) {
            uint32_t pv[kMarkBatch];
#pragma unroll
            for (int r = 0; r < kMarkBatch; ++r) pv[r] = t0 + 32 * r < T ? (uint32_t)__ldg(P + t0 + 32 * r) : ~0u;
#pragma unroll
            for (int r = 0; r < kMarkBatch; ++r)
                if (pv[r] != ~0u) atomicOr(&bits[pv[r] >> 5], 1u << (pv[r] & 31));
        }
    }
    __syncwarp();
    int u = 0;
    for (int64_t i = lane; i < words; i += 32) {
        const uint32_t wv = bits[i];
        if (in_smem) dst[i] = wv;
        u += __popc(wv);
    }
    for (int o = 16; o > 0; o >>= 1) u += __shfl_xor_sync(0xffffffffu, u, o);
    if (lane == 0) ucount[pair] = u;            // candidates of the pair
}

// One tensor-core tile: A row (first query slot), B row (first corpus row),
// cluster, and (query tile << 16 | row tile); and what its epilogue needs
// (umeta: query slots in the tile, cluster size, and the bitmap word of the
// tile's first slot at its first column, low and high halves).  Written once
// per search so the producer, MMA and epilogue warps each read a tile's
// coordinates with one or two independent loads.  Each block also writes the
// code bound of its cluster's pair slots (slot_bound: the slot's query's B).
__global__ void tc_units_kernel(const int32_t* __restrict__ unit_off, const int32_t* __restrict__ off,
                                const int64_t* __restrict__ cl_off, const int64_t* __restrict__ bm_off,
                                const int32_t* __restrict__ pairs, const float* __restrict__ qbound, int c, int ncl,
                                int order, int4* __restrict__ units, int4* __restrict__ umeta,
                                float* __restrict__ slot_bound) {
    const int j = blockIdx.x;
    const int64_t n_c = cl_off[j + 1] - cl_off[j];
    for (int sl = off[j] + threadIdx.x; sl < off[j + 1]; sl += blockDim.x) slot_bound[sl] = qbound[pairs[sl] / c];
    const int u0 = unit_off[j], u1 = unit_off[j + 1];
    if (u1 <= u0) return;
    const int nrt = (int)((n_c + tc::kBN - 1) / tc::kBN);
    const int cnt = off[j + 1] - off[j];
    const int64_t words = bitmap_words(n_c);
    for (int u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
        const int local = u - u0;
        // order 0: query tiles outer; 1: row tiles outer
        const int nit = (u1 - u0) / nrt;
        const int it = order ? local % nit : local / nrt;
        const int rt = order ? local / nit : local % nrt;
        units[u] = make_int4(off[j] + it * tc::kBM, (int)(cl_off[j] + (int64_t)rt * tc::kBN), j, (it << 16) | rt);
        const int64_t w0 = bm_off[j] + (int64_t)it * tc::kBM * words + rt * (tc::kBN / 32);
        umeta[u] = make_int4(min(tc::kBM, cnt - it * tc::kBM), (int)n_c, (int)(uint32_t)(w0 & 0xffffffffll),
                             (int)(w0 >> 32));
    }
}

struct TcArgs {
    const int4* units;
    const int4* umeta;          // per tile: slots in it, cluster size, first bitmap word (lo, hi)
    const float* slot_bound;    // per pair slot: the code bound B of its query
    const int32_t* unit_off;
    const int32_t* off;
    const int32_t* cnt;
    const int64_t* cl_off;
    const int32_t* pairs;
    const int64_t* bm_off;
    int ncl;
    uint16_t* dense;            // per pair: approximate score codes over its cluster's positions
    const float* qbound;        // per query: the codes' range bound B
    int c;                      // probes per query (pair = query * c + probe)
    const uint32_t* bitmap;     // per pair: candidate bitmap (mark_kernel)
    float* cmax;                // per pair and bitmap word: best candidate score of those 32 positions
    const float* slot_scale;    // FP8 form: per slot query scale (else null)
    const float* col_scale;     // FP8 form: per corpus row scale, reordered rows
};

struct TcSched {
    const TcArgs* a;
    __device__ int count() const { return a->unit_off[a->ncl]; }
    __device__ void coords(int u, int& arow, int& brow) const {
        const int4 t = a->units[u];
        arow = t.x;
        brow = t.y;
    }
};

// The epilogue writes every score of the tile, dense, as a 16-bit code
// (score_code over the query's [-B, B]): row r of a pair slot s in cluster j
// is dense + (bm_off[j] + (s - off[j]) * words_j) * 32, one code per cluster
// position (pitch 32 * words_j, a multiple of 32, so the rows and every
// 32-column group are 64-byte aligned).  A warp converts its 32 rows x 32
// columns (one row per lane), transposes them through shared memory and
// stores them 8 rows x 64 bytes per instruction.  It also writes, per pair
// and 32 positions, the best candidate's score as its code maps back
// (code_score of the smallest candidate code).  Which positions are
// candidates is read from the pair's bitmap, here and in the select.
//
// Epilogue warps of tc_score_kernel: 12 (three per TMEM lane quarter, taking
// 3, 3 and 2 of its 8 column groups; with the producer and MMA warps at most
// four warps per scheduler, which leaves each thread 128 registers), with all
// of the kind's stages of K.  A warp's transpose stage is 32 rows x 16 words (two codes per
// word): word j of row r sits at r * 16 + (j ^ (r >> 1)), so the 32 lanes'
// row writes hit 32 banks, and a row's four aligned 16-byte groups stay
// aligned (their words permuted inside) for the 16-byte reads.
constexpr int kEpiWords = 16;
template <class Kind> struct ScorePlan {
    static constexpr int kEpiWarps = 12;
    static constexpr int kStages = Kind::kStages;
    static constexpr int kThreads = tc::threads_for(kEpiWarps);
    static constexpr int kStageBytes = kStages * Kind::kOps * (tc::kTileA + tc::kTileB) + 1024;
    static constexpr int kSmem = kStageBytes + kEpiWarps * 32 * kEpiWords * 4;
    static_assert(kSmem + 1024 <= 227 * 1024, "score kernel shared memory (with room for the static part)");
};

// 16-bit code of s in one instruction after the FMA: rint((B - s) * inv),
// saturated to [0, 65535] by the conversion.
__device__ __forceinline__ uint32_t score_code_sat(float s, float inv, float binv) {
    const float x = __fmaf_rn(-s, inv, binv);
    unsigned short h;
    asm("cvt.rni.sat.u16.f32 %0, %1;" : "=h"(h) : "f"(x));
    return h;
}

template <int kEpiWarps>
struct TcEpi {
    const TcArgs* a;
    uint32_t* stage;            // this warp's 32 x kEpiWords words (packed code pairs, swizzled)
    uint16_t* drow;             // this lane's dense row at the tile's first column (null: no pair)
    float B, inv, binv, step;   // this row's code range: bound, 65535 / 2B, B * inv, 2B / 65535
    int ncols;                  // columns of the tile inside the row pitch (a multiple of 32)
    float rs;                   // FP8 form: this row's query scale
    const float* cs;            // FP8 form: row scales of the tile's corpus rows (null: unscaled)
    int ncs;                    // rows of the tile inside the cluster
    float* crow;                // this lane's chunk maxima at the tile's first word (null: no pair)
    uint32_t bits[tc::kBN / 32];  // this lane's candidate bits over the tile's 256 columns

    __device__ void begin(int u, int row) {
        const int4 t = __ldg(a->units + u);
        const int4 um = __ldg(a->umeta + u);
        const int rt = t.w & 0xffff;
        const int in_tile = um.x;
        const int64_t n_c = um.y;
        const int64_t words = bitmap_words(n_c);
        const int p0 = rt * tc::kBN;
        ncols = (int)min((int64_t)tc::kBN, words * 32 - p0);
        const bool live = row < in_tile;
        // this lane's pair: bitmap word at the tile's first column
        const int64_t wt = ((int64_t)(uint32_t)um.w << 32 | (uint32_t)um.z) + (int64_t)row * words;
        drow = live ? a->dense + wt * 32 : nullptr;
        B = live ? __ldg(a->slot_bound + t.x + row) : 1.f;
        if (!(B > 0.f)) B = 1.f;                              // no scores to code (|q| = 0)
        inv = __fdiv_rn(65535.f, __fmul_rn(2.f, B));
        binv = __fmul_rn(B, inv);
        step = code_step(B);
        crow = live ? a->cmax + wt : nullptr;
        // this warp's column groups of the tile (kEpiWarps / 4 warps share each row;
        // the same split as the engine's)
        constexpr int kGpw = ((tc::kBN / 32) + kEpiWarps / 4 - 1) / (kEpiWarps / 4);
        const int g0 = ((((int)threadIdx.x >> 5) - 2) >> 2) * kGpw;
#pragma unroll
        for (int w = 0; w < tc::kBN / 32; ++w)
            bits[w] = (live && 32 * w < ncols && w >= g0 && w < g0 + kGpw) ? __ldg(a->bitmap + wt + w) : 0u;
        cs = nullptr;
        if (a->slot_scale) {
            rs = live ? a->slot_scale[t.x + row] : 0.f;
            cs = a->col_scale + t.y;
            ncs = (int)min((int64_t)tc::kBN, n_c - p0);
        }
    }

    // Called by all 32 lanes of the warp (lane = accumulator row).
    __device__ void operator()(int, int, int col0, const uint32_t (&v)[32]) {
        if (col0 >= ncols) return;                           // the same in every lane (per tile)
        uint32_t w = 0;
#pragma unroll
        for (int i = 0; i < tc::kBN / 32; ++i)               // a select, not a local-memory index
            if (i == (col0 >> 5)) w = bits[i];
        // this lane's row as codes (FP8 form: score = acc * query scale * row
        // scale; rows past the cluster: 0) into the stage, and its best
        // candidate's score
        const int lane = threadIdx.x & 31;
        float m = -INFINITY;
        const int swz = lane >> 1;
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
            float x0 = __uint_as_float(v[i]), x1 = __uint_as_float(v[i + 1]);
            if (cs) {
                x0 = x0 * rs * (col0 + i < ncs ? __ldg(cs + col0 + i) : 0.f);
                x1 = x1 * rs * (col0 + i + 1 < ncs ? __ldg(cs + col0 + i + 1) : 0.f);
            }
            stage[lane * kEpiWords + ((i >> 1) ^ swz)] =
                __byte_perm(score_code_sat(x0, inv, binv), score_code_sat(x1, inv, binv), 0x5410);
            m = fmaxf(m, ((w >> i) & 1u) ? x0 : -INFINITY);
            m = fmaxf(m, ((w >> (i + 1)) & 1u) ? x1 : -INFINITY);
        }
        if (crow) crow[col0 >> 5] = m > -INFINITY ? code_score(score_code_sat(m, inv, binv), B, step) : -INFINITY;
        __syncwarp();
        // lane: row rr + lane / 4, 16-byte group lane % 4 (8 codes) of it
        const int sub = lane >> 2, cg = lane & 3;
#pragma unroll
        for (int rr = 0; rr < 32; rr += 8) {
            const int r = rr + sub;
            uint16_t* dst = reinterpret_cast<uint16_t*>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(drow), r));
            const int rs2 = r >> 1;
            uint4 q = reinterpret_cast<const uint4*>(stage + r * kEpiWords)[cg ^ (rs2 >> 2)];
            // logical word e of the group is physical word e ^ (rs2 & 3): undo the XOR by two swaps
            if (rs2 & 1) {
                const uint32_t t0 = q.x, t2 = q.z;
                q.x = q.y; q.y = t0; q.z = q.w; q.w = t2;
            }
            if (rs2 & 2) {
                const uint32_t t0 = q.x, t1 = q.y;
                q.x = q.z; q.y = q.w; q.z = t0; q.w = t1;
            }
            if (dst) *reinterpret_cast<uint4*>(dst + col0 + cg * 8) = q;
        }
        __syncwarp();
    }

    __device__ void done(int, int) {}
};

template <class Kind>
__global__ void __launch_bounds__(ScorePlan<Kind>::kThreads, 1)
    tc_score_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                    const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo, int kchunks,
                    TcArgs args, int* err) {
    using Plan = ScorePlan<Kind>;
    extern __shared__ unsigned char smem[];
    __shared__ tc::Ctl ctl;
    TcSched sched{&args};
    TcEpi<Plan::kEpiWarps> epi;
    epi.a = &args;
    // transpose staging after the engine's stages (1024-byte aligned start), one slice per epilogue warp
    unsigned char* aligned = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem) + 1023) &
                                                              ~(uintptr_t)1023);
    epi.stage = reinterpret_cast<uint32_t*>(aligned + (Plan::kStageBytes - 1024)) +
                (size_t)(threadIdx.x >= 64 ? (threadIdx.x >> 5) - 2 : 0) * 32 * kEpiWords;
    tc::gemm_tiles<Kind, TcSched, TcEpi<Plan::kEpiWarps>, Plan::kEpiWarps, Plan::kStages>(
        &mAhi, &mAlo, &mBhi, &mBlo, kchunks, sched, epi, err, smem, ctl);
}


// Exact re-score of the selected lists (tensor-core paths): the 3xTF32 and
// FP16 paths select the ks best approximate scores plus a guard band of twice
// their error bound, the served BF16 form a shortlist of rerank * k; every
// listed id is scored again here on the CUDA cores with exactly the SIMT
// path's arithmetic, the list re-sorted (score descending, id ascending) and
// the best k kept.  One block per query; a list holds its entries first, then
// -1s (S slots).  The block first resolves every listed id to its corpus row
// (key[r] = row << 32 | id, ~0 for none), so a warp's row loads do not wait on
// the id and row-map loads; with d <= 32 kV float4 per lane (kV > 0) a warp
// issues all loads of its two rows before the first product.
template <int kV>
__global__ void __launch_bounds__(512) rescore_kernel(const float* __restrict__ Q, const float* __restrict__ X,
                                                      const int32_t* __restrict__ row_of, int d, int S,
                                                      const int64_t* in_ids, int k, int64_t* out_ids,
                                                      float* out_scores, int64_t n,
                                                      unsigned long long* bounds, const int32_t* __restrict__ qorder) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_nr;
    float* qv = reinterpret_cast<float*>(smem);
    uint64_t* key = reinterpret_cast<uint64_t*>(smem + align_up_dev((size_t)d * 4, 16));
    const int64_t q = qorder ? qorder[blockIdx.x] : blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int d4 = d / 4;
    if (tid == 0) s_nr = 0;
    for (int i = tid; i < d4; i += blockDim.x)
        reinterpret_cast<float4*>(qv)[i] = reinterpret_cast<const float4*>(Q + q * d)[i];
    __syncthreads();
    // the list holds its entries first, then -1s
    for (int r = tid; r < S; r += blockDim.x) {
        int64_t id = in_ids[q * S + r];
        if (id >= 0) atomicMax(&s_nr, r + 1);
        if (id >= n) {
            atomicAdd(bounds, 1ull);
            id = -1;
        }
        key[r] = id >= 0 ? ((uint64_t)(uint32_t)row_of[id] << 32) | (uint64_t)(uint32_t)id : ~0ull;
    }
    __syncthreads();
    const int nr = s_nr;
    // two rows per warp at a time (each row's sum in the SIMT path's order)
    const float4* y4 = reinterpret_cast<const float4*>(qv);
    for (int r0 = 2 * warp; r0 < nr; r0 += 2 * nwarps) {
        uint64_t kv[2];
        const float4* x4[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            kv[h] = r0 + h < nr ? key[r0 + h] : ~0ull;
            x4[h] = kv[h] != ~0ull ? reinterpret_cast<const float4*>(X + (int64_t)(kv[h] >> 32) * d) : nullptr;
        }
        float acc[2] = {0.f, 0.f};
        if constexpr (kV > 0) {
            float4 xv[2][kV];
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int t = 0; t < kV; ++t)
                    xv[h][t] = x4[h] && lane + 32 * t < d4 ? __ldg(x4[h] + lane + 32 * t)
                                                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int t = 0; t < kV; ++t) {
                if (lane + 32 * t >= d4) break;
                const float4 y = y4[lane + 32 * t];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    acc[h] = fmaf(xv[h][t].x, y.x, acc[h]);
                    acc[h] = fmaf(xv[h][t].y, y.y, acc[h]);
                    acc[h] = fmaf(xv[h][t].z, y.z, acc[h]);
                    acc[h] = fmaf(xv[h][t].w, y.w, acc[h]);
                }
            }
        } else {
            for (int i = lane; i < d4; i += 32) {
                const float4 y = y4[i];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!x4[h]) continue;
                    const float4 x = __ldg(x4[h] + i);
                    acc[h] = fmaf(x.x, y.x, acc[h]);
                    acc[h] = fmaf(x.y, y.y, acc[h]);
                    acc[h] = fmaf(x.z, y.z, acc[h]);
                    acc[h] = fmaf(x.w, y.w, acc[h]);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            for (int o = 16; o > 0; o >>= 1) acc[h] += __shfl_xor_sync(0xffffffffu, acc[h], o);
            if (lane == 0 && r0 + h < nr)
                key[r0 + h] = x4[h] ? ((uint64_t)(~float_order(acc[h])) << 32) | (kv[h] & 0xffffffffull) : ~0ull;
        }
    }
    const int SP = nr > 1 ? next_pow2_dev(nr) : 1;
    for (int u = nr + tid; u < SP; u += blockDim.x) key[u] = ~0ull;
    if (nr == 0 && tid == 0) key[0] = ~0ull;
    __syncthreads();
    block_bitonic(key, SP);
    for (int r = tid; r < k; r += blockDim.x) {
        const uint64_t kv = r < nr ? key[r] : ~0ull;
        if (kv == ~0ull) {
            out_ids[q * k + r] = -1;
            out_scores[q * k + r] = -INFINITY;
        } else {
            out_ids[q * k + r] = (int64_t)(uint32_t)kv;
            out_scores[q * k + r] = float_from_order(~(uint32_t)(kv >> 32));
        }
    }
}

// rescore_kernel's instance for a dimension: all loads of a row pair in
// flight at once when d <= 1024.
inline const void* rescore_fn(int d) {
    switch ((d / 4 + 31) / 32) {
        case 1: return (const void*)rescore_kernel<1>;
        case 2: return (const void*)rescore_kernel<2>;
        case 3: return (const void*)rescore_kernel<3>;
        case 4: return (const void*)rescore_kernel<4>;
        case 5: return (const void*)rescore_kernel<5>;
        case 6: return (const void*)rescore_kernel<6>;
        case 7: return (const void*)rescore_kernel<7>;
        case 8: return (const void*)rescore_kernel<8>;
        default: return (const void*)rescore_kernel<0>;
    }
}

// The candidates of one (query, probed cluster) pair for the selects: the
// pair's dense row of approximate scores over its cluster's positions and its
// candidate bitmap (both written per pair slot, see mark_kernel and TcEpi).
struct DenseArgs {
    const uint16_t* dense;
    const float* qbound;        // per query: the codes' range bound B
    const float* cmax;
    const uint32_t* bitmap;
    const int64_t* bm_off;
    const int32_t* off;
    const int32_t* slot_of;
    const int32_t* route;
    const int64_t* cl_off;
    const int64_t* orig_id;
    const int32_t* ucount;      // candidates per pair
    // guarded modes: queries whose band did not fit their list, each with the
    // band's lower score bound (rescore_band_kernel re-scores them)
    int32_t* ovf;
    float* ovf_thr;
    int32_t* ovf_count;
};

// A guarded query whose band (every candidate scoring at least t) outgrew its
// list: listed for the exact re-score of the whole band.
__device__ __forceinline__ void record_overflow(const DenseArgs& d, int64_t q, float t) {
    if (!d.ovf) return;
    const int i = atomicAdd(d.ovf_count, 1);
    d.ovf[i] = (int32_t)q;
    d.ovf_thr[i] = t;
}

struct PairRow {
    const uint16_t* row;        // score codes (score_code)
    const uint32_t* bm;
    const float* cm;            // best candidate score per bitmap word
    int64_t cb;                 // first row of the cluster in the reordered corpus
    int n_c;
};

__device__ __forceinline__ PairRow pair_row(const DenseArgs& d, int64_t pair) {
    const int32_t slot = d.slot_of[pair];
    const int j = d.route[pair];
    const int64_t cb = d.cl_off[j];
    const int64_t n_c = d.cl_off[j + 1] - cb;
    const int64_t wbase = d.bm_off[j] + (int64_t)(slot - d.off[j]) * bitmap_words(n_c);
    return PairRow{d.dense + wbase * 32, d.bitmap + wbase, d.cmax + wbase, cb, (int)n_c};
}

__device__ __forceinline__ bool is_cand(const PairRow& r, int pos) { return (r.bm[pos >> 5] >> (pos & 31)) & 1u; }

__device__ __forceinline__ uint64_t sel_key(float sc, uint32_t low) {
    return ((uint64_t)(~float_order(sc)) << 32) | (uint64_t)low;
}

// Exact re-score of a guarded query's whole band, for the queries whose band
// outgrew the list the selects hand to rescore_kernel (listed by
// record_overflow; none in ordinary workloads, many under massive near-ties):
// every candidate of the query's c pairs whose approximate score (its code
// mapped back) is at least the band's bound t is scored exactly, with
// rescore_kernel's arithmetic, and the k best (score descending, id ascending)
// replace what rescore_kernel wrote.  One block per listed query (grid-stride
// over the list); candidates are taken kBandChunk positions of the pairs at a
// time, scored, and merged with the k best so far by a block sort.
constexpr int kBandChunk = 1024;

__global__ void __launch_bounds__(256) rescore_band_kernel(DenseArgs da, const float* __restrict__ Q,
                                                           const float* __restrict__ X, int d, int c, int k,
                                                           int64_t* __restrict__ out_ids,
                                                           float* __restrict__ out_scores) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PairRow s_pr[LIDER_MAX_C];
    __shared__ int s_n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    // key: the KB (>= k) best so far, then the chunk's keys, then leftovers of
    // earlier sorts (all exact, none twice); 2 kBandChunk >= KB + kBandChunk
    const int KB = next_pow2_dev(k);
    constexpr int kSort = 2 * kBandChunk;
    float* qv = reinterpret_cast<float*>(smem);
    uint64_t* key = reinterpret_cast<uint64_t*>(smem + align_up_dev((size_t)d * 4, 16));
    int32_t* crow = reinterpret_cast<int32_t*>(key + kSort);            // the chunk's cluster positions
    const int n_ovf = *da.ovf_count;
    const int d4 = d / 4;
    for (int oi = blockIdx.x; oi < n_ovf; oi += gridDim.x) {
        const int64_t q = da.ovf[oi];
        const float t = da.ovf_thr[oi];
        const float cB = da.qbound[q] > 0.f ? da.qbound[q] : 1.f, cstep = code_step(cB);
        __syncthreads();                              // the previous query's reads are done
        for (int i = tid; i < d4; i += blockDim.x)
            reinterpret_cast<float4*>(qv)[i] = reinterpret_cast<const float4*>(Q + q * d)[i];
        for (int i = tid; i < kSort; i += blockDim.x) key[i] = ~0ull;
        if (tid < c) s_pr[tid] = pair_row(da, q * c + tid);
        __syncthreads();
        for (int p = 0; p < c; ++p) {
            const PairRow pr = s_pr[p];
            for (int base = 0; base < pr.n_c; base += kBandChunk) {
                if (tid == 0) s_n = 0;
                __syncthreads();
                for (int pos = base + tid; pos < min(pr.n_c, base + kBandChunk); pos += blockDim.x) {
                    if (is_cand(pr, pos) && code_score(pr.row[pos], cB, cstep) >= t)
                        crow[atomicAdd(&s_n, 1)] = pos;
                }
                __syncthreads();
                const int nb = s_n;
                __syncthreads();                       // every thread has read s_n
                if (nb == 0) continue;                 // the same in every thread
                // exact scores, one row per warp, in rescore_kernel's order
                const float4* y4 = reinterpret_cast<const float4*>(qv);
                for (int r = warp; r < kBandChunk; r += nwarps) {
                    if (r >= nb) {
                        if (lane == 0) key[KB + r] = ~0ull;
                        continue;
                    }
                    const int64_t row = pr.cb + crow[r];
                    const float4* x4 = reinterpret_cast<const float4*>(X + row * d);
                    float acc = 0.f;
                    for (int i = lane; i < d4; i += 32) {
                        const float4 y = y4[i];
                        const float4 x = __ldg(x4 + i);
                        acc = fmaf(x.x, y.x, acc);
                        acc = fmaf(x.y, y.y, acc);
                        acc = fmaf(x.z, y.z, acc);
                        acc = fmaf(x.w, y.w, acc);
                    }
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0) key[KB + r] = sel_key(acc, (uint32_t)__ldg(da.orig_id + row));
                }
                __syncthreads();
                block_bitonic(key, kSort);             // the KB best of all lead
            }
        }
        for (int r = tid; r < k; r += blockDim.x) {
            const uint64_t kv = key[r];
            out_ids[q * k + r] = kv == ~0ull ? -1 : (int64_t)(uint32_t)kv;
            out_scores[q * k + r] = kv == ~0ull ? -INFINITY : float_from_order(~(uint32_t)(kv >> 32));
        }
    }
}

// Load the pair rows of query q into s_pr (threads 0..c-1) and the candidate
// total (thread 0); returns nothing, callers __syncthreads().
__device__ __forceinline__ void load_pairs(const DenseArgs& d, int64_t q, int c, PairRow* s_pr, int* s_total,
                                           int32_t* trace_ucount, bool count, unsigned long long* counters) {
    const int tid = threadIdx.x;
    if (tid < c) s_pr[tid] = pair_row(d, q * c + tid);
    if (tid == 0) {
        int o = 0;
        for (int p = 0; p < c; ++p) {
            const int U = d.ucount[q * c + p];
            o += U;
            if (trace_ucount) trace_ucount[q * c + p] = U;
        }
        *s_total = o;
        if (count) atomicAdd(&counters[CNT_CANDIDATES], (unsigned long long)o);
    }
}

// Per-query selection (tensor paths), multi-level fallback: the ks best keys
// over the candidates of the query's c pairs.  Bucket selection on the score
// between the best and the worst candidate finds the bucket holding the ks-th
// key; a crowded bucket is refined (up to three levels, each a new histogram
// of that bucket's keys).  The selected keys, mapped to corpus ids, are sorted
// (score descending, id ascending).  One block per query of `redo`.
constexpr int kSelCap = 4096;
constexpr int kSelLevels = 3;

__global__ void __launch_bounds__(256) select_query_kernel(DenseArgs da, int c, int ks,
                                                           const float* __restrict__ qguard, int guarded, int so,
                                                           int64_t* __restrict__ out_ids, float* __restrict__ out_scores,
                                                           int32_t* __restrict__ trace_ucount,
                                                           const int32_t* __restrict__ redo,
                                                           const int32_t* __restrict__ redo_count,
                                                           unsigned long long* counters) {
    __shared__ uint64_t keys[kSelCap];
    __shared__ uint32_t bins[kBins];
    __shared__ float lv_lo[kSelLevels], lv_hi[kSelLevels], lv_scale[kSelLevels];
    __shared__ int lv_sel[kSelLevels];
    __shared__ int s_levels, s_total, s_n;
    __shared__ float s_thr;
    __shared__ int s_band;
    __shared__ uint32_t s_lo_ord, s_hi_ord;
    __shared__ PairRow s_pr[LIDER_MAX_C];
    // redo: the queries select_hist_kernel left to this kernel (block b takes
    // redo[b]); otherwise block b takes query b
    if (redo && (int)blockIdx.x >= *redo_count) return;
    const int64_t q = redo ? redo[blockIdx.x] : blockIdx.x;
    const int tid = threadIdx.x;
    const float cB = da.qbound[q] > 0.f ? da.qbound[q] : 1.f, cstep = code_step(cB);   // the codes' range
    if (tid == 0) { s_lo_ord = 0xffffffffu; s_hi_ord = 0u; s_n = 0; }
    load_pairs(da, q, c, s_pr, &s_total, redo ? nullptr : trace_ucount, !redo, counters);
    __syncthreads();
    // pass 0: score range (as ordered keys)
    uint32_t kmin = 0xffffffffu, kmax = 0u;
    for (int p = 0; p < c; ++p) {
        const PairRow pr = s_pr[p];
        for (int pos = tid; pos < pr.n_c; pos += blockDim.x) {
            if (!is_cand(pr, pos)) continue;
            const uint32_t h = ~float_order(code_score(pr.row[pos], cB, cstep));
            kmin = min(kmin, h);
            kmax = max(kmax, h);
        }
    }
    atomicMin(&s_lo_ord, kmin);
    atomicMax(&s_hi_ord, kmax);
    __syncthreads();
    const int total = s_total;
    const int need = min(ks, total);
    // level l: keys whose score lies in [lv_lo, lv_hi]; bucket = (hi - s) * scale
    auto bucket = [&](int l, float sc) -> uint32_t {
        const float x = __fmul_rn(__fadd_rn(lv_hi[l], -sc), lv_scale[l]);
        return (uint32_t)fminf(fmaxf(x, 0.f), (float)(kBins - 1));
    };
    // status of a key after the first `levels` levels: 1 selected, 0 rejected, 2 undecided
    auto status = [&](float sc, int levels) -> int {
        for (int l = 0; l < levels; ++l) {
            if (sc > lv_hi[l]) return 1;
            const uint32_t b = bucket(l, sc);
            if (b < (uint32_t)lv_sel[l]) return 1;
            if (b > (uint32_t)lv_sel[l]) return 0;
        }
        return 2;
    };
    if (tid == 0) {
        lv_hi[0] = float_from_order(~s_lo_ord);       // best score
        lv_lo[0] = float_from_order(~s_hi_ord);       // worst score
        s_levels = 0;
    }
    __syncthreads();
    int above = 0;
    for (int l = 0; l < kSelLevels && need > 0; ++l) {
        if (tid == 0) {
            const float span = lv_hi[l] - lv_lo[l];
            lv_scale[l] = span > 0.f ? (float)kBins / span : 0.f;
        }
        for (int b = tid; b < kBins; b += blockDim.x) bins[b] = 0u;
        __syncthreads();
        for (int p = 0; p < c; ++p) {
            const PairRow pr = s_pr[p];
            for (int pos = tid; pos < pr.n_c; pos += blockDim.x) {
                if (!is_cand(pr, pos)) continue;
                const float sc = code_score(pr.row[pos], cB, cstep);
                if (status(sc, l) == 2) atomicAdd(&bins[bucket(l, sc)], 1u);
            }
        }
        __syncthreads();
        if (tid == 0) {
            uint32_t cum = 0;
            int bsel = kBins - 1;
            for (int b = 0; b < kBins; ++b) {
                if (above + (int)(cum + bins[b]) >= need) { bsel = b; break; }
                cum += bins[b];
            }
            lv_sel[l] = bsel;
            s_levels = l + 1;
            // refine when the chosen bucket would not fit next to everything above it
            if (l + 1 < kSelLevels && above + (int)cum + (int)bins[bsel] > kSelCap && lv_scale[l] > 0.f) {
                lv_hi[l + 1] = __fadd_rn(lv_hi[l], -(float)bsel / lv_scale[l]);
                lv_lo[l + 1] = __fadd_rn(lv_hi[l], -(float)(bsel + 1) / lv_scale[l]);
                s_n = above + (int)cum;          // keys above the refined bucket
            } else {
                s_n = -1;                        // done
            }
        }
        __syncthreads();
        if (s_n < 0) break;
        above = s_n;
        __syncthreads();
    }
    __syncthreads();                 // every thread has read the loop's last flag
    const int levels = s_levels;
    if (tid == 0) {
        s_n = 0;
        // guard band: every key whose approximate score is within twice the
        // error bound of the chosen bucket's lower edge (and so of the ks-th
        // key) joins the list, so the exact re-score sees the exact top ks
        s_thr = INFINITY;
        if (guarded && levels > 0) {
            const int l = levels - 1;
            const float edge = lv_scale[l] > 0.f ? __fadd_rn(lv_hi[l], -(float)(lv_sel[l] + 1) / lv_scale[l])
                                                 : lv_lo[l];
            s_thr = edge - 2.f * qguard[q];
        }
    }
    __syncthreads();
    const float thr = s_thr;
    // collect the selected keys as (score, corpus id) keys: first those better
    // than the last chosen bucket (fewer than ks), then that bucket's keys
    // while room remains (overflow only drops keys of equal bucket, the last
    // refinement's resolution)
    for (int pass = 0; pass < 2 && need > 0; ++pass) {
        for (int p = 0; p < c; ++p) {
            const PairRow pr = s_pr[p];
            for (int pos = tid; pos < pr.n_c; pos += blockDim.x) {
                if (!is_cand(pr, pos)) continue;
                const float sc = code_score(pr.row[pos], cB, cstep);
                const int st = status(sc, levels);
                bool take;
                if (st == 2) {
                    const uint32_t b = bucket(levels - 1, sc), bs = (uint32_t)lv_sel[levels - 1];
                    take = pass == 0 ? b < bs : (b == bs || (b > bs && sc >= thr));
                } else {
                    take = pass == 0 ? st == 1 : (st == 0 && sc >= thr);
                }
                if (take) {
                    const int slot = atomicAdd(&s_n, 1);
                    if (slot < kSelCap) keys[slot] = sel_key(sc, (uint32_t)da.orig_id[pr.cb + pos]);
                }
            }
        }
        __syncthreads();
    }
    __syncthreads();
    const int n = max(0, min(s_n, kSelCap));
    const bool spilled = s_n > kSelCap;
    const int SP = n > 1 ? next_pow2_dev(n) : 1;
    for (int u = n + tid; u < SP; u += blockDim.x) keys[u] = ~0ull;
    __syncthreads();
    block_bitonic(keys, SP);
    // guard mode: keep every key within twice the error bound of the ks-th
    // best approximate score (the exact top ks is among them); else the ks best
    int keep = min(need, n);
    if (guarded && keep > 0) {
        const float vk = float_from_order(~(uint32_t)(keys[keep - 1] >> 32));
        const float t = vk - 2.f * qguard[q];
        if (tid == 0) s_band = keep;
        __syncthreads();
        for (int r = keep + tid; r < n; r += blockDim.x)
            if (float_from_order(~(uint32_t)(keys[r] >> 32)) >= t) atomicMax(&s_band, r + 1);
        __syncthreads();
        const int band = s_band;
        if (tid == 0 && (spilled || band > so)) {
            atomicAdd(&counters[CNT_SEL_OVERFLOW], 1ull);
            record_overflow(da, q, t);
        }
        keep = min(band, so);
    }
    for (int r = tid; r < so; r += blockDim.x) {
        if (r < keep) {
            const uint64_t kv = keys[r];
            out_ids[q * so + r] = (int64_t)(uint32_t)kv;
            out_scores[q * so + r] = float_from_order(~(uint32_t)(kv >> 32));
        } else {
            out_ids[q * so + r] = -1;
            out_scores[q * so + r] = -INFINITY;
        }
    }
}

// Per-query selection (tensor paths).  The bins are fixed by a bound B >=
// |approximate score| of the query (no range pass): bin = floor((B - score) *
// kHistBins / 2B), bin 0 holding the best scores.  Way 1 (small ks) bins the
// per-chunk candidate maxima, way 2 every candidate; the bin where the count
// reaches ks fixes a threshold (lowered by the guard band and one bin, or
// sub-bin, for rounding), and the candidates above it are collected in
// shared memory.  A query whose collection would exceed kHistCand is appended
// to `redo` and left to select_query_kernel.
constexpr int kHistBins = 2048;
constexpr int kHistCand = 2048;

// The r-th smallest (1-based, counting repeats) of n 32-bit words word(i),
// i < n, by a block-wide radix select: the bits the smallest and the largest
// word share are the answer's; passes over the next digits of up to 8 bits,
// most significant first, each count the words that match the bits chosen so
// far in a 256-bin shared histogram.  All threads call it; r in [1, n].
// `passes` < 4 stops once the bits at or above 32 - 8 passes are chosen: the
// result is then the largest word sharing the r-th smallest word's bits down
// to the last digit taken, an upper bound on it.
template <class Word>
__device__ __forceinline__ uint32_t block_kth_smallest(Word word, int n, int r, uint32_t* hist256, int* s_pick,
                                                     int passes = 4) {
    __shared__ uint32_t s_lohi[2];
    const int tid = threadIdx.x, lane = tid & 31;
    // the words' common leading bits (those of their minimum and maximum) are
    // the answer's; the digit passes start below them
    uint32_t lo = 0xffffffffu, hi = 0u;
    for (int i = tid; i < n; i += blockDim.x) {
        const uint32_t v = word(i);
        lo = min(lo, v);
        hi = max(hi, v);
    }
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if (tid == 0) {
        s_lohi[0] = 0xffffffffu;
        s_lohi[1] = 0u;
    }
    __syncthreads();
    if (lane == 0) {
        atomicMin(&s_lohi[0], lo);
        atomicMax(&s_lohi[1], hi);
    }
    __syncthreads();
    lo = s_lohi[0];
    hi = s_lohi[1];
    __syncthreads();                               // every thread has read s_lohi
    if (lo == hi) return lo;
    const int target = 32 - 8 * passes;            // bits at or above it are resolved
    int top = 31 - __clz(lo ^ hi), low;
    uint32_t mask = top == 31 ? 0u : ~((2u << top) - 1u), prefix = lo & mask;
    do {
        low = max(top - 7, 0);
        const uint32_t dm = (2u << (top - low)) - 1u;   // the digit's bits
        for (int b = tid; b < 256; b += blockDim.x) hist256[b] = 0u;
        __syncthreads();
        // one atomic per distinct digit of a warp's words
        for (int i0 = tid - lane; i0 < n; i0 += blockDim.x) {
            const int i = i0 + lane;
            uint32_t dig = 0xffffffffu;
            if (i < n) {
                const uint32_t v = word(i);
                if ((v & mask) == prefix) dig = (v >> low) & dm;
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, dig);
            if (dig != 0xffffffffu && lane == __ffs(peers) - 1) atomicAdd(&hist256[dig], (uint32_t)__popc(peers));
        }
        __syncthreads();
        if (tid < 32) {
            // lane owns bins 8 lane .. 8 lane + 7; the first bin whose running
            // count reaches r holds the r-th smallest
            uint32_t cnt[8], sum = 0u;
#pragma unroll
            for (int b = 0; b < 8; ++b) { cnt[b] = hist256[8 * lane + b]; sum += cnt[b]; }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t run = incl - sum;
            const bool mine = run < (uint32_t)r && incl >= (uint32_t)r;
            if (mine) {
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    if (run + cnt[b] >= (uint32_t)r) {
                        s_pick[0] = 8 * lane + b;
                        s_pick[1] = r - (int)run;
                        break;
                    }
                    run += cnt[b];
                }
            }
        }
        __syncthreads();
        prefix |= (uint32_t)s_pick[0] << low;
        mask |= dm << low;
        r = s_pick[1];
        __syncthreads();                           // every thread has read s_pick
        top = low - 1;
    } while (low > target);
    return low > 0 ? prefix | ((1u << low) - 1u) : prefix;
}

__global__ void __launch_bounds__(512) select_hist_kernel(
        DenseArgs da, int c, int ks, const float* __restrict__ qguard, const float* __restrict__ qbound, int guarded,
        int so, int64_t* __restrict__ out_ids, float* __restrict__ out_scores, int32_t* __restrict__ trace_ucount,
        int32_t* __restrict__ redo, int32_t* __restrict__ redo_count, unsigned long long* counters) {
    __shared__ uint32_t hist[kHistBins];          // bin counts; then (way 1) the listed chunks
    __shared__ uint64_t cand[kHistCand];          // collected keys
    __shared__ PairRow s_pr[LIDER_MAX_C];
    __shared__ int s_total, s_cnt, s_bt, s_band, s_nh, s_ct;
    __shared__ float s_thr;
    __shared__ uint32_t s_rhist[256];              // radix select; sub-bins of the chosen bin
    __shared__ int s_pick[2];
    __shared__ int s_wo[LIDER_MAX_C + 1];          // first chunk-maximum word of each pair
    const int64_t q = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31;
    for (int b = tid; b < kHistBins; b += blockDim.x) hist[b] = 0u;
    if (tid == 0) s_cnt = 0;
    load_pairs(da, q, c, s_pr, &s_total, trace_ucount, true, counters);
    __syncthreads();
    const int total = s_total;
    const int need = min(ks, total);
    const float B = qbound[q];
    const float scale = B > 0.f ? (float)kHistBins / (2.f * B) : 0.f;
    const float cB = B > 0.f ? B : 1.f, cstep = code_step(cB);   // the score codes' range
    auto bin_of = [&](float sc) -> int {
        const float x = __fmul_rn(__fadd_rn(B, -sc), scale);
        return (int)fminf(fmaxf(x, 0.f), (float)(kHistBins - 1));
    };
    // The passes read a pair's row as float4 groups (4 positions; the row
    // pitch is a multiple of 32 and positions past n_c have no bitmap bit),
    // kU groups per thread in flight; the bitmap only decides which count.
    constexpr int kU = 4;
    const int bd = blockDim.x;
    auto load_groups = [&](const PairRow& pr, int g0, float4 (&sc)[kU], uint32_t (&wv)[kU]) {
        const int ng = (pr.n_c + 3) >> 2;
#pragma unroll
        for (int r = 0; r < kU; ++r) {
            const int g = g0 + r * bd;
            wv[r] = 0u;
            if (g < ng) {
                wv[r] = (__ldg(pr.bm + (g >> 3)) >> ((g & 7) * 4)) & 0xfu;
                const uint2 cd = __ldg(reinterpret_cast<const uint2*>(pr.row) + g);
                sc[r] = make_float4(code_score(cd.x & 0xffffu, cB, cstep), code_score(cd.x >> 16, cB, cstep),
                                    code_score(cd.y & 0xffffu, cB, cstep), code_score(cd.y >> 16, cB, cstep));
            }
        }
    };
    auto comp = [](const float4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; };
    // Way 1 (need <= 4 * blockDim), on the chunk maxima the tensor epilogue
    // wrote (per pair and 32 positions, the best candidate score there): a
    // histogram of the maxima over the query's bins; the bin where their
    // count reaches `need` holds a score reached by at least `need` distinct
    // candidates (one per chunk), so the ks-th best is not below its lower
    // edge.  Every candidate at or above that edge less twice the guard (and
    // one bin for rounding) lies in a chunk whose maximum falls in a bin up to
    // the last one to collect: only those chunks are read.
    constexpr int kKeep = 4;
    bool small_lists = true;                        // positions fit the (list, position) packing
    for (int p = 0; p < c; ++p) small_lists = small_lists && s_pr[p].n_c < (1 << 27);
    const bool by_max = need > 0 && need <= kKeep * bd && small_lists;
    // The chunk maxima of the c pairs as one sequence of words: word g is
    // word g - s_wo[p] of pair p, for the p with s_wo[p] <= g < s_wo[p + 1].
    constexpr int kBatch = 4;
    if (tid == 0) {
        int o = 0;
        for (int p = 0; p < c; ++p) {
            s_wo[p] = o;
            o += (s_pr[p].n_c + 31) >> 5;
        }
        s_wo[c] = o;
    }
    __syncthreads();
    const int n_words = s_wo[c];
    // (pair, word) of word g; p is a hint, never past g's pair (the scans
    // below visit each thread's words in increasing order)
    auto word_at = [&](int g, int& p, int& w) {
        while (g >= s_wo[p + 1]) ++p;
        w = g - s_wo[p];
    };
    if (by_max) {
        // a thread's words g = tid + r bd: up to kRegW of them stay in
        // registers (loads all in flight), more are read again below
        constexpr int kRegW = 16;
        const bool in_regs = n_words <= kRegW * bd;
        float vm[kRegW];
        int hp = 0;                                 // this thread's current pair
        if (in_regs) {
#pragma unroll
            for (int r = 0; r < kRegW; ++r) {
                const int g = tid + r * bd;
                vm[r] = -INFINITY;
                if (g < n_words) {
                    int w;
                    word_at(g, hp, w);
                    vm[r] = __ldg(s_pr[hp].cm + w);
                }
            }
#pragma unroll
            for (int r = 0; r < kRegW; ++r)
                if (vm[r] > -INFINITY) atomicAdd(&hist[bin_of(vm[r])], 1u);
        } else {
            for (int g0 = tid; g0 < n_words; g0 += kBatch * bd) {
                float vb[kBatch];
#pragma unroll
                for (int r = 0; r < kBatch; ++r) {
                    const int g = g0 + r * bd;
                    vb[r] = -INFINITY;
                    if (g < n_words) {
                        int w;
                        word_at(g, hp, w);
                        vb[r] = __ldg(s_pr[hp].cm + w);
                    }
                }
#pragma unroll
                for (int r = 0; r < kBatch; ++r)
                    if (vb[r] > -INFINITY) atomicAdd(&hist[bin_of(vb[r])], 1u);
            }
        }
        __syncthreads();
        // the first bin where the maxima's count reaches need (none: fewer
        // chunks with candidates than need, take all), 32 bins per step
        if (tid < 32) {
            uint32_t cum = 0u;
            int bsel = -1;
            for (int b0 = 0; b0 < kHistBins; b0 += 32) {
                uint32_t v = hist[b0 + lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += t;
                }
                const unsigned reach = __ballot_sync(0xffffffffu, cum + v >= (uint32_t)need);
                if (reach) {
                    const int l = __ffs(reach) - 1;
                    bsel = b0 + l;
                    cum += __shfl_sync(0xffffffffu, v, l) - hist[bsel];   // maxima before bin bsel
                    break;
                }
                cum += __shfl_sync(0xffffffffu, v, 31);
            }
            for (int u = lane; u < 256; u += 32) s_rhist[u] = 0u;
            if (lane == 0) {
                s_bt = bsel;
                s_band = (int)cum;
            }
        }
        __syncthreads();
        const int bsel = s_bt;
        // bin bsel split into 256 sub-bins (the maxima held in registers, or
        // read again)
        const bool refine = bsel >= 0 && scale > 0.f;
        auto sub_count = [&](float m) {
            if (m > -INFINITY && bin_of(m) == bsel) {
                const float x = __fmul_rn(__fadd_rn(B, -m), scale);
                const int sub = (int)fminf(fmaxf((x - (float)bsel) * 256.f, 0.f), 255.f);
                atomicAdd(&s_rhist[sub], 1u);
            }
        };
        if (refine && in_regs) {
#pragma unroll
            for (int r = 0; r < kRegW; ++r) sub_count(vm[r]);
        } else if (refine) {
            int hs = 0;
            for (int g0 = tid; g0 < n_words; g0 += kBatch * bd) {
                float vb[kBatch];
#pragma unroll
                for (int r = 0; r < kBatch; ++r) {
                    const int g = g0 + r * bd;
                    vb[r] = -INFINITY;
                    if (g < n_words) {
                        int w;
                        word_at(g, hs, w);
                        vb[r] = __ldg(s_pr[hs].cm + w);
                    }
                }
#pragma unroll
                for (int r = 0; r < kBatch; ++r) sub_count(vb[r]);
            }
        }
        __syncthreads();
        if (tid < 32) {
            // the sub-bin where the count reaches need (lane owns 8 sub-bins)
            int sub_sel = 255;
            if (refine) {
                uint32_t cnt[8], sum = 0u;
#pragma unroll
                for (int u = 0; u < 8; ++u) { cnt[u] = s_rhist[8 * lane + u]; sum += cnt[u]; }
                uint32_t incl = sum;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const uint32_t r = (uint32_t)(need - s_band);
                uint32_t run = incl - sum;
                int mine = -1;
                if (run < r && incl >= r) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        if (run + cnt[u] >= r) { mine = 8 * lane + u; break; }
                        run += cnt[u];
                    }
                }
                const unsigned who = __ballot_sync(0xffffffffu, mine >= 0);
                if (who) sub_sel = __shfl_sync(0xffffffffu, mine, __ffs(who) - 1);
            }
            if (lane == 0) {
                // the score threshold: the chosen (sub-)bin's lower edge, less
                // one (sub-)bin for rounding and, in guarded modes, twice the guard
                float thr = -INFINITY;
                if (bsel >= 0 && scale > 0.f) {
                    const float fb = refine ? (float)bsel + (float)(sub_sel + 2) / 256.f : (float)(bsel + 2);
                    thr = __fadd_rn(B, -fb / scale);
                    if (guarded) thr = thr - 2.f * qguard[q];
                }
                s_thr = thr;
                s_nh = 0;
                // the largest code whose score clears thr (-1: none), code_score
                // being non-increasing in the code
                int lo = -1, hi = 65536;
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (code_score((uint32_t)mid, cB, cstep) >= thr) lo = mid;
                    else hi = mid;
                }
                s_ct = lo;
            }
        }
        __syncthreads();
        const float thr = s_thr;
        const int ct = s_ct;
        // the chunks whose maximum clears thr, as one list (pair << 24 |
        // word) in hist, free again once warp 0 has read the counts; a listed
        // chunk holds a candidate to collect, so more than kHistCand of them
        // overflow the collection below as well
        auto list_hit = [&](float m, int p, int w) {
            if (m > -INFINITY && m >= thr) {                 // (-inf: past the words, or no candidate)
                const int i = atomicAdd(&s_nh, 1);
                if (i < kHistBins) hist[i] = ((uint32_t)p << 24) | (uint32_t)w;
            }
        };
        int hq = 0;                                 // this thread's current pair
        if (in_regs) {
#pragma unroll
            for (int r = 0; r < kRegW; ++r) {
                const int g = tid + r * bd;
                if (g < n_words && vm[r] > -INFINITY) {
                    int w;
                    word_at(g, hq, w);
                    list_hit(vm[r], hq, w);
                }
            }
        } else {
            for (int g0 = tid; g0 < n_words; g0 += kBatch * bd) {
                float vb[kBatch];
                int pb[kBatch], wb[kBatch];
#pragma unroll
                for (int r = 0; r < kBatch; ++r) {
                    const int g = g0 + r * bd;
                    vb[r] = -INFINITY;
                    pb[r] = 0;
                    wb[r] = 0;
                    if (g < n_words) {
                        word_at(g, hq, wb[r]);
                        pb[r] = hq;
                        vb[r] = __ldg(s_pr[hq].cm + wb[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < kBatch; ++r) list_hit(vb[r], pb[r], wb[r]);
            }
        }
        __syncthreads();
        const int nh = s_nh;
        if (nh > kHistCand) {
            if (tid == 0) redo[atomicAdd(redo_count, 1)] = (int32_t)q;
            return;
        }
        // the listed chunks, one per thread at a time with all its loads in
        // flight; guarded modes key a candidate by (pair << 27 | position)
        // (the ids of the band are looked up when it is written), the served
        // forms by corpus id (their ties order by it)
        constexpr int kHitBatch = 1;
        for (int i0 = tid; i0 < nh; i0 += kHitBatch * bd) {
            uint4 cd[kHitBatch][4];
            uint32_t bw[kHitBatch], hv[kHitBatch];
#pragma unroll
            for (int u = 0; u < kHitBatch; ++u) {
                const int i = i0 + u * bd;
                bw[u] = 0u;
                hv[u] = 0u;
                if (i < nh) {
                    hv[u] = hist[i];
                    const PairRow& pr = s_pr[hv[u] >> 24];
                    const int w = (int)(hv[u] & 0xffffffu);
                    bw[u] = __ldg(pr.bm + w);
#pragma unroll
                    for (int g8 = 0; g8 < 4; ++g8) cd[u][g8] = __ldg(reinterpret_cast<const uint4*>(pr.row + 32 * w) + g8);
                }
            }
#pragma unroll
            for (int u = 0; u < kHitBatch; ++u) {
                if (!bw[u]) continue;
                const int p = (int)(hv[u] >> 24), w = (int)(hv[u] & 0xffffffu);
                const uint32_t cw[8] = {cd[u][0].x, cd[u][0].y, cd[u][0].z, cd[u][0].w,
                                        cd[u][1].x, cd[u][1].y, cd[u][1].z, cd[u][1].w};
                const uint32_t cw2[8] = {cd[u][2].x, cd[u][2].y, cd[u][2].z, cd[u][2].w,
                                         cd[u][3].x, cd[u][3].y, cd[u][3].z, cd[u][3].w};
                auto code_at = [&](int i) -> uint32_t {
                    const uint32_t x = i < 16 ? cw[i >> 1] : cw2[(i - 16) >> 1];
                    return (i & 1) ? x >> 16 : x & 0xffffu;
                };
                // score >= thr exactly when code <= ct (code_score decreases)
                uint32_t take = 0u;
#pragma unroll
                for (int i = 0; i < 32; ++i)
                    if (((bw[u] >> i) & 1u) && (int)code_at(i) <= ct) take |= 1u << i;
                const int nt = __popc(take);
                if (nt == 0) continue;
                int slot = atomicAdd(&s_cnt, nt);
                const int64_t idb = s_pr[p].cb + 32 * w;
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    if ((take >> i) & 1u) {
                        if (slot < kHistCand)
                            cand[slot] = sel_key(code_score(code_at(i), cB, cstep),
                                                 guarded ? ((uint32_t)p << 27) | (uint32_t)(32 * w + i)
                                                         : (uint32_t)__ldg(da.orig_id + idb + i));
                        ++slot;
                    }
                }
            }
        }
    }
    // Threshold, way 2 (larger need): histogram
    if (need > 0 && !by_max) {
        for (int p = 0; p < c; ++p) {
            const PairRow pr = s_pr[p];
            const int ng = (pr.n_c + 3) >> 2;
            for (int g0 = tid; g0 < ng; g0 += kU * bd) {
                float4 sc[kU];
                uint32_t wv[kU];
                load_groups(pr, g0, sc, wv);
#pragma unroll
                for (int r = 0; r < kU; ++r)
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if ((wv[r] >> i) & 1u) atomicAdd(&hist[bin_of(comp(sc[r], i))], 1u);
            }
        }
    }
    __syncthreads();
    // the bin reaching `need`, then the last bin to collect
    if (tid == 0 && !by_max) {
        int bt = -1;
        if (need > 0) {
            uint32_t cum = 0;
            int bsel = kHistBins - 1;
            for (int b = 0; b < kHistBins; ++b) {
                cum += hist[b];
                if ((int)cum >= need) { bsel = b; break; }
            }
            bt = bsel;
            if (guarded && scale > 0.f) {
                // lower edge of bsel, minus the band and one bin of rounding
                const float edge = __fadd_rn(B, -(float)(bsel + 1) / scale);
                const float t = edge - 2.f * qguard[q] - 1.f / scale;
                bt = max(bsel, bin_of(t));
            }
            uint32_t upto = 0;
            for (int b = 0; b <= bt; ++b) upto += hist[b];
            if ((int)upto > kHistCand) bt = -2;       // too many: the fallback kernel takes this query
        }
        s_bt = bt;
    }
    __syncthreads();
    const int bt = s_bt;
    if (bt == -2) {
        if (tid == 0) redo[atomicAdd(redo_count, 1)] = (int32_t)q;
        return;
    }
    // pass 2: collect the candidates above the threshold (way 1) or in bins
    // 0..bt (way 2) as (score word, corpus id); a warp reserves its keys with
    // one atomic
    if (bt >= 0 && !by_max) {
        for (int p = 0; p < c; ++p) {
            const PairRow pr = s_pr[p];
            const int ng = (pr.n_c + 3) >> 2;
            for (int base0 = 0; base0 < ng; base0 += kU * bd) {
                float4 sc[kU];
                uint32_t wv[kU];
                load_groups(pr, base0 + tid, sc, wv);
                uint32_t take[kU];
                int mine = 0;
#pragma unroll
                for (int r = 0; r < kU; ++r) {
                    take[r] = 0u;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if (!((wv[r] >> i) & 1u)) continue;
                        if (bin_of(comp(sc[r], i)) <= bt) take[r] |= 1u << i;
                    }
                    mine += __popc(take[r]);
                }
                int incl = mine;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int wtotal = __shfl_sync(0xffffffffu, incl, 31);
                int base = 0;
                if (lane == 31 && wtotal) base = atomicAdd(&s_cnt, wtotal);
                base = __shfl_sync(0xffffffffu, base, 31);
                int slot = base + incl - mine;
#pragma unroll
                for (int r = 0; r < kU; ++r) {
                    const int g = base0 + tid + r * bd;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        if ((take[r] >> i) & 1u) {
                            if (slot < kHistCand)
                                cand[slot] = sel_key(comp(sc[r], i), (uint32_t)__ldg(da.orig_id + pr.cb + 4 * g + i));
                            ++slot;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (s_cnt > kHistCand) {                           // way 1 collected too many: fallback kernel
        if (tid == 0) redo[atomicAdd(redo_count, 1)] = (int32_t)q;
        return;
    }
    const int n = min(s_cnt, kHistCand);
    // a key's corpus id (way 1 of the guarded modes keys by pair and position)
    const bool packed = by_max && guarded;
    auto id_of = [&](uint64_t kv) -> int64_t {
        const uint32_t lo = (uint32_t)kv;
        return packed ? __ldg(da.orig_id + s_pr[lo >> 27].cb + (lo & 0x7ffffffu)) : (int64_t)lo;
    };
    if (guarded && need > 0 && n > 0) {
        // Guarded modes: the list is every key within twice the error bound of
        // the need-th best approximate score, in no particular order (the
        // re-score orders it).  The need-th best score comes from a radix
        // select over the keys' score words; only a band longer than the list
        // (counted as an overflow) needs the sort below to keep the best `so`.
        const int keep0 = min(need, n);
        // (three digits: the band's bound at most 2^8 float steps lower, so
        // the band keeps every key it needs and at most a few more)
        const uint32_t wk = block_kth_smallest([&](int i) { return (uint32_t)(cand[i] >> 32); }, n, keep0,
                                               s_rhist, s_pick, 3);
        const float t = float_from_order(~wk) - 2.f * qguard[q];
        if (tid == 0) { s_band = 0; s_bt = 0; }
        __syncthreads();
        int mine = 0;
        for (int r = tid; r < n; r += blockDim.x)
            mine += float_from_order(~(uint32_t)(cand[r] >> 32)) >= t;
        if (mine) atomicAdd(&s_band, mine);
        __syncthreads();
        const int band = s_band;
        if (band <= so) {
            for (int r = tid; r < n; r += blockDim.x) {
                const uint64_t kv = cand[r];
                const float sc = float_from_order(~(uint32_t)(kv >> 32));
                if (sc >= t) {
                    const int slot = atomicAdd(&s_bt, 1);
                    out_ids[q * so + slot] = id_of(kv);
                    out_scores[q * so + slot] = sc;
                }
            }
            for (int r = band + tid; r < so; r += blockDim.x) {
                out_ids[q * so + r] = -1;
                out_scores[q * so + r] = -INFINITY;
            }
            return;
        }
        __syncthreads();
    }
    if (!guarded && need > 0 && n > 0) {
        // Served forms: the list is the `keep` best keys by (score descending,
        // id ascending), in no particular order (the re-rank orders it).  The
        // keep-th smallest 64-bit key comes from two radix selects: its score
        // word, then its id among the keys of that score word.
        const int keep = min(need, n);
        const uint32_t whi = block_kth_smallest([&](int i) { return (uint32_t)(cand[i] >> 32); }, n, keep,
                                                s_rhist, s_pick);
        if (tid == 0) { s_band = 0; s_bt = 0; }
        __syncthreads();
        int less = 0;
        for (int r = tid; r < n; r += blockDim.x) less += (uint32_t)(cand[r] >> 32) < whi;
        if (less) atomicAdd(&s_band, less);
        __syncthreads();
        const int r2 = keep - s_band;                  // >= 1: whi is the keep-th smallest word
        const uint32_t wlo = block_kth_smallest(
            [&](int i) {
                const uint64_t kv = cand[i];
                return (uint32_t)(kv >> 32) == whi ? (uint32_t)kv : 0xffffffffu;   // ids stay below 2^31
            },
            n, r2, s_rhist, s_pick);
        const uint64_t kstar = ((uint64_t)whi << 32) | wlo;
        for (int r = tid; r < n; r += blockDim.x) {
            const uint64_t kv = cand[r];
            if (kv <= kstar) {
                const int slot = atomicAdd(&s_bt, 1);
                out_ids[q * so + slot] = (int64_t)(uint32_t)kv;
                out_scores[q * so + slot] = float_from_order(~(uint32_t)(kv >> 32));
            }
        }
        for (int r = keep + tid; r < so; r += blockDim.x) {
            out_ids[q * so + r] = -1;
            out_scores[q * so + r] = -INFINITY;
        }
        return;
    }
    const int SP = n > 1 ? next_pow2_dev(n) : 1;
    for (int u = n + tid; u < SP; u += blockDim.x) cand[u] = ~0ull;
    __syncthreads();
    block_bitonic(cand, SP);
    int keep = min(need, n);
    if (guarded && keep > 0) {
        // every key within twice the error bound of the ks-th best approximate
        // score (the exact top ks is among them)
        const float vk = float_from_order(~(uint32_t)(cand[keep - 1] >> 32));
        const float t = vk - 2.f * qguard[q];
        if (tid == 0) s_band = keep;
        __syncthreads();
        for (int r = keep + tid; r < n; r += blockDim.x)
            if (float_from_order(~(uint32_t)(cand[r] >> 32)) >= t) atomicMax(&s_band, r + 1);
        __syncthreads();
        const int band = s_band;
        if (tid == 0 && band > so) {
            atomicAdd(&counters[CNT_SEL_OVERFLOW], 1ull);
            record_overflow(da, q, t);
        }
        keep = min(band, so);
    }
    for (int r = tid; r < so; r += blockDim.x) {
        if (r < keep) {
            const uint64_t kv = cand[r];
            out_ids[q * so + r] = id_of(kv);
            out_scores[q * so + r] = float_from_order(~(uint32_t)(kv >> 32));
        } else {
            out_ids[q * so + r] = -1;
            out_scores[q * so + r] = -INFINITY;
        }
    }
}

// ------------------------------------------------------------------ merge --
// Warp per query; lane p < c walks list p (kp entries, sorted best first);
// the ks best heads are written out (score descending, id ascending).
__global__ void merge_kernel(const float* __restrict__ pscore, const int64_t* __restrict__ pid, int64_t nq,
                             int c, int kp, int ks, int64_t* __restrict__ out_ids, float* __restrict__ out_scores) {
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (q >= nq) return;
    const int64_t lbase = (q * c + lane) * (int64_t)kp;
    int head = 0;
    float hs = -INFINITY;
    int64_t hid = -1;
    if (lane < c) { hs = pscore[lbase]; hid = pid[lbase]; }
    for (int r = 0; r < ks; ++r) {
        // best head: score desc, id asc; exhausted lists (id -1) lose
        float bs = hs;
        int64_t bid = hid;
        int bl = lane;
        for (int o = 16; o > 0; o >>= 1) {
            const float os = __shfl_xor_sync(0xffffffffu, bs, o);
            const int64_t oid = __shfl_xor_sync(0xffffffffu, bid, o);
            const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
            bool take;
            if (oid < 0) take = false;
            else if (bid < 0) take = true;
            else take = (os > bs) || (os == bs && oid < bid);
            if (take) { bs = os; bid = oid; bl = ol; }
        }
        if (lane == 0) {
            out_ids[q * ks + r] = bid;
            out_scores[q * ks + r] = bid < 0 ? -INFINITY : bs;
        }
        if (bid < 0) continue;
        if (lane == bl) {
            ++head;
            if (head < kp) { hs = pscore[lbase + head]; hid = pid[lbase + head]; }
            else { hs = -INFINITY; hid = -1; }
        }
    }
}

}  // namespace
}  // namespace lider

namespace lider {

namespace {

struct Workspace {
    unsigned long long* counters;
    int32_t* cnt;
    int32_t* off;
    int32_t* cursor;
    int32_t* item_off;
    double* tq;
    uint64_t* qkeys;
    double* rscore;
    int32_t* route;
    int32_t* pairs;
    int32_t* qorder;        // tensor modes: queries grouped by their best cluster (re-score order)
    int32_t* wstart;
    int32_t* wlen;
    float* pscore;
    int64_t* pid;
    uint64_t* pbuf;
    int64_t* sl_ids;            // tensor paths: per-query list before the re-score (nq x so)
    float* sl_scores;
    float* qscale;              // FP16 path: per-query power-of-two scale
    float* qguard;              // tensor paths: error bound of a query's approximate scores
    float* qbound;              // tensor paths: bound on |approximate score| of a query
    float* qnorm;               // tensor paths: |q| rounded up (hash error bound)
    int32_t* hrecheck;          // tensor paths: hash values recomputed exactly (q * H + h)
    int32_t* n_hrecheck;        // (cleared)
    int32_t* redo;              // tensor paths: queries left to the multi-level select
    int32_t* redo_count;        // (cleared)
    int32_t* ovf_count;         // guarded modes: queries whose band outgrew the list (cleared)
    int32_t* ovf;               //   those queries
    float* ovf_thr;             //   and their bands' lower score bounds
    int32_t* pcount;            // tensor path: candidates per pair (cleared; written by mark_kernel)
    uint16_t* dense;            // tensor paths: per pair slot, approximate score codes over its cluster
    float* cmax;                // tensor paths: per pair slot and bitmap word, the best candidate score
    int32_t* slot_of;           // tensor paths: pair -> its slot in cluster order
    int32_t* unit_off;
    int64_t* bm_off;            // tensor paths: per-cluster bitmap offsets (words)
    uint32_t* bitmap;           // tensor paths: per-pair candidate bitmaps
    int4* units;                // tensor path: tile descriptors
    int4* umeta;                // tensor path: per tile, what the epilogue needs
    float* slot_bound;          // tensor path: per pair slot, its query's code bound
    float* qs_hi;               // tensor routing: queries, TF32 head / tail
    float* qs_lo;
    float* qp_hi;               // tensor path: queries in pair order, TF32 head / tail
    float* qp_lo;
    float* slot_scale;          // FP8 path: per pair slot, the query's scale
    int* tc_err;
    int ncl;
    size_t zero_bytes;   // counters + cnt, cleared at the start of a search
    size_t total;
};

// Carve one allocation into the search buffers (base == nullptr: sizes only).
// List lengths of one search: per pair (kp) and per query before the final
// re-score (ks).  The served BF16 form keeps a shortlist of rerank * k.
struct Shape {
    int mode, R, kp, ks;
    int so;                    // tensor paths: stride of the selected lists (ks + guard band)
    int64_t bitmap_words;      // bound on the candidate bitmaps of one search
};

Shape search_shape(const lider_index* ix, int k, int64_t nq = 0, int c = 0) {
    Shape sh;
    sh.mode = ix->params.score_mode;
    sh.R = ix->params.r0 * k;
    // a query probes c distinct clusters, so its bitmaps take at most the
    // words of the c largest clusters
    sh.bitmap_words = (c > 0 && c <= ix->g.ncl) ? nq * ix->top_words[c] : 0;
    const int T_cap = ix->g.L * sh.R;
    if (sh.mode == LIDER_SCORE_BF16 || sh.mode == LIDER_SCORE_FP8) {
        sh.ks = ix->params.rerank * k;
        sh.kp = std::min(sh.ks, T_cap);
        sh.so = sh.ks;
    } else {
        sh.ks = k;
        sh.kp = k;
        // room for the guard band: 3xTF32's is a few keys, FP16's ~1e-3 |q| |x|
        sh.so = std::min(kSelCap, sh.mode == LIDER_SCORE_F16 ? 4 * k + 64 : 2 * k + 32);
    }
    return sh;
}

// Carve one allocation into the search buffers (base == nullptr: sizes only).
Workspace carve(unsigned char* base, const Geometry& g, int64_t nq, int c, const Shape& sh) {
    Workspace w{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base ? base + o : nullptr;
        o = align_up(o + bytes, 256);
        return p;
    };
    const bool tensor = sh.mode != LIDER_SCORE_SIMT;
    const int64_t np = nq * c;
    w.counters = (unsigned long long*)take(CNT_SLOTS * sizeof(unsigned long long));
    w.cnt = (int32_t*)take((size_t)g.ncl * 4);
    w.tc_err = (int*)take(16);
    w.pcount = tensor ? (int32_t*)take((size_t)np * 4) : nullptr;
    w.redo_count = tensor ? (int32_t*)take(16) : nullptr;
    w.ovf_count = tensor ? (int32_t*)take(16) : nullptr;
    w.n_hrecheck = tensor ? (int32_t*)take(16) : nullptr;
    w.zero_bytes = o;
    w.unit_off = (int32_t*)take((size_t)(g.ncl + 1) * 4);
    w.bm_off = (int64_t*)take((size_t)(g.ncl + 1) * 8);
    w.bitmap = tensor ? (uint32_t*)take((size_t)sh.bitmap_words * 4) : nullptr;
    w.ncl = g.ncl;
    // tiles <= sum_j ceil(cnt_j/128) * ceil(n_c/256) <= (np/128 + ncl) * max_row_tiles
    const size_t max_units = (size_t)((np + tc::kBM - 1) / tc::kBM + g.ncl) * (size_t)g.max_row_tiles;
    w.units = tensor ? (int4*)take(max_units * 16) : nullptr;
    w.umeta = tensor ? (int4*)take(max_units * 16) : nullptr;
    w.slot_bound = tensor ? (float*)take((size_t)np * 4) : nullptr;
    const size_t qelem = sh.mode == LIDER_SCORE_FP8 ? 1 : (sh.mode == LIDER_SCORE_BF16 || sh.mode == LIDER_SCORE_F16) ? 2 : 4;
    w.qp_hi = tensor ? (float*)take((size_t)np * g.d * qelem) : nullptr;
    w.qp_lo = sh.mode == LIDER_SCORE_TENSOR ? (float*)take((size_t)np * g.d * 4) : nullptr;
    w.slot_scale = sh.mode == LIDER_SCORE_FP8 ? (float*)take((size_t)np * 4) : nullptr;
    w.qs_hi = tensor ? (float*)take((size_t)nq * g.d * 4) : nullptr;
    w.qs_lo = tensor ? (float*)take((size_t)nq * g.d * 4) : nullptr;
    w.off = (int32_t*)take((size_t)(g.ncl + 1) * 4);
    w.cursor = (int32_t*)take((size_t)g.ncl * 4);
    w.item_off = (int32_t*)take((size_t)(g.ncl + 1) * 4);
    w.tq = (double*)take((size_t)nq * g.H * 8);
    w.qkeys = (uint64_t*)take((size_t)nq * g.L * 8);
    w.rscore = (double*)take((size_t)nq * g.ncl * 8);
    w.route = (int32_t*)take((size_t)np * 4);
    w.pairs = (int32_t*)take((size_t)np * 4);
    w.qorder = tensor ? (int32_t*)take((size_t)nq * 4) : nullptr;
    w.wstart = (int32_t*)take((size_t)np * g.L * 4);
    w.wlen = (int32_t*)take((size_t)np * g.L * 4);
    w.pscore = tensor ? nullptr : (float*)take((size_t)np * sh.kp * 4);
    w.pid = tensor ? nullptr : (int64_t*)take((size_t)np * sh.kp * 8);
    w.pbuf = tensor ? nullptr : (uint64_t*)take((size_t)np * g.L * sh.R * 8);
    w.dense = tensor ? (uint16_t*)take((size_t)sh.bitmap_words * 32 * 2) : nullptr;
    w.cmax = tensor ? (float*)take((size_t)sh.bitmap_words * 4) : nullptr;
    w.slot_of = tensor ? (int32_t*)take((size_t)np * 4) : nullptr;
    w.sl_ids = tensor ? (int64_t*)take((size_t)nq * sh.so * 8) : nullptr;
    w.sl_scores = tensor ? (float*)take((size_t)nq * sh.so * 4) : nullptr;
    w.qscale = tensor ? (float*)take((size_t)nq * 4) : nullptr;
    w.qguard = tensor ? (float*)take((size_t)nq * 4) : nullptr;
    w.qbound = tensor ? (float*)take((size_t)nq * 4) : nullptr;
    w.qnorm = tensor ? (float*)take((size_t)nq * 4) : nullptr;
    w.hrecheck = tensor ? (int32_t*)take((size_t)nq * g.H * 4) : nullptr;
    w.redo = tensor ? (int32_t*)take((size_t)nq * 4) : nullptr;
    w.ovf = tensor ? (int32_t*)take((size_t)nq * 4) : nullptr;
    w.ovf_thr = tensor ? (float*)take((size_t)nq * 4) : nullptr;
    w.total = o;
    return w;
}

// Shape and cap checks; with `buffers`, also the pointers and the device.
// Caps of one pass of the search (nq queries searched with one workspace).
int check_pass_caps(const lider_index* ix, int64_t nq, int k, int c) {
    if (nq * c > (int64_t)INT32_MAX) return fail(LIDER_ELIMIT, "lider_search: nq * c exceeds 2^31-1");
    if (ix->params.score_mode != LIDER_SCORE_SIMT && nq * ix->g.H > (int64_t)INT32_MAX)
        return fail(LIDER_ELIMIT, "lider_search: nq * L * m exceeds 2^31-1; search fewer queries per call");
    // tensor paths: per pair, a bitmap word and 32 16-bit score codes per 32 positions
    if (ix->params.score_mode != LIDER_SCORE_SIMT && c <= ix->g.ncl &&
        nq * ix->top_words[c] > ((int64_t)1 << 30))
        return fail(LIDER_ELIMIT, "lider_search: the per-pair score rows of this batch exceed 64 GiB; search fewer "
                                  "queries per call");
    return LIDER_OK;
}

// Shape and cap checks; with `buffers`, also the pointers and the device.
// `pass_caps`: whether nq must also fit one pass (lider_search splits larger
// batches into passes itself).
int check_search_args(const lider_index* ix, const float* Q, int64_t nq, int k, int c, const void* ids,
                      const void* scores, bool buffers = true, bool pass_caps = true) {
    if (!ix) return fail(LIDER_EINVAL, "lider_search: index is NULL");
    if (nq < 0) return fail(LIDER_EINVAL, "lider_search: nq < 0");
    if (k < 1) return fail(LIDER_EINVAL, "lider_search: k must be >= 1");
    if (c < 1 || c > ix->g.ncl) return fail(LIDER_EINVAL, "lider_search: c must be in [1, n_clusters]");
    if (k > LIDER_MAX_K) return fail(LIDER_ELIMIT, "lider_search: k exceeds LIDER_MAX_K");
    if (c > LIDER_MAX_C) return fail(LIDER_ELIMIT, "lider_search: c exceeds LIDER_MAX_C");
    const int64_t R = (int64_t)ix->params.r0 * k;
    if (R * ix->g.L > LIDER_MAX_LR) return fail(LIDER_ELIMIT, "lider_search: L * r0 * k exceeds LIDER_MAX_LR");
    if ((ix->params.score_mode == LIDER_SCORE_BF16 || ix->params.score_mode == LIDER_SCORE_FP8) &&
        (int64_t)ix->params.rerank * k > 4096)
        return fail(LIDER_ELIMIT, "lider_search: rerank * k exceeds 4096");
    int rc;
    if (pass_caps && (rc = check_pass_caps(ix, nq, k, c))) return rc;
    if (!buffers) return LIDER_OK;
    if (nq > 0 && (!Q || !ids || !scores)) return fail(LIDER_EINVAL, "lider_search: NULL buffer");
    if (reinterpret_cast<uintptr_t>(Q) % 16 != 0)
        return fail(LIDER_EINVAL, "lider_search: queries must start on a 16-byte boundary");
    int dev = -1;
    LIDER_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != ix->device) return fail(LIDER_EINVAL, "lider_search: index lives on another device");
    return LIDER_OK;
}

// Queries per pass of lider_search: the tuning's probe_batch (0: the whole
// batch), halved until a pass meets the per-pass caps and its scratch stays
// within the index's pass budget (48 GiB, and 3/4 of the device memory left
// free after the build).  The scratch of a pass is sized for the worst case
// (every query probing the c largest clusters).
int64_t pass_size(const lider_index* ix, int64_t nq, int k, int c) {
    int64_t pb = ix->tune.probe_batch > 0 ? std::min<int64_t>(nq, ix->tune.probe_batch) : nq;
    while (pb > 1) {
        const bool fits = (pb * c <= (int64_t)INT32_MAX) &&
                          (ix->params.score_mode == LIDER_SCORE_SIMT ||
                           (pb * ix->g.H <= (int64_t)INT32_MAX && pb * ix->top_words[c] <= ((int64_t)1 << 30))) &&
                          carve(nullptr, ix->g, pb, c, search_shape(ix, k, pb, c)).total <= ix->pass_budget;
        if (fits) break;
        pb = (pb + 1) / 2;
    }
    return std::max<int64_t>(pb, 1);
}

// Queries that reach the device in chunks (lider_search_host): chunk i holds
// queries [bounds[i], bounds[i+1]) and is in device memory once event ready[i]
// has completed.  The per-query front of the search (hash, route) runs chunk by
// chunk as they arrive; the rest waits for the whole batch.
struct FrontFeed {
    int n;
    const int64_t* bounds;
    const cudaEvent_t* ready;
};

// Enqueue the search on `st` using workspace `w`.
int enqueue_search(const lider_index* ix, const float* Q, int64_t nq, int k, int c, int64_t* out_ids,
                   float* out_scores, const lider_trace* tr, const Workspace& w, cudaStream_t st,
                   const FrontFeed* feed = nullptr) {
    const Geometry& g = ix->g;
    const int R = ix->params.r0 * k;
    const int64_t np = nq * c;
    int rc;
    void* const* ev = tr ? tr->events : nullptr;
    auto mark = [&](int phase) -> int {
        if (ev && ev[phase]) LIDER_CUDA_TRY(cudaEventRecord((cudaEvent_t)ev[phase], st));
        return LIDER_OK;
    };
    LIDER_CUDA_TRY(cudaMemsetAsync(w.counters, 0, w.zero_bytes, st));

    // 1-2. hash and route, chunk by chunk: queries [q0, q1)
    const bool tensor_route = ix->params.score_mode != LIDER_SCORE_SIMT;
    // Tensor paths: steps that depend only on earlier ones run on the index's
    // second stream beside the main one (the hash recheck and the key packing
    // beside the top-c and the grouping; the queries' gather and the tile
    // descriptors beside the locate and the marking), joined by events.
    const bool fork = tensor_route && ix->side && ix->params.route_kind != LIDER_ROUTE_CORE;
    struct Events {
        cudaEvent_t e[4] = {};
        ~Events() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } fe_ev;
    if (fork)
        for (cudaEvent_t& x : fe_ev.e) LIDER_CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
    cudaStream_t side = fork ? ix->side : st;
    auto fork_to_side = [&](cudaEvent_t ev) -> int {      // the side stream continues after st's work so far
        LIDER_CUDA_TRY(cudaEventRecord(ev, st));
        LIDER_CUDA_TRY(cudaStreamWaitEvent(side, ev, 0));
        return LIDER_OK;
    };
    auto join_side = [&](cudaEvent_t ev) -> int {         // st continues after the side stream's work so far
        LIDER_CUDA_TRY(cudaEventRecord(ev, side));
        LIDER_CUDA_TRY(cudaStreamWaitEvent(st, ev, 0));
        return LIDER_OK;
    };
    // hash values too close to a bucket edge for the tiles' error, recomputed
    // exactly; then the packed keys of the whole batch (on the side stream
    // after the last front launch: with one chunk, beside the top-c)
    bool keys_launched = false;
    auto launch_keys = [&](bool forked) -> int {
        keys_launched = true;
        if (fork && !forked && (rc = fork_to_side(fe_ev.e[0]))) return rc;
        if (tensor_route) {
            hash_recheck_kernel<<<(unsigned)(16 * ix->num_sms), 32, (size_t)2 * g.d * sizeof(float), side>>>(
                Q, g.A, g.bproj, g.W, g.d, g.H, w.hrecheck, w.n_hrecheck, w.tq);
            LIDER_LAUNCH_CHECK("hash_recheck_kernel");
        }
        if ((rc = launch_pack(w.tq, nq, g.L, g.m, g.beta, g.hash_kind, 0, g.L, 1, w.qkeys,
                              &w.counters[CNT_QBOUNDARY], &w.counters[CNT_QCLAMPED], side)))
            return rc;
        if (tr && tr->qkeys)
            LIDER_CUDA_TRY(cudaMemcpyAsync(tr->qkeys, w.qkeys, (size_t)nq * g.L * 8, cudaMemcpyDeviceToDevice, side));
        return LIDER_OK;
    };
    // SIMT mode: Dot2 hash values, then exact FP64 routing scores and top-c
    auto simt_chunk = [&](int64_t q0, int64_t q1, bool last) -> int {
        const int64_t n = q1 - q0;
        const float* Qc = Q + q0 * g.d;
        int32_t* trace_route = tr && tr->route ? tr->route + q0 * c : nullptr;
        if ((rc = launch_hash_t(Qc, n, g.d, g.A, g.bproj, g.H, g.W, w.tq + q0 * g.H, st))) return rc;
        if (last && (rc = mark(LIDER_PHASE_ROUTE))) return rc;
        if ((rc = launch_scores(Qc, n, g.d, g.C, g.half_norm, g.ncl, w.rscore + q0 * g.ncl, st))) return rc;
        topc_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(w.rscore + q0 * g.ncl, n, g.ncl, c,
                                                                 w.route + q0 * c, trace_route);
        LIDER_LAUNCH_CHECK("topc_kernel");
        return LIDER_OK;
    };
    // tensor modes: one front_tc_kernel launch for the chunk's hash values and
    // routing scores, then the top-c of each query (with its guards)
    auto tensor_chunk = [&](int64_t q0, int64_t q1, bool last) -> int {
        const int64_t n = q1 - q0;
        const float* Qc = Q + q0 * g.d;
        int32_t* trace_route = tr && tr->route ? tr->route + q0 * c : nullptr;
        CUtensorMap mqs_h, mqs_l;      // the chunk's queries as TF32 head / tail
        if ((rc = launch_split_tf32(Qc, n * g.d, w.qs_hi + q0 * g.d, w.qs_lo + q0 * g.d, st))) return rc;
        if ((rc = make_tensor_map(&mqs_h, w.qs_hi + q0 * g.d, n, g.d, tc::kBM))) return rc;
        if ((rc = make_tensor_map(&mqs_l, w.qs_lo + q0 * g.d, n, g.d, tc::kBM))) return rc;
        qnorm_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(Qc, n, g.d, w.qnorm + q0);
        LIDER_LAUNCH_CHECK("qnorm_kernel");
        float* S = reinterpret_cast<float*>(w.rscore) + q0 * g.ncl;
        FrontSched fs{(int)n, ix->front_hp / tc::kBN, (int)cdiv(g.ncl, tc::kBN), ix->front_hp};
        FrontEpi fe;
        fe.t = w.tq + q0 * g.H;
        fe.b = g.bproj;
        fe.a_norm = ix->a_norm;
        fe.qnorm = w.qnorm + q0;
        fe.recheck = w.hrecheck;
        fe.n_recheck = w.n_hrecheck;
        fe.W = (float)g.W;
        fe.guard = kTcGuard;
        fe.H = g.H;
        fe.q0 = (int)q0;
        fe.hyper = g.hash_kind == LIDER_HASH_HYPERPLANE;
        fe.S = S;
        fe.half_norm = g.half_norm;
        fe.ncl = g.ncl;
        fe.nq = (int)n;
        fe.nth = fs.nth;
        fe.ntr = fs.ntr;
        if ((rc = smem_attr((const void*)front_tc_kernel, (int)(tc::kSmemBytes)))) return rc;
        const int kchunks = (g.d + tc::KindTf32x3::kBK - 1) / tc::KindTf32x3::kBK;
        auto launch_front = [&](const FrontSched& sch, const FrontEpi& epi, cudaStream_t s2) -> int {
            const int64_t tiles = cdiv(n, tc::kBM) * (sch.nth + sch.ntr);
            front_tc_kernel<<<(unsigned)std::min<int64_t>(tiles, ix->num_sms), tc::kThreads, tc::kSmemBytes, s2>>>(
                mqs_h, mqs_l, ix->map_fhi, ix->map_flo, kchunks, sch, epi, w.tc_err);
            LIDER_LAUNCH_CHECK("front_tc_kernel");
            return LIDER_OK;
        };
        if (fork && last && q0 == 0) {
            // one chunk: the routing tiles on this stream, the hash tiles (and
            // then the recheck and packing) on the side stream, so the top-c
            // starts after one round of tiles
            if ((rc = fork_to_side(fe_ev.e[0]))) return rc;
            FrontSched fr = fs, fh = fs;
            FrontEpi er = fe, eh = fe;
            fr.nth = er.nth = 0;
            fh.ntr = eh.ntr = 0;
            if ((rc = launch_front(fr, er, st))) return rc;
            if ((rc = launch_front(fh, eh, side))) return rc;
            if ((rc = mark(LIDER_PHASE_ROUTE))) return rc;
            if ((rc = launch_keys(true))) return rc;
        } else {
            if ((rc = launch_front(fs, fe, st))) return rc;
            if (last && (rc = mark(LIDER_PHASE_ROUTE))) return rc;
        }
        // guard: the tensor-core error of one score stays below kTcGuard |q| |mu|
        topc_exact_kernel<<<(unsigned)cdiv(n * 32, 256), 256, g.ncl <= kTopcStageCols ? 8 * g.ncl * 4 : 0, st>>>(
            S, Qc, g.C, g.half_norm, n, g.ncl, g.d, c, kTcGuard * ix->max_cnorm, w.route + q0 * c, trace_route,
            guard_mode(ix->params.score_mode), ix->max_xnorm, ix->x_scale, ix->xres_max, ix->xhat_max,
            w.qscale + q0, w.qguard + q0, w.qbound + q0, &w.counters[CNT_ROUTE_FALLBACK]);
        LIDER_LAUNCH_CHECK("topc_exact_kernel");
        return LIDER_OK;
    };
    if ((rc = mark(LIDER_PHASE_HASH))) return rc;
    const int nch = feed ? feed->n : 1;
    for (int i = 0; i < nch; ++i) {
        const int64_t q0 = feed ? feed->bounds[i] : 0, q1 = feed ? feed->bounds[i + 1] : nq;
        if (feed) LIDER_CUDA_TRY(cudaStreamWaitEvent(st, feed->ready[i], 0));
        const bool last = i == nch - 1;
        if (q1 > q0) {
            if ((rc = tensor_route ? tensor_chunk(q0, q1, last) : simt_chunk(q0, q1, last))) return rc;
        } else if (last && (rc = mark(LIDER_PHASE_ROUTE))) {
            return rc;
        }
    }
    if (!keys_launched && (rc = launch_keys(false))) return rc;
    if (ix->params.route_kind == LIDER_ROUTE_CORE) {
        // Layer-1 centroids retriever: replaces the route of the exact scan
        // (whose per-query error bounds the tensor paths still use)
        const RouteCoreShape rcs = route_core_shape(g, ix->params.r0, c);
        if ((rc = smem_attr((const void*)route_core_kernel, rcs.wpb * rcs.warp_bytes))) return rc;
        route_core_kernel<<<(unsigned)cdiv(nq, rcs.wpb), (unsigned)(32 * rcs.wpb), (size_t)rcs.wpb * rcs.warp_bytes,
                            st>>>(g, ix->ckeys, ix->cpos, ix->croot, ix->cleaf, w.qkeys, Q, nq, c, rcs.Rc, rcs.words,
                                  rcs.cap, rcs.warp_bytes,
                                  tensor_route ? reinterpret_cast<const float*>(w.rscore) : nullptr,
                                  kTcGuard * ix->max_cnorm, tensor_route ? nullptr : w.rscore, w.route,
                                  tr ? tr->route : nullptr);
        LIDER_LAUNCH_CHECK("route_core_kernel");
    }
    // 3. group
    if ((rc = mark(LIDER_PHASE_GROUP))) return rc;
    const int G = std::max(1, std::min(kMaxGroup, (96 * 1024) / (g.d * 4)));
    const bool one_block = g.ncl <= kGroupMaxCl && np <= kGroupMaxPairs;
    if (one_block) {
        group_kernel<<<1, kGroupThreads, 0, st>>>(w.route, np, c, g.ncl, G, g.cl_off, w.cnt, w.off, w.item_off,
                                                  w.unit_off, w.bm_off, w.pairs, w.qorder);
        LIDER_LAUNCH_CHECK("group_kernel");
    } else {
        group_count_kernel<<<(unsigned)cdiv(np, 256), 256, 0, st>>>(w.route, np, w.cnt);
        LIDER_LAUNCH_CHECK("group_count_kernel");
        group_scan_kernel<<<1, 1024, 0, st>>>(w.cnt, g.ncl, G, g.cl_off, w.off, w.cursor, w.item_off, w.unit_off,
                                              w.bm_off);
        LIDER_LAUNCH_CHECK("group_scan_kernel");
        group_fill_kernel<<<(unsigned)cdiv(np, 256), 256, 0, st>>>(w.route, np, w.cursor, w.pairs);
        LIDER_LAUNCH_CHECK("group_fill_kernel");
    }
    // the side stream: hash recheck and packing done, now the pairs exist
    if (fork && (rc = join_side(fe_ev.e[1]))) return rc;
    if (fork && (rc = fork_to_side(fe_ev.e[2]))) return rc;
    if (w.qorder && !one_block) {
        primary_order_kernel<<<(unsigned)g.ncl, 256, 0, st>>>(w.pairs, w.off, c, w.qorder, &w.counters[CNT_QORDER]);
        LIDER_LAUNCH_CHECK("primary_order_kernel");
    }
    // 4. locate + expand
    if ((rc = mark(LIDER_PHASE_LOCATE))) return rc;
    locate_kernel<<<(unsigned)cdiv(np * g.L, 256), 256, 0, st>>>(
        g, np, c, R, k, w.route, w.qkeys, w.wstart, w.wlen, tr ? tr->pstar : nullptr, tr ? tr->wstart : nullptr,
        tr ? tr->wlen : nullptr, w.counters);
    LIDER_LAUNCH_CHECK("locate_kernel");
    // 5. candidate union, exact scores and per-pair top-k
    const Shape sh = search_shape(ix, k);
    DenseArgs da{};                    // tensor paths: what the selects (and the band re-score) read
    if ((rc = mark(LIDER_PHASE_GATHER))) return rc;
    if (sh.mode != LIDER_SCORE_SIMT) {
        const bool h16 = sh.mode == LIDER_SCORE_BF16 || sh.mode == LIDER_SCORE_F16;
        CUtensorMap mqh, mql;
        if (sh.mode == LIDER_SCORE_FP8) {
            uint8_t* qp = reinterpret_cast<uint8_t*>(w.qp_hi);
            qgather_f8_kernel<<<(unsigned)cdiv(np * 32, 256), 256, 0, side>>>(Q, w.pairs, np, c, g.d, w.slot_scale, qp);
            LIDER_LAUNCH_CHECK("qgather_f8_kernel");
            if ((rc = make_tensor_map8(&mqh, qp, np, g.d, tc::kBM))) return rc;
            mql = mqh;
        } else if (h16) {
            uint16_t* qp = reinterpret_cast<uint16_t*>(w.qp_hi);
            if (sh.mode == LIDER_SCORE_BF16) {
                qgather_bf16_kernel<<<(unsigned)cdiv(np * 32, 256), 256, 0, side>>>(Q, w.pairs, np, c, g.d, qp);
                LIDER_LAUNCH_CHECK("qgather_bf16_kernel");
            } else {
                qgather_f16_kernel<<<(unsigned)cdiv(np * 32, 256), 256, 0, side>>>(Q, w.pairs, np, c, g.d, w.qscale,
                                                                                 qp);
                LIDER_LAUNCH_CHECK("qgather_f16_kernel");
            }
            if ((rc = make_tensor_map(&mqh, qp, np, g.d, tc::kBM, true))) return rc;
            mql = mqh;
        } else {
            qgather_kernel<<<(unsigned)cdiv(np * 32, 256), 256, 0, side>>>(Q, w.pairs, np, c, g.d, w.qp_hi, w.qp_lo);
            LIDER_LAUNCH_CHECK("qgather_kernel");
            if ((rc = make_tensor_map(&mqh, w.qp_hi, np, g.d, tc::kBM))) return rc;
            if ((rc = make_tensor_map(&mql, w.qp_lo, np, g.d, tc::kBM))) return rc;
        }
        // a warp per pair; bitmaps up to 48 KB per block of warps are built in shared memory
        const int mark_wpb = ix->tune.mark_threads / 32;
        const int max_words = g.max_row_tiles * (tc::kBN / 32);
        const int mark_words = std::min(max_words, (48 * 1024 / 4) / mark_wpb);
        mark_kernel<<<(unsigned)cdiv(np, mark_wpb), (unsigned)ix->tune.mark_threads,
                      (size_t)mark_wpb * mark_words * 4, st>>>(
            w.pairs, w.route, w.off, g.cl_off, w.bm_off, w.wstart, g.pos, g.n, g.L, R, w.bitmap, w.slot_of, w.pcount,
            mark_words, np);
        LIDER_LAUNCH_CHECK("mark_kernel");
        if ((rc = mark(LIDER_PHASE_SCORE))) return rc;
        tc_units_kernel<<<g.ncl, 128, 0, side>>>(w.unit_off, w.off, g.cl_off, w.bm_off, w.pairs, w.qbound, c,
                                                 g.ncl, ix->tune.tile_order, w.units, w.umeta, w.slot_bound);
        LIDER_LAUNCH_CHECK("tc_units_kernel");
        if (fork && (rc = join_side(fe_ev.e[3]))) return rc;
        TcArgs ta;
        ta.units = w.units;
        ta.umeta = w.umeta;
        ta.slot_bound = w.slot_bound;
        ta.unit_off = w.unit_off;
        ta.off = w.off;
        ta.cnt = w.cnt;
        ta.cl_off = g.cl_off;
        ta.pairs = w.pairs;
        ta.bm_off = w.bm_off;
        ta.ncl = g.ncl;
        ta.dense = w.dense;
        ta.qbound = w.qbound;
        ta.c = c;
        ta.bitmap = w.bitmap;
        ta.cmax = w.cmax;
        ta.slot_scale = sh.mode == LIDER_SCORE_FP8 ? w.slot_scale : nullptr;
        ta.col_scale = ix->x_rowscale;
        // A = queries of the tile (128 rows, box 128), B = cluster rows (256, box 256)
        auto launch_score = [&](auto kind, const CUtensorMap& mb0, const CUtensorMap& mb1) -> int {
            using Kind = decltype(kind);
            using Plan = ScorePlan<Kind>;
            if ((rc = smem_attr((const void*)tc_score_kernel<Kind>, Plan::kSmem))) return rc;
            tc_score_kernel<Kind><<<ix->num_sms, Plan::kThreads, Plan::kSmem, st>>>(
                mqh, mql, mb0, mb1, (g.d + Kind::kBK - 1) / Kind::kBK, ta, w.tc_err);
            LIDER_LAUNCH_CHECK("tc_score_kernel");
            return LIDER_OK;
        };
        if (sh.mode == LIDER_SCORE_FP8) rc = launch_score(tc::KindF8{}, ix->map_xf8, ix->map_xf8);
        else if (sh.mode == LIDER_SCORE_BF16) rc = launch_score(tc::KindBf16{}, ix->map_xh16, ix->map_xh16);
        else if (sh.mode == LIDER_SCORE_F16) rc = launch_score(tc::KindF16{}, ix->map_xh16, ix->map_xh16);
        else rc = launch_score(tc::KindTf32x3{}, ix->map_xhi, ix->map_xlo);
        if (rc) return rc;
        if ((rc = mark(LIDER_PHASE_SELECT))) return rc;
        // 3xTF32 and FP16 paths: a guard band makes the re-scored top k exact;
        // the served BF16 form keeps its approximate shortlist
        const int guarded = sh.mode != LIDER_SCORE_BF16 && sh.mode != LIDER_SCORE_FP8;
        da.dense = w.dense;
        da.qbound = w.qbound;
        da.cmax = w.cmax;
        da.bitmap = w.bitmap;
        da.bm_off = w.bm_off;
        da.off = w.off;
        da.slot_of = w.slot_of;
        da.route = w.route;
        da.cl_off = g.cl_off;
        da.orig_id = g.orig_id;
        da.ucount = w.pcount;
        da.ovf = guarded ? w.ovf : nullptr;
        da.ovf_thr = w.ovf_thr;
        da.ovf_count = w.ovf_count;
        select_hist_kernel<<<(unsigned)nq, (unsigned)ix->tune.select_threads, 0, st>>>(da, c, sh.ks, w.qguard, w.qbound, guarded, sh.so, w.sl_ids,
                                                         w.sl_scores, tr ? tr->ucount : nullptr, w.redo, w.redo_count,
                                                         w.counters);
        LIDER_LAUNCH_CHECK("select_hist_kernel");
        select_query_kernel<<<(unsigned)nq, 256, 0, st>>>(da, c, sh.ks, w.qguard, guarded, sh.so, w.sl_ids,
                                                          w.sl_scores, tr ? tr->ucount : nullptr, w.redo, w.redo_count,
                                                          w.counters);
        LIDER_LAUNCH_CHECK("select_query_kernel");
    } else {
        if ((rc = mark(LIDER_PHASE_SCORE))) return rc;
        ScoreArgs sa;
        sa.g = g;
        sa.Q = Q;
        sa.c = c;
        sa.G = G;
        sa.k = k;
        sa.T_cap = g.L * R;
        sa.region_bytes = (int)align_up(std::max((size_t)G * g.d * 4,
                                                 ((size_t)next_pow2(sa.T_cap) + kCandCap) * 8), 16);
        sa.off = w.off;
        sa.cnt = w.cnt;
        sa.item_off = w.item_off;
        sa.pairs = w.pairs;
        sa.wstart = w.wstart;
        sa.pbuf = w.pbuf;
        sa.pscore = w.pscore;
        sa.pid = w.pid;
        sa.trace_ucount = tr ? tr->ucount : nullptr;
        sa.counters = w.counters;
        const size_t smem = (size_t)sa.region_bytes + (size_t)(kTile / 2) * 4;
        const void* kern = nullptr;
        switch ((g.d % 128 == 0 && g.d <= 1024) ? g.d / 128 : 0) {
            case 1: kern = (const void*)score_group_kernel<1>; break;
            case 2: kern = (const void*)score_group_kernel<2>; break;
            case 3: kern = (const void*)score_group_kernel<3>; break;
            case 4: kern = (const void*)score_group_kernel<4>; break;
            case 5: kern = (const void*)score_group_kernel<5>; break;
            case 6: kern = (const void*)score_group_kernel<6>; break;
            case 7: kern = (const void*)score_group_kernel<7>; break;
            case 8: kern = (const void*)score_group_kernel<8>; break;
            default: kern = (const void*)score_group_kernel<0>; break;
        }
        if ((rc = smem_attr((const void*)kern, (int)smem))) return rc;
        int per_sm = 0;
        LIDER_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kScoreThreads, smem));
        if (per_sm < 1) return fail(LIDER_ELIMIT, "lider_search: score kernel does not fit on an SM");
        const int64_t max_items = cdiv(np, G) + g.ncl;
        const int grid = (int)std::min<int64_t>(max_items, (int64_t)per_sm * ix->num_sms);
        void* kargs[] = {&sa};
        LIDER_CUDA_TRY(cudaLaunchKernel(kern, dim3(grid), dim3(kScoreThreads), kargs, smem, st));
        if ((rc = mark(LIDER_PHASE_SELECT))) return rc;
    }
    // 6. merge (SIMT path), or the exact FP32 re-score of the selected lists (tensor paths)
    if ((rc = mark(LIDER_PHASE_MERGE))) return rc;
    if (sh.mode == LIDER_SCORE_SIMT) {
        merge_kernel<<<(unsigned)cdiv(nq * 32, 256), 256, 0, st>>>(w.pscore, w.pid, nq, c, sh.kp, sh.ks, out_ids,
                                                                   out_scores);
        LIDER_LAUNCH_CHECK("merge_kernel");
    } else {
        const size_t rs_smem = align_up((size_t)g.d * 4, 16) + (size_t)next_pow2(sh.so) * 8;
        const void* rs_kern = rescore_fn(g.d);
        if ((rc = smem_attr(rs_kern, (int)rs_smem))) return rc;
        {
            const float* rq = Q;
            const float* rx = g.X;
            const int32_t* rrow = g.row_of;
            int rd = (int)g.d, rS = (int)sh.so, rk = (int)k;
            const int64_t* rin = w.sl_ids;
            int64_t rn = g.n;
            unsigned long long* rb = &w.counters[CNT_BOUNDS];
            const int32_t* ro = w.qorder;
            void* rargs[] = {&rq, &rx, &rrow, &rd, &rS, &rin, &rk, &out_ids, &out_scores, &rn, &rb, &ro};
            LIDER_CUDA_TRY(cudaLaunchKernel(rs_kern, dim3((unsigned)nq), dim3((unsigned)ix->tune.rescore_threads),
                                            rargs, rs_smem, st));
        }
        if (da.ovf) {
            // the listed queries' whole bands, exactly (returns at once when none is listed)
            const size_t bd_smem = align_up((size_t)g.d * 4, 16) + (size_t)2 * kBandChunk * 8 + (size_t)kBandChunk * 4;
            if ((rc = smem_attr((const void*)rescore_band_kernel, (int)bd_smem))) return rc;
            rescore_band_kernel<<<(unsigned)std::min<int64_t>(nq, 2 * ix->num_sms), 256, bd_smem, st>>>(
                da, Q, g.X, g.d, c, k, out_ids, out_scores);
            LIDER_LAUNCH_CHECK("rescore_band_kernel");
        }
    }
    return mark(LIDER_NUM_PHASES);
}

int read_stats(const Workspace& w, int64_t nq, int c, lider_search_stats* stats, cudaStream_t st) {
    unsigned long long h[CNT_SLOTS] = {};
    int tc_err = 0;
    int32_t tiles = 0;
    LIDER_CUDA_TRY(cudaMemcpyAsync(h, w.counters, sizeof(h), cudaMemcpyDeviceToHost, st));
    LIDER_CUDA_TRY(cudaMemcpyAsync(&tc_err, w.tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    if (w.qp_hi)
        LIDER_CUDA_TRY(cudaMemcpyAsync(&tiles, w.unit_off + w.ncl, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    LIDER_CUDA_TRY(cudaStreamSynchronize(st));
    if (tc_err)
        return fail(LIDER_ECUDA, "lider_search: tensor-core scoring stopped after a wait timed out (code " +
                                     std::to_string(tc_err) + ")");
    if (h[CNT_BOUNDS])
        return fail(LIDER_ECUDA, "lider_search: " + std::to_string(h[CNT_BOUNDS]) +
                                     " accesses failed a bounds check and were skipped");
    stats->n_queries = nq;
    stats->pairs = nq * c;
    stats->candidates = (int64_t)h[CNT_CANDIDATES];
    stats->qkey_boundary = (int64_t)h[CNT_QBOUNDARY];
    stats->qkey_clamped = (int64_t)h[CNT_QCLAMPED];
    stats->locate_fallback = (int64_t)h[CNT_FALLBACK];
    stats->empty_pairs = (int64_t)h[CNT_EMPTY];
    stats->tc_tiles = tiles;
    stats->route_fallback = (int64_t)h[CNT_ROUTE_FALLBACK];
    stats->select_overflow = (int64_t)h[CNT_SEL_OVERFLOW];
    stats->rmi_oor = (int64_t)h[CNT_OOR];
    stats->rmi_le = (int64_t)h[CNT_LE];
    stats->rmi_oor_le = (int64_t)h[CNT_OOR_LE];
    stats->passes = 1;
    return LIDER_OK;
}

// Counters of one more pass added to a search's.
void add_stats(lider_search_stats* acc, const lider_search_stats& ps) {
    acc->n_queries += ps.n_queries;
    acc->pairs += ps.pairs;
    acc->candidates += ps.candidates;
    acc->qkey_boundary += ps.qkey_boundary;
    acc->qkey_clamped += ps.qkey_clamped;
    acc->locate_fallback += ps.locate_fallback;
    acc->empty_pairs += ps.empty_pairs;
    acc->tc_tiles += ps.tc_tiles;
    acc->route_fallback += ps.route_fallback;
    acc->select_overflow += ps.select_overflow;
    acc->rmi_oor += ps.rmi_oor;
    acc->rmi_le += ps.rmi_le;
    acc->rmi_oor_le += ps.rmi_oor_le;
    acc->passes += ps.passes;
}

int pool_alloc(const lider_index* ix, void** p, size_t bytes, cudaStream_t st) {
    // under stream capture the scratch becomes a graph allocation node
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cap == cudaStreamCaptureStatusActive ? cudaMallocAsync(p, bytes ? bytes : 256, st)
                                                        : cudaMallocFromPoolAsync(p, bytes ? bytes : 256, ix->pool, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LIDER_ENOMEM, std::string("lider_search: scratch allocation of ") + std::to_string(bytes) +
                                      " bytes failed: " + cudaGetErrorString(e));
    }
    return LIDER_OK;
}

}  // namespace

// lider_search: the batch in passes of pass_size queries, one after the other
// on the stream, sharing one workspace (allocated once per call from the
// index's pool, or as a graph allocation under capture).  With several
// passes, trace arrays are filled pass by pass; phase events time the first
// pass's start (events[0]) to the last pass's end, the boundaries between
// them those of the last pass.
int search_entry(const lider_index* ix, const float* Q, int64_t nq, int k, int c, int64_t* out_ids,
                 float* out_scores, const lider_trace* tr, lider_search_stats* stats, void* stream) {
    int rc = check_search_args(ix, Q, nq, k, c, out_ids, out_scores, true, false);
    if (rc) return rc;
    if (stats) *stats = lider_search_stats{};
    if (nq == 0) return LIDER_OK;
    const int64_t pb = pass_size(ix, nq, k, c);
    if ((rc = check_pass_caps(ix, pb, k, c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Workspace sz = carve(nullptr, ix->g, pb, c, search_shape(ix, k, pb, c));
    void* mem = nullptr;
    if ((rc = pool_alloc(ix, &mem, sz.total, st))) return rc;
    const int d = ix->g.d, L = ix->g.L;
    for (int64_t q0 = 0; q0 < nq && rc == LIDER_OK; q0 += pb) {
        const int64_t n = std::min(pb, nq - q0);
        Workspace w = carve((unsigned char*)mem, ix->g, n, c, search_shape(ix, k, n, c));
        lider_trace t{};
        const lider_trace* tp = nullptr;
        if (tr) {
            auto at = [&](auto* p, int64_t per) { return p ? p + q0 * per : p; };
            t.route = at(tr->route, c);
            t.qkeys = at(tr->qkeys, L);
            t.pstar = at(tr->pstar, (int64_t)c * L);
            t.wstart = at(tr->wstart, (int64_t)c * L);
            t.wlen = at(tr->wlen, (int64_t)c * L);
            t.ucount = at(tr->ucount, c);
            // phase events: all of them on the last pass, and the first pass's start
            const bool last = q0 + n >= nq;
            void* const* ev = tr->events;
            static thread_local void* ev_first[LIDER_NUM_PHASES + 1];
            if (ev && !last) {
                for (int i = 0; i <= LIDER_NUM_PHASES; ++i) ev_first[i] = (q0 == 0 && i == 0) ? ev[0] : nullptr;
                t.events = ev_first;
            } else if (ev && q0 > 0) {
                static thread_local void* ev_last[LIDER_NUM_PHASES + 1];
                for (int i = 0; i <= LIDER_NUM_PHASES; ++i) ev_last[i] = ev[i];
                ev_last[0] = nullptr;                         // recorded at the first pass
                t.events = ev_last;
            } else {
                t.events = ev;
            }
            tp = &t;
        }
        rc = enqueue_search(ix, Q + q0 * d, n, k, c, out_ids + q0 * k, out_scores + q0 * k, tp, w, st);
        if (rc == LIDER_OK && stats) {
            lider_search_stats ps{};
            if ((rc = read_stats(w, n, c, &ps, st)) == LIDER_OK) add_stats(stats, ps);
        }
    }
    cudaError_t e = cudaFreeAsync(mem, st);
    if (rc == LIDER_OK && e != cudaSuccess) return cuda_fail(e, "cudaFreeAsync");
    return rc;
}

int search_scratch_entry(const lider_index* ix, int64_t nq, int k, int c, size_t* bytes) {
    if (!bytes) return fail(LIDER_EINVAL, "lider_search_scratch_bytes: bytes is NULL");
    *bytes = 0;
    int rc = check_search_args(ix, nullptr, nq, k, c, nullptr, nullptr, false, false);
    if (rc) return rc;
    if (nq == 0) return LIDER_OK;
    const int64_t pb = pass_size(ix, nq, k, c);
    if ((rc = check_pass_caps(ix, pb, k, c))) return rc;
    *bytes = carve(nullptr, ix->g, pb, c, search_shape(ix, k, pb, c)).total;
    return LIDER_OK;
}

bool tuning_valid(const lider_tuning& t) {
    auto in = [](int v, std::initializer_list<int> set) {
        for (int x : set)
            if (v == x) return true;
        return false;
    };
    return in(t.select_threads, {64, 128, 256, 512}) && in(t.rescore_threads, {64, 128, 256, 512}) &&
           in(t.mark_threads, {32, 64, 128, 256}) && in(t.tile_order, {0, 1}) && t.probe_batch >= 0;
}

// Coordinate descent over the launch shapes, timing whole searches.
int autotune_entry(lider_index* ix, const float* Q, int64_t nq, int k, int c, int reps, lider_tuning* chosen,
                   double* best_ms, void* stream) {
    if (!ix) return fail(LIDER_EINVAL, "lider_autotune: index is NULL");
    if (reps < 1) return fail(LIDER_EINVAL, "lider_autotune: reps must be >= 1");
    if (nq < 1) return fail(LIDER_EINVAL, "lider_autotune: nq must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t* ids = nullptr;
    float* sc = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = LIDER_OK;
    const lider_tuning start = ix->tune;
    auto cleanup = [&] {
        if (ids) cudaFree(ids);
        if (sc) cudaFree(sc);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&ids, (size_t)nq * k * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc(&sc, (size_t)nq * k * sizeof(float));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "lider_autotune: setup");
    }
    auto time_it = [&](const lider_tuning& t, double* ms) -> int {
        ix->tune = t;
        int r = search_entry(ix, Q, nq, k, c, ids, sc, nullptr, nullptr, st);
        if (r) return r;
        std::vector<float> v(reps);
        for (int i = 0; i < reps; ++i) {
            LIDER_CUDA_TRY(cudaEventRecord(e0, st));
            if ((r = search_entry(ix, Q, nq, k, c, ids, sc, nullptr, nullptr, st))) return r;
            LIDER_CUDA_TRY(cudaEventRecord(e1, st));
            LIDER_CUDA_TRY(cudaEventSynchronize(e1));
            LIDER_CUDA_TRY(cudaEventElapsedTime(&v[i], e0, e1));
        }
        std::sort(v.begin(), v.end());
        *ms = v[reps / 2];
        return LIDER_OK;
    };
    lider_tuning best = start;
    double best_t = 0;
    if ((rc = time_it(best, &best_t))) {
        ix->tune = start;
        cleanup();
        return rc;
    }
    // probe batches: the whole batch (0: as large as a pass allows) and
    // passes of a half, a quarter and an eighth of what fits
    const int64_t pb0 = pass_size(ix, nq, k, c);
    const int pb_v[] = {0, (int)std::max<int64_t>(1, (pb0 + 1) / 2), (int)std::max<int64_t>(1, (pb0 + 3) / 4),
                        (int)std::max<int64_t>(1, (pb0 + 7) / 8)};
    static const int sel_v[] = {64, 128, 256, 512}, res_v[] = {64, 128, 256, 512}, mark_v[] = {32, 64, 128, 256},
                     ord_v[] = {0, 1};
    for (int round = 0; round < 2 && rc == LIDER_OK; ++round) {
        for (int f = 0; f < 5 && rc == LIDER_OK; ++f) {
            const int* vals = f == 0 ? sel_v : f == 1 ? res_v : f == 2 ? mark_v : f == 3 ? ord_v : pb_v;
            const int nv = f == 3 ? 2 : 4;
            for (int i = 0; i < nv && rc == LIDER_OK; ++i) {
                lider_tuning cand = best;
                int* field = f == 0 ? &cand.select_threads : f == 1 ? &cand.rescore_threads
                           : f == 2 ? &cand.mark_threads : f == 3 ? &cand.tile_order : &cand.probe_batch;
                if (*field == vals[i]) continue;
                *field = vals[i];
                double t = 0;
                rc = time_it(cand, &t);
                if (rc == LIDER_OK && t < best_t) {
                    best = cand;
                    best_t = t;
                }
            }
        }
    }
    ix->tune = rc == LIDER_OK ? best : start;
    cleanup();
    if (rc) return rc;
    if (chosen) *chosen = best;
    if (best_ms) *best_ms = best_t;
    return LIDER_OK;
}

// The address a kernel can use for host memory that is pinned and mapped into
// the device's address space (cudaHostAlloc, torch's pinned memory), or null.
void* device_view(const void* host) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// End to end on host buffers, in the passes lider_search would make.  The
// queries go to the device on a second stream, each pass's in up to
// kHostChunks copies, and the hash and route of each chunk start as soon as
// it has landed, so the copies overlap the per-query front of the search (and
// a later pass's copies the earlier passes).  When the result buffers are
// pinned and mapped, each pass's final re-score writes its ids and scores into
// them directly (no copy back); otherwise each pass's results are copied back
// after it.
constexpr int kHostChunks = 4;

int search_host_entry(const lider_index* ix, const float* Qh, int64_t nq, int k, int c, int64_t* ids_h,
                      float* scores_h, lider_search_stats* stats, void* stream) {
    int rc = check_search_args(ix, Qh, nq, k, c, ids_h, scores_h, true, false);
    if (rc) return rc;
    if (stats) *stats = lider_search_stats{};
    if (nq == 0) return LIDER_OK;
    const int64_t pb = pass_size(ix, nq, k, c);
    if ((rc = check_pass_caps(ix, pb, k, c))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int d = ix->g.d;
    int64_t* ids_view = static_cast<int64_t*>(device_view(ids_h));
    float* scores_view = static_cast<float*>(device_view(scores_h));
    const bool direct = ids_view && scores_view;
    const size_t qb = (size_t)nq * d * 4, ib = direct ? 0 : (size_t)nq * k * 8, sb = direct ? 0 : (size_t)nq * k * 4;
    const size_t o_ids = align_up(qb, 256), o_sc = align_up(o_ids + ib, 256);
    Workspace sz = carve(nullptr, ix->g, pb, c, search_shape(ix, k, pb, c));
    const size_t o_ws = align_up(o_sc + sb, 256);
    void* mem = nullptr;
    if ((rc = pool_alloc(ix, &mem, o_ws + sz.total, st))) return rc;
    unsigned char* m = (unsigned char*)mem;
    float* Qd = (float*)m;
    int64_t* idd = direct ? ids_view : (int64_t*)(m + o_ids);
    float* scd = direct ? scores_view : (float*)(m + o_sc);

    // chunk bounds, pass by pass: pass p owns chunks [first[p], first[p+1])
    const int64_t npass = (nq + pb - 1) / pb;
    std::vector<int64_t> bounds;              // absolute query offsets
    std::vector<int> first;
    for (int64_t q0 = 0; q0 < nq; q0 += pb) {
        const int64_t n = std::min(pb, nq - q0);
        const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, n / 2048));
        first.push_back((int)bounds.size());
        for (int i = 0; i < nch; ++i) bounds.push_back(q0 + n * i / nch);
    }
    first.push_back((int)bounds.size());
    bounds.push_back(nq);
    const int nchunks = (int)bounds.size() - 1;
    cudaStream_t cs = nullptr;
    std::vector<cudaEvent_t> evs(nchunks + 1, nullptr);
    auto cleanup = [&]() {
        for (cudaEvent_t e : evs)
            if (e) cudaEventDestroy(e);
        if (cs) cudaStreamDestroy(cs);
    };
    // copy-in on a stream of its own, ordered after the caller's stream
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int i = 0; e == cudaSuccess && i <= nchunks; ++i) e = cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(evs[nchunks], st);        // the caller's earlier work comes first
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, evs[nchunks], 0);
    for (int i = 0; e == cudaSuccess && i < nchunks; ++i) {
        const size_t off = (size_t)bounds[i] * d, len = (size_t)(bounds[i + 1] - bounds[i]) * d;
        e = cudaMemcpyAsync(Qd + off, Qh + off, len * 4, cudaMemcpyHostToDevice, cs);
        if (e == cudaSuccess) e = cudaEventRecord(evs[i], cs);
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "lider_search_host: copying the queries in");
    for (int64_t p = 0; p < npass && !rc; ++p) {
        const int64_t q0 = p * pb, n = std::min(pb, nq - q0);
        int64_t rel[kHostChunks + 1];
        const int nch = first[p + 1] - first[p];
        for (int i = 0; i <= nch; ++i) rel[i] = bounds[first[p] + i] - q0;
        const FrontFeed feed{nch, rel, evs.data() + first[p]};
        Workspace w = carve(m + o_ws, ix->g, n, c, search_shape(ix, k, n, c));
        rc = enqueue_search(ix, Qd + q0 * d, n, k, c, idd + q0 * k, scd + q0 * k, nullptr, w, st, &feed);
        if (!rc && !direct &&
            (e = cudaMemcpyAsync(ids_h + q0 * k, idd + q0 * k, (size_t)n * k * 8, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
            rc = cuda_fail(e, "cudaMemcpyAsync(ids)");
        if (!rc && !direct &&
            (e = cudaMemcpyAsync(scores_h + q0 * k, scd + q0 * k, (size_t)n * k * 4, cudaMemcpyDeviceToHost, st)) !=
                cudaSuccess)
            rc = cuda_fail(e, "cudaMemcpyAsync(scores)");
        if (!rc && stats) {
            lider_search_stats ps{};
            if (!(rc = read_stats(w, n, c, &ps, st))) add_stats(stats, ps);
        }
    }
    // a complete search waited for every chunk's event on st; after a failure
    // the copies may still run, so they finish before the memory is released
    if (rc && cs) cudaStreamSynchronize(cs);
    e = cudaFreeAsync(mem, st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && !rc) rc = cuda_fail(e, "cudaStreamSynchronize");
    cleanup();
    return rc;
}

}  // namespace lider

// ---------------------------------------------------------------------------
// Search without any device allocation.
//
// Some callers cannot allocate device memory when they search: a service that
// reserves all of its GPU memory up front and must not grow its footprint
// afterwards, code that runs while another framework owns the CUDA allocator,
// or a latency-critical thread where cudaMalloc (or a pool that may need to
// grow) could block or fail under memory pressure.  lider_search_noalloc runs
// the same kernels as lider_search, but its scratch lives in the fixed device
// array below instead of coming from the index's pool.
//
// The array is LIDER_NOALLOC_SCRATCH_BYTES long.  Every GPU on which this
// library's device code is loaded holds it until the process exits.  In host
// code `lider_noalloc_scratch` only names a host-side stand-in, so its device
// address is looked up once per device (cudaGetSymbolAddress, with that device
// current) on the first call there; make that first call before any stream
// capture.  All calls share the array: calls whose work overlaps on the GPU
// (other streams, or other host threads) race on it and must be serialised by
// the caller.  The array keeps the last call's contents; every search clears
// its counters before use and writes every other scratch word before reading.
static __device__ __align__(256) unsigned char lider_noalloc_scratch[LIDER_NOALLOC_SCRATCH_BYTES];

namespace lider {
namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_base[kMaxDevices] = {};
void* g_noalloc_ctx[kMaxDevices] = {};         // the context the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);

// The current CUDA context (null when the driver entry point is missing).
void* current_context() {
    static CtxGetCurrentFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            p = nullptr;
        cudaGetLastError();
        return (CtxGetCurrentFn)p;
    }();
    CUcontext ctx = nullptr;
    if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    return ctx;
}

// Device address of the static scratch on the current device `dev`, looked up
// once per (device, context): after a device reset the module is loaded again
// in a new context and the array can sit at another address.
int noalloc_scratch(int dev, unsigned char** out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(LIDER_ELIMIT, "lider_search_noalloc: device ordinal too large");
    void* ctx = current_context();
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_base[dev] || g_noalloc_ctx[dev] != ctx) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, lider_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(lider_noalloc_scratch)");
        if (!p) return fail(LIDER_ECUDA, "lider_search_noalloc: scratch symbol has no device address");
        g_noalloc_base[dev] = static_cast<unsigned char*>(p);
        g_noalloc_ctx[dev] = ctx;
    }
    *out = g_noalloc_base[dev];
    return LIDER_OK;
}

int search_noalloc_impl(const lider_index* ix, const float* Q, int64_t nq, int k, int c, int64_t* out_ids,
                        float* out_scores, lider_search_stats* stats, void* stream) {
    int rc = check_search_args(ix, Q, nq, k, c, out_ids, out_scores);
    if (rc) return rc;
    if (stats) *stats = lider_search_stats{};
    if (nq == 0) return LIDER_OK;
    const Workspace need = carve(nullptr, ix->g, nq, c, search_shape(ix, k, nq, c));
    if (need.total > (size_t)LIDER_NOALLOC_SCRATCH_BYTES)
        return fail(LIDER_ELIMIT, "lider_search_noalloc: this batch needs " + std::to_string(need.total) +
                                      " bytes of scratch, more than the fixed LIDER_NOALLOC_SCRATCH_BYTES (" +
                                      std::to_string((size_t)LIDER_NOALLOC_SCRATCH_BYTES) +
                                      "); search fewer queries per call");
    unsigned char* base = nullptr;
    if ((rc = noalloc_scratch(ix->device, &base))) return rc;
    const Workspace w = carve(base, ix->g, nq, c, search_shape(ix, k, nq, c));
    cudaStream_t st = (cudaStream_t)stream;
    rc = enqueue_search(ix, Q, nq, k, c, out_ids, out_scores, nullptr, w, st);
    if (rc == LIDER_OK && stats) rc = read_stats(w, nq, c, stats, st);
    return rc;
}

}  // namespace
}  // namespace lider

extern "C" int lider_search_noalloc(const lider_index* index, const float* queries, int64_t nq, int32_t k,
                                    int32_t c, int64_t* out_ids, float* out_scores, lider_search_stats* stats,
                                    void* stream) {
    try {
        return lider::search_noalloc_impl(index, queries, nq, k, c, out_ids, out_scores, stats, stream);
    } catch (...) {
        return lider::fail(LIDER_ECUDA, "lider_search_noalloc: internal error");
    }
}
