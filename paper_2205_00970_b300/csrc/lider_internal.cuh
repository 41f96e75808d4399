// Internal definitions shared by the LIDER CUDA translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lider.h"

namespace lider {

// ---------------------------------------------------------------- errors ----
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define LIDER_CUDA_TRY(expr)                                   \
    do {                                                       \
        cudaError_t _e = (expr);                               \
        if (_e != cudaSuccess) return ::lider::cuda_fail(_e, #expr); \
    } while (0)

#define LIDER_LAUNCH_CHECK(name)                               \
    do {                                                       \
        cudaError_t _e = cudaGetLastError();                   \
        if (_e != cudaSuccess) return ::lider::cuda_fail(_e, name); \
    } while (0)

// ----------------------------------------------------------------- index ----
struct RmiLeaf {          // one second-stage linear model and its error window
    double a;             // intercept
    double b;             // slope
    int32_t lo;           // min(first position of key - prediction)
    int32_t hi;           // max(...)
};
static_assert(sizeof(RmiLeaf) == 24, "RmiLeaf layout");

struct RmiRoot {          // first stage and re-scaling range of one (cluster, array)
    double a0, b0;
    uint64_t x_min, x_max;
};

constexpr int kRouteCoreMaxClusters = 8192;    // LIDER_ROUTE_CORE cap on n_clusters (shared memory of one warp)

struct Geometry {         // everything a search kernel needs, passed by value
    int64_t n;
    int32_t d, ncl, L, m, F, beta, B, H;
    int32_t max_row_tiles;  // ceil(largest cluster / 256)
    int32_t hash_kind;      // LIDER_HASH_PSTABLE or LIDER_HASH_HYPERPLANE
    int32_t raw_keys;       // 1: the RMIs take raw key values (no re-scaling)
    double W;
    const float* X;         // n x d, rows grouped by cluster
    const int64_t* orig_id; // n
    const int64_t* cl_off;  // ncl + 1
    const float* C;         // ncl x d
    const double* half_norm;// ncl
    const float* A;         // H x d
    const float* bproj;     // H
    const uint64_t* keys;   // L x n
    const int32_t* pos;     // L x n, cluster-local row of each sorted entry
    const RmiRoot* root;    // ncl x L
    const RmiLeaf* leaf;    // ncl x L x F
    const float* X_hi;      // n x d, TF32 head of X (tensor-core scoring)
    const float* X_lo;      // n x d, X - X_hi
    const int32_t* row_of;  // n, row of X holding corpus id i (inverse of orig_id)
    const uint16_t* X_h16;  // n x d, 16-bit copy of X: BF16 (served form) or scaled FP16
};

}  // namespace lider

struct lider_index {
    lider::Geometry g;
    lider_params params;
    int device = 0;
    std::vector<int64_t> h_cl_off;
    std::vector<int64_t> top_words;  // [c] = bitmap words of the c largest clusters
    // owned device buffers
    float* X = nullptr;
    int64_t* orig_id = nullptr;
    int64_t* cl_off = nullptr;
    float* C = nullptr;
    double* half_norm = nullptr;
    float* A = nullptr;
    float* bproj = nullptr;
    uint64_t* keys = nullptr;
    int32_t* pos = nullptr;
    lider::RmiRoot* root = nullptr;
    lider::RmiLeaf* leaf = nullptr;
    float* X_hi = nullptr;
    float* X_lo = nullptr;
    int32_t* row_of = nullptr;
    uint16_t* X_h16 = nullptr;  // BF16 copy (served form) or FP16 copy of x_scale * X
    // front operand of the tensor modes, TF32 head / tail: projections in rows
    // [0, H), zero rows up to front_hp (H rounded up to 256), centroids in rows
    // [front_hp, front_hp + n_clusters)
    float* F_hi = nullptr;
    float* F_lo = nullptr;
    int front_hp = 0;
    CUtensorMap map_fhi;        // TMA maps over F_hi / F_lo, boxes of 32 x 256
    CUtensorMap map_flo;
    float* a_norm = nullptr;    // |a_h| per projection (rounded up)
    float max_cnorm = 0.f;      // largest centroid norm (routing error guard)
    float max_xnorm = 0.f;      // largest corpus row norm (candidate error guard)
    float x_scale = 1.f;        // FP16 mode: power of two applied to X before rounding
    float xres_max = 0.f;       // FP16 mode: max over rows of |fp16(x_scale x) - x_scale x| (rounded up)
    float xhat_max = 0.f;       // FP16 mode: max over rows of |fp16(x_scale x)| (rounded up)
    CUtensorMap map_xh16;       // TMA map over X_h16, boxes of 64 x 256
    uint8_t* X_f8 = nullptr;    // FP8 e4m3 copy of X, one scale per row (served FP8 form)
    float* x_rowscale = nullptr;
    CUtensorMap map_xf8;        // TMA map over X_f8, boxes of 128 x 256
    CUtensorMap map_xhi;        // TMA maps over X_hi / X_lo, boxes of 32 x 256
    CUtensorMap map_xlo;
    // Layer-1 centroids retriever (LIDER_ROUTE_CORE): one core model over the
    // centroids, laid out like one cluster of ncl entries
    uint64_t* ckeys = nullptr;          // L x ncl sorted keys of the centroids
    int32_t* cpos = nullptr;            // L x ncl centroid index of each entry
    lider::RmiRoot* croot = nullptr;    // L
    lider::RmiLeaf* cleaf = nullptr;    // L x F
    cudaMemPool_t pool = nullptr;
    cudaStream_t side = nullptr;        // second stream for the search's independent steps
    // how the index was built (lider_build_info)
    lider_cluster_params cluster{};     // k-means parameters (clustered only)
    bool clustered = false;             // k-means ran inside the build
    bool projections_drawn = false;     // A and b were drawn from the seed
    double kmeans_ms = 0.0;             // host wall time of the k-means iterations
    double build_ms = 0.0;              // host wall time of the whole build
    size_t pass_budget = 0;             // search scratch one pass may take (set at the end of the build)
    lider_tuning tune{128, 128, 64, 1, 0};    // launch shapes (lider_autotune; defaults measured on mid)
    int score_blocks_per_sm = 1;
    int num_sms = 148;
};

namespace lider {

// ------------------------------------------------------ Dot2 arithmetic ----
// Compensated dot product (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Algorithm Dot2): TwoProduct via FMA and
// TwoSum, accumulated in FP32; s + c carries about twice the working
// precision.  All operations use explicit round-to-nearest intrinsics so that
// the compiler cannot contract or reassociate them.
struct Dot2 {
    float s, c;
};

__device__ __forceinline__ void dot2_step(Dot2& acc, float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);              // exact: a*b = p + e
    float t = __fadd_rn(acc.s, p);
    float z = __fadd_rn(t, -acc.s);
    float err = __fadd_rn(__fadd_rn(acc.s, -__fadd_rn(t, -z)), __fadd_rn(p, -z));  // exact: s+p = t+err
    acc.s = t;
    acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

__device__ __forceinline__ double dot2_value(const Dot2& acc) {
    return __dadd_rn((double)acc.s, (double)acc.c);
}

// ----------------------------------------------- hashkey distance dist_e ----
// Packed key: element j (j = 0 most significant, i.e. h_1) in bits
// [beta*(m-1-j), beta*(m-j)).  Returns (KL << 57) | KD_e so that one unsigned
// comparison orders pairs exactly like dist_e = KL + KD_e / 2^(beta*B)
// (Sec. 4.2).  Requires beta*B <= 56.
__device__ __forceinline__ uint64_t dist_code(uint64_t a, uint64_t q, int m, int beta, int B) {
    uint64_t x = a ^ q;
    if (x == 0) return 0;
    int nb = m * beta;
    int lz = __clzll(x) - (64 - nb);
    int lcp = lz / beta;
    int rem = m - lcp;                           // elements after the prefix (>= 1)
    int wb = beta * B;
    uint64_t mask = (wb >= 64) ? ~0ull : ((1ull << wb) - 1);
    uint64_t da, dq;
    if (B <= rem) {
        int sh = beta * (rem - B);
        da = (a >> sh) & mask;
        dq = (q >> sh) & mask;
    } else {
        int rb = beta * rem;
        uint64_t rmask = (rb >= 64) ? ~0ull : ((1ull << rb) - 1);
        int sh = beta * (B - rem);
        da = (a & rmask) << sh;
        dq = (q & rmask) << sh;
    }
    uint64_t kd = da > dq ? da - dq : dq - da;
    return ((uint64_t)(m - lcp) << 57) | kd;
}

// Order-preserving map of an FP32 score to uint32 (ascending).
__device__ __forceinline__ uint32_t float_order(float f) {
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_from_order(uint32_t u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ------------------------------------------------------------ re-scaling ----
// r = (x - x_min) / (x_max - x_min) * (n_c - 1), Sec. 5.1; the difference is an
// exact integer, converted to FP64 with round-to-nearest; a key below x_min
// gives r < 0 (query keys only).  raw: no re-scaling, r = x rounded to FP64
// (the ablation of Sec. 7.4).
__device__ __forceinline__ double rescale_key(uint64_t x, uint64_t x_min, uint64_t x_max, int64_t n_c,
                                              bool raw = false) {
    if (raw) return __ull2double_rn(x);
    if (x_max == x_min) return 0.0;
    double num = (x >= x_min) ? __ull2double_rn(x - x_min) : -__ull2double_rn(x_min - x);
    double den = __ull2double_rn(x_max - x_min);
    return __dmul_rn(__ddiv_rn(num, den), (double)(n_c - 1));
}

// Leaf of the second RMI stage: clamp(floor((a0 + b0 r) * F / n_c), 0, F-1).
__device__ __forceinline__ int rmi_leaf(double a0, double b0, double r, int F, int64_t n_c) {
    double g = __ddiv_rn(__dmul_rn(__dadd_rn(a0, __dmul_rn(b0, r)), (double)F), (double)n_c);
    g = floor(g);
    if (!(g > 0.0)) return 0;                   // also catches NaN
    if (g >= (double)(F - 1)) return F - 1;
    return (int)g;
}

// Clamped floor prediction of a linear model: clamp(floor(a + b r), 0, n_c - 1).
__device__ __forceinline__ int64_t rmi_predict(double a, double b, double r, int64_t n_c) {
    double p = floor(__dadd_rn(a, __dmul_rn(b, r)));
    if (!(p > 0.0)) return 0;
    if (p >= (double)(n_c - 1)) return n_c - 1;
    return (int64_t)p;
}

// ---------------------------------------------------- locate and expand ----
// One sorted array K[0..n_c) of a core model and a query key x: the RMI
// prediction ph (Sec. 5.2), the exact lower bound p searched inside the
// leaf's error window, with a fallback to the whole array when the window
// misses it (counted in fb), and the expansion window [s, s + T),
// T = min(R, n_c): the first T picks of the greedy merge of the left run
// (p-1, p-2, ...) and the right run (p, p+1, ...) by dist_e, ties to the left
// (Sec. 4.2, Sec. 4.3).  Both runs are non-decreasing in dist_e (Lemmas 2
// and 3), so the picks form one window [p - t, p - t + T) whose t is found by
// a co-rank search: the largest count such that left item t-1 precedes right
// item T-t.  n_c >= 1.
struct Located {
    int64_t ph, p, s, T;
};

__device__ __forceinline__ Located locate_window(const uint64_t* __restrict__ K, int64_t n_c, const RmiRoot& rt,
                                                 const RmiLeaf* __restrict__ leaves, int F, uint64_t x, int64_t R,
                                                 int m, int beta, int B, bool raw, unsigned& fb) {
    Located o;
    const double r = rescale_key(x, rt.x_min, rt.x_max, n_c, raw);
    const int f = rmi_leaf(rt.a0, rt.b0, r, F, n_c);
    const RmiLeaf lf = leaves[f];
    o.ph = rmi_predict(lf.a, lf.b, r, n_c);
    int64_t lo = max((int64_t)0, o.ph + lf.lo);
    int64_t hi = min(n_c, o.ph + (int64_t)lf.hi + 1);
    if (lo > hi) lo = hi = min(max(o.ph, (int64_t)0), n_c);
    // the lower bound lies in [lo, hi] iff K[lo-1] < x and K[hi] >= x
    if (lo > 0 && K[lo - 1] >= x) {
        ++fb;
        hi = lo - 1;
        lo = 0;
    } else if (hi < n_c && K[hi] < x) {
        ++fb;
        lo = hi + 1;
        hi = n_c;
    }
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (K[mid] < x) lo = mid + 1; else hi = mid;
    }
    o.p = lo;
    o.T = min(R, n_c);
    const int64_t nr = n_c - o.p;
    int64_t tlo = max((int64_t)0, o.T - nr), thi = min(o.T, o.p);
    while (tlo < thi) {
        const int64_t mid = (tlo + thi + 1) >> 1;
        const uint64_t dl = dist_code(K[o.p - mid], x, m, beta, B);
        const uint64_t dr = dist_code(K[o.p + (o.T - mid)], x, m, beta, B);
        if (dl <= dr) tlo = mid; else thi = mid - 1;
    }
    o.s = o.p - tlo;
    return o;
}

// ------------------------------------------------------- small utilities ----
inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
__device__ __forceinline__ size_t align_up_dev(size_t x, size_t a) { return (x + a - 1) / a * a; }
__device__ __forceinline__ int next_pow2_dev(int x) { return x <= 1 ? 1 : 1 << (32 - __clz(x - 1)); }

// Device kernels shared between translation units (defined in kernels.cu).
int launch_hash_t(const float* X, int64_t n, int d, const float* A, const float* b, int H,
                  double W, double* t_out, cudaStream_t s);
int launch_scores(const float* X, int64_t n, int d, const float* C, const double* half_norm,
                  int ncl, double* out, cudaStream_t s);
int launch_split_tf32(const float* x, int64_t n, float* hi, float* lo, cudaStream_t s);
int make_tensor_map(CUtensorMap* map, const void* base, int64_t rows, int d, int box_rows, bool bf16 = false);
int launch_to_bf16(const float* x, int64_t n, uint16_t* out, cudaStream_t s);
int launch_to_f16(const float* x, int64_t n, float scale, uint16_t* out, cudaStream_t s);
int launch_to_f8_rows(const float* x, int64_t n, int d, float* scale, uint8_t* out, cudaStream_t s);
int make_tensor_map8(CUtensorMap* map, const void* base, int64_t rows, int d, int box_rows);
// Power of two s with s * amax in [2^13, 2^14) (1 for amax == 0): scaled
// values stay in FP16's normal range with room below its maximum.
float f16_scale_host(float amax);
int launch_pack(const double* t, int64_t n, int L, int m, int beta, int hash_kind, int64_t row_offset,
                int64_t key_stride_row, int64_t key_stride_arr, uint64_t* keys,
                unsigned long long* n_boundary, unsigned long long* n_clamped, cudaStream_t s);

}  // namespace lider
