// Index construction (Sec. 3.3.2 "LIDER is built as follows", Sec. 3.3.1 for
// one core model): cluster the corpus by k-means (Sec. 3.2; Lloyd iterations
// on the device from Forgy rows, unless the caller gives the centroids),
// partition it by nearest centroid, hash every point into L packed hashkeys
// (projections given, or drawn from the seed), sort each (cluster, array)
// segment by key (ties by id), then fit one two-stage linear RMI per segment
// on re-scaled keys (Sec. 5.1, Sec. 5.2) and record each leaf's error window.
//
// Build is not on the search hot path; its sorts use CUB.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_radix_sort.cuh>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <unordered_set>

#include <cuda_fp16.h>

#include "lider_internal.cuh"

namespace lider {

namespace {

constexpr int64_t kRowChunk = 131072;   // rows per hashing / assignment pass

__global__ void half_norm_kernel(const float* __restrict__ C, int ncl, int d, double* __restrict__ hn) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncl) return;
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        const double v = (double)C[(int64_t)j * d + i];
        s = __dadd_rn(s, __dmul_rn(v, v));      // each product is exact in FP64
    }
    hn[j] = 0.5 * s;
}

// Nearest centroid per row: argmax of x.mu - |mu|^2/2, ties -> lower index.
__global__ void argmax_rows_kernel(const double* __restrict__ S, int64_t n, int ncl,
                                   int64_t row_offset, int32_t* __restrict__ asg) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double best = -INFINITY;
    int bj = 0x7fffffff;
    for (int j = lane; j < ncl; j += 32) {
        const double v = S[row * ncl + j];
        if (v > best || (v == best && j < bj)) { best = v; bj = j; }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ov > best || (ov == best && oj < bj)) { best = ov; bj = oj; }
    }
    if (lane == 0) asg[row_offset + row] = bj;
}

__global__ void iota_kernel(int64_t* __restrict__ v, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = i;
}

// cl_off[j] = first position of cluster j in the sorted assignment.
__global__ void cluster_offsets_kernel(const int32_t* __restrict__ sorted_asg, int64_t n, int ncl,
                                       int64_t* __restrict__ cl_off) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > ncl) return;
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (sorted_asg[mid] < j) lo = mid + 1; else hi = mid;
    }
    cl_off[j] = lo;
}

// X_re[row] = corpus[orig_id[row]]: one warp per row, float4 copies.
__global__ void gather_rows_kernel(const float* __restrict__ src, const int64_t* __restrict__ ids,
                                   int64_t n, int d, float* __restrict__ dst) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float4* s = reinterpret_cast<const float4*>(src + ids[row] * (int64_t)d);
    float4* o = reinterpret_cast<float4*>(dst + row * (int64_t)d);
    for (int i = lane; i < d / 4; i += 32) o[i] = s[i];
}

// Largest row norm (out[0], rounded up) and largest |x_ij| (out[1]), as the
// bits of non-negative floats (atomicMax on the bits orders them); warp per
// row, FP64 sum of squares.
__global__ void max_norms_kernel(const float* __restrict__ X, int64_t n, int d, unsigned int* __restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float* x = X + row * d;
    double s = 0.0;
    float amax = 0.f;
    for (int i = lane; i < d; i += 32) {
        s = fma((double)x[i], (double)x[i], s);
        amax = fmaxf(amax, fabsf(x[i]));
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    }
    if (lane == 0) {
        atomicMax(out, __float_as_uint(__double2float_ru(sqrt(s))));
        atomicMax(out + 1, __float_as_uint(amax));
    }
}

// |row| of each of n rows (warp per row, FP64 sum of squares, rounded up).
__global__ void row_norms_kernel(const float* __restrict__ X, int64_t n, int d, float* __restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double s = 0.0;
    for (int i = lane; i < d; i += 32) s = fma((double)X[row * d + i], (double)X[row * d + i], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[row] = __double2float_ru(sqrt(s));
}

// FP16 copy's rounding: per row, |fp16(s x) - s x| into out[0] and |fp16(s x)|
// into out[1], maxima as float bits (rounded up); warp per row, FP64 sums.
__global__ void f16_residual_kernel(const float* __restrict__ X, int64_t n, int d, float scale,
                                    unsigned int* __restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    double r2 = 0.0, h2 = 0.0;
    for (int i = lane; i < d; i += 32) {
        const float v = X[row * d + i] * scale;
        const float h = __half2float(__float2half_rn(v));
        const double r = (double)h - (double)v;
        r2 = fma(r, r, r2);
        h2 = fma((double)h, (double)h, h2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        r2 += __shfl_xor_sync(0xffffffffu, r2, o);
        h2 += __shfl_xor_sync(0xffffffffu, h2, o);
    }
    if (lane == 0) {
        atomicMax(out, __float_as_uint(__double2float_ru(sqrt(r2))));
        atomicMax(out + 1, __float_as_uint(__double2float_ru(sqrt(h2))));
    }
}

__global__ void inverse_ids_kernel(const int64_t* __restrict__ orig_id, int64_t n, int32_t* __restrict__ row_of) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) row_of[orig_id[r]] = (int32_t)r;
}

// pos[l][row] = row - cl_off[cluster(row)], the cluster-local row index.
__global__ void local_pos_kernel(const int32_t* __restrict__ sorted_asg, const int64_t* __restrict__ cl_off,
                                 int64_t n, int L, int32_t* __restrict__ pos) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    const int32_t p = (int32_t)(row - cl_off[sorted_asg[row]]);
    for (int l = 0; l < L; ++l) pos[(int64_t)l * n + row] = p;
}

// ---------------------------------------------------------------- k-means ----
// Forgy initialisation: the n_clusters initial centroids are distinct rows of
// the training rows, drawn by Floyd's sampling algorithm (Bentley and Floyd,
// 1987) from the counter-based SplitMix64 generator (Steele, Lea and Flood,
// 2014): draw i is mix64(seed + (i + 1) * 0x9E3779B97F4A7C15 mod 2^64), and the
// integer uniform on [0, j] is that draw mod (j + 1).  Rows ascending.
uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t splitmix64_dev(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

std::vector<int64_t> forgy_rows(uint64_t seed, int64_t n, int64_t count) {
    std::unordered_set<int64_t> chosen;
    chosen.reserve((size_t)count * 2);
    uint64_t i = 0;
    for (int64_t j = n - count; j < n; ++j, ++i) {
        const int64_t t = (int64_t)(splitmix64(seed, i) % (uint64_t)(j + 1));
        chosen.insert(chosen.count(t) ? j : t);
    }
    std::vector<int64_t> rows(chosen.begin(), chosen.end());
    std::sort(rows.begin(), rows.end());
    return rows;
}

// Lloyd update (Sec. 3.2): centroid j becomes the mean of its rows, summed in
// FP64 over the rows in ascending order (four interleaved partial sums joined
// in a fixed order, so the result does not depend on scheduling) and rounded to
// FP32, the precision the index keeps; a cluster without rows keeps its
// centroid.  Block (cluster, 128 dimensions), thread per dimension: the
// member rows' loads are coalesced across the block.
__global__ void __launch_bounds__(128) centroid_mean_kernel(const float* __restrict__ X, int d,
                                                            const int64_t* __restrict__ rows,
                                                            const int64_t* __restrict__ off, float* __restrict__ C) {
    const int j = blockIdx.x;
    const int i = blockIdx.y * blockDim.x + threadIdx.x;
    if (i >= d) return;
    const int64_t s = off[j], e = off[j + 1];
    if (s >= e) return;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int64_t r = s;
    for (; r + 4 <= e; r += 4) {
        a0 = __dadd_rn(a0, (double)X[rows[r] * d + i]);
        a1 = __dadd_rn(a1, (double)X[rows[r + 1] * d + i]);
        a2 = __dadd_rn(a2, (double)X[rows[r + 2] * d + i]);
        a3 = __dadd_rn(a3, (double)X[rows[r + 3] * d + i]);
    }
    for (; r < e; ++r) a0 = __dadd_rn(a0, (double)X[rows[r] * d + i]);
    const double sum = __dadd_rn(__dadd_rn(a0, a1), __dadd_rn(a2, a3));
    C[(int64_t)j * d + i] = __double2float_rn(__ddiv_rn(sum, (double)(e - s)));
}

// LSH draws from the seed when the caller gives none (Sec. 4.1: the hash
// family is random): a_hi ~ N(0, 1) by the Box-Muller transform of two
// SplitMix64 draws, b_h ~ U[0, W) (kept below W after rounding to FP32); the
// two streams start from states derived from the seed.  Hyperplane hashes take
// no offsets (b = 0).
constexpr uint64_t kStreamA = 0x4C49444552000001ull;   // derived-state indices of
constexpr uint64_t kStreamB = 0x4C49444552000002ull;   // the two streams

__global__ void draw_projections_kernel(uint64_t seed, int H, int d, float W, bool hyper, float* __restrict__ A,
                                        float* __restrict__ b) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t sa = splitmix64_dev(seed, kStreamA), sb = splitmix64_dev(seed, kStreamB);
    if (e < (int64_t)H * d) {
        const uint64_t r1 = splitmix64_dev(sa, 2 * (uint64_t)e), r2 = splitmix64_dev(sa, 2 * (uint64_t)e + 1);
        const double u1 = ((double)(r1 >> 11) + 1.0) * 0x1.0p-53;    // (0, 1]
        const double u2 = (double)(r2 >> 11) * 0x1.0p-53;            // [0, 1)
        A[e] = (float)(sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2));
    }
    if (e < H) {
        if (hyper) {
            b[e] = 0.f;
        } else {
            const double u = (double)(splitmix64_dev(sb, (uint64_t)e) >> 11) * 0x1.0p-53;
            float v = (float)(u * (double)W);
            if (!(v < W)) v = nextafterf(W, 0.f);
            b[e] = v;
        }
    }
}

// ---------------------------------------------------------------- RMI fit ----
__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        red[32] = t;
    }
    __syncthreads();
    return red[32];
}

__device__ __forceinline__ int64_t seg_lower_bound(const uint64_t* K, int64_t n, uint64_t x) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (K[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// One block per (cluster j, array l).  Root: least squares of position i on
// r_i.  Leaves: the root's prediction selects leaf floor(pred * F / n_c);
// since r_i is non-decreasing along the sorted array and the root slope is
// non-negative, every leaf owns one contiguous run of positions, found here by
// binary search.  Each leaf fits its own least squares (zero variance: slope
// 0, intercept = mean position; empty: copy of the root) and records
// [min, max] of (first position of key_i) - prediction_i.  raw: the model
// learns the raw key values instead of re-scaled ones (Sec. 7.4 ablation).
__global__ void __launch_bounds__(256) rmi_fit_kernel(
        const uint64_t* __restrict__ keys, const int64_t* __restrict__ cl_off, int64_t n,
        int L, int F, bool raw, RmiRoot* __restrict__ roots, RmiLeaf* __restrict__ leaves,
        int* __restrict__ err_flag) {
    __shared__ double red[33];
    const int j = blockIdx.x, l = blockIdx.y;
    const int64_t base = cl_off[j];
    const int64_t n_c = cl_off[j + 1] - base;
    RmiRoot* root = roots + (int64_t)j * L + l;
    RmiLeaf* lf = leaves + ((int64_t)j * L + l) * F;
    if (n_c == 0) {
        if (threadIdx.x == 0) *root = RmiRoot{0.0, 0.0, 0ull, 0ull};
        for (int f = threadIdx.x; f < F; f += blockDim.x) lf[f] = RmiLeaf{0.0, 0.0, 0, 0};
        return;
    }
    const uint64_t* K = keys + (int64_t)l * n + base;
    const uint64_t x_min = K[0], x_max = K[n_c - 1];

    // root least squares, two passes
    double sr = 0.0, sy = 0.0;
    for (int64_t i = threadIdx.x; i < n_c; i += blockDim.x) {
        sr += rescale_key(K[i], x_min, x_max, n_c, raw);
        sy += (double)i;
    }
    sr = block_sum(sr, red);
    sy = block_sum(sy, red);
    const double rbar = sr / (double)n_c, ybar = sy / (double)n_c;
    const double r_first = rescale_key(K[0], x_min, x_max, n_c, raw);
    const double r_last = rescale_key(K[n_c - 1], x_min, x_max, n_c, raw);
    double a0, b0;
    if (r_first == r_last) {
        a0 = ybar; b0 = 0.0;
    } else {
        double sxx = 0.0, sxy = 0.0;
        for (int64_t i = threadIdx.x; i < n_c; i += blockDim.x) {
            const double dr = rescale_key(K[i], x_min, x_max, n_c, raw) - rbar;
            sxx += dr * dr;
            sxy += dr * ((double)i - ybar);
        }
        sxx = block_sum(sxx, red);
        sxy = block_sum(sxy, red);
        b0 = sxy / sxx;
        a0 = ybar - b0 * rbar;
    }
    if (threadIdx.x == 0) {
        *root = RmiRoot{a0, b0, x_min, x_max};
        if (b0 < 0.0) atomicExch(err_flag, 1);   // contiguity of leaves needs b0 >= 0
    }
    if (b0 < 0.0) return;

    for (int f = threadIdx.x; f < F; f += blockDim.x) {
        // first position whose leaf is >= f, and >= f + 1
        int64_t bounds[2];
        for (int e = 0; e < 2; ++e) {
            int64_t lo = 0, hi = n_c;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const double r = rescale_key(K[mid], x_min, x_max, n_c, raw);
                if (rmi_leaf(a0, b0, r, F, n_c) < f + e) lo = mid + 1; else hi = mid;
            }
            bounds[e] = lo;
        }
        const int64_t s = bounds[0], t = bounds[1];
        if (s >= t) {
            lf[f] = RmiLeaf{a0, b0, 0, 0};
            continue;
        }
        const int64_t cnt = t - s;
        double lr = 0.0, ly = 0.0;
        for (int64_t i = s; i < t; ++i) {
            lr += rescale_key(K[i], x_min, x_max, n_c, raw);
            ly += (double)i;
        }
        const double lrbar = lr / (double)cnt, lybar = ly / (double)cnt;
        double a, b;
        if (rescale_key(K[s], x_min, x_max, n_c, raw) == rescale_key(K[t - 1], x_min, x_max, n_c, raw)) {
            a = lybar; b = 0.0;
        } else {
            double sxx = 0.0, sxy = 0.0;
            for (int64_t i = s; i < t; ++i) {
                const double dr = rescale_key(K[i], x_min, x_max, n_c, raw) - lrbar;
                sxx += dr * dr;
                sxy += dr * ((double)i - lybar);
            }
            b = sxy / sxx;
            a = lybar - b * lrbar;
        }
        int64_t elo = INT64_MAX, ehi = INT64_MIN;
        for (int64_t i = s; i < t; ++i) {
            const double r = rescale_key(K[i], x_min, x_max, n_c, raw);
            const int64_t lb = (i > s && K[i - 1] != K[i]) ? i : seg_lower_bound(K, i, K[i]);
            const int64_t e = lb - rmi_predict(a, b, r, n_c);
            elo = min(elo, e);
            ehi = max(ehi, e);
        }
        lf[f] = RmiLeaf{a, b, (int32_t)elo, (int32_t)ehi};
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    template <class T> T* as() { return static_cast<T*>(p); }
};

int dev_alloc(void** p, size_t bytes, const char* what) {
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(LIDER_ENOMEM, std::string("cudaMalloc failed for ") + what + " (" +
                                      std::to_string(bytes) + " bytes): " + cudaGetErrorString(e));
    }
    return LIDER_OK;
}

void release(lider_index* ix) {
    if (!ix) return;
    void* bufs[] = {ix->X, ix->orig_id, ix->cl_off, ix->C, ix->half_norm, ix->A, ix->bproj,
                    ix->keys, ix->pos, ix->root, ix->leaf, ix->X_hi, ix->X_lo, ix->row_of, ix->X_h16, ix->F_hi, ix->F_lo,
                    ix->a_norm, ix->X_f8, ix->x_rowscale, ix->ckeys, ix->cpos, ix->croot,
                    ix->cleaf};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (ix->pool) cudaMemPoolDestroy(ix->pool);
    if (ix->side) cudaStreamDestroy(ix->side);
    delete ix;
}

// Lloyd's k-means (Sec. 3.2) over the first ns rows of X: Forgy rows, then
// `iters` rounds of exact nearest-centroid assignment (Dot2 scores of
// x.mu - |mu|^2/2 finished in FP64, ties to the lower index; the same
// arithmetic as the partition below) and centroid means (centroid_mean_kernel).
// C receives the FP32 centroids.  The other buffers are scratch: asg and
// asg_sorted hold ns int32, ids_in and ids_sorted ns int64, off ncl + 1 int64,
// sbuf chunk x ncl FP64.
int kmeans_run(const float* X, int64_t ns, int d, int ncl, int iters, uint64_t seed, float* C, double* hn,
               double* sbuf, int64_t chunk, int32_t* asg, int32_t* asg_sorted, int64_t* ids_in, int64_t* ids_sorted,
               int64_t* off, cudaStream_t st) {
    {
        const std::vector<int64_t> init = forgy_rows(seed, ns, ncl);
        LIDER_CUDA_TRY(cudaMemcpyAsync(ids_in, init.data(), init.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        gather_rows_kernel<<<(unsigned)cdiv((int64_t)ncl * 32, 256), 256, 0, st>>>(X, ids_in, ncl, d, C);
        LIDER_LAUNCH_CHECK("gather_rows_kernel<forgy>");
        LIDER_CUDA_TRY(cudaStreamSynchronize(st));   // `init` is host memory of this scope
    }
    int end_bit = 1;
    while ((1ll << end_bit) <= ncl) ++end_bit;
    size_t tmp_bytes = 0;
    LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, asg, asg_sorted, ids_in, ids_sorted, ns, 0,
                                                   end_bit, st));
    DevBuf tmp;
    int rc;
    if ((rc = dev_alloc(&tmp.p, tmp_bytes, "k-means sort scratch"))) return rc;
    for (int it = 0; it < iters; ++it) {
        half_norm_kernel<<<(unsigned)cdiv(ncl, 128), 128, 0, st>>>(C, ncl, d, hn);
        LIDER_LAUNCH_CHECK("half_norm_kernel");
        for (int64_t r0 = 0; r0 < ns; r0 += chunk) {
            const int64_t rows = std::min(chunk, ns - r0);
            if ((rc = launch_scores(X + r0 * d, rows, d, C, hn, ncl, sbuf, st))) return rc;
            argmax_rows_kernel<<<(unsigned)cdiv(rows * 32, 256), 256, 0, st>>>(sbuf, rows, ncl, r0, asg);
            LIDER_LAUNCH_CHECK("argmax_rows_kernel");
        }
        iota_kernel<<<(unsigned)cdiv(ns, 256), 256, 0, st>>>(ids_in, ns);
        LIDER_LAUNCH_CHECK("iota_kernel");
        LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, asg, asg_sorted, ids_in, ids_sorted, ns, 0,
                                                       end_bit, st));
        cluster_offsets_kernel<<<(unsigned)cdiv(ncl + 1, 128), 128, 0, st>>>(asg_sorted, ns, ncl, off);
        LIDER_LAUNCH_CHECK("cluster_offsets_kernel");
        centroid_mean_kernel<<<dim3((unsigned)ncl, (unsigned)cdiv(d, 128)), 128, 0, st>>>(X, d, ids_sorted, off, C);
        LIDER_LAUNCH_CHECK("centroid_mean_kernel");
    }
    LIDER_CUDA_TRY(cudaStreamSynchronize(st));    // tmp is freed on return
    return LIDER_OK;
}

int build_impl(const float* corpus, int64_t n, int32_t d, const float* centroids, int32_t ncl,
               const lider_cluster_params* cp, const float* A, const float* b, const lider_params* P,
               cudaStream_t st, lider_index** out) {
    using clock = std::chrono::steady_clock;
    const auto t_start = clock::now();
    if (!out) return fail(LIDER_EINVAL, "lider_build: out is NULL");
    *out = nullptr;
    if (!corpus || !P) return fail(LIDER_EINVAL, "lider_build: NULL argument");
    if (cp) {
        if (centroids) return fail(LIDER_EINVAL, "lider_build: centroids are given and would also be clustered");
        if ((A == nullptr) != (b == nullptr)) return fail(LIDER_EINVAL, "lider_build: give both A and b, or neither");
        ncl = cp->n_clusters;
        if (cp->kmeans_iters < 0 || cp->kmeans_iters > 100000)
            return fail(LIDER_EINVAL, "lider_build: kmeans_iters must be in [0, 100000]");
        if (cp->kmeans_sample < 0) return fail(LIDER_EINVAL, "lider_build: kmeans_sample must be >= 0");
    } else if (!centroids || !A || !b) {
        return fail(LIDER_EINVAL, "lider_build: NULL argument");
    }
    if (n < 1 || n > (int64_t)INT32_MAX) return fail(LIDER_EINVAL, "lider_build: n must be in [1, 2^31-1]");
    if (d < 4 || d % 4 != 0) return fail(LIDER_EINVAL, "lider_build: d must be a positive multiple of 4");
    if (d > LIDER_MAX_D) return fail(LIDER_ELIMIT, "lider_build: d exceeds LIDER_MAX_D");
    if (ncl < 1) return fail(LIDER_EINVAL, "lider_build: n_clusters must be >= 1");
    const int64_t n_train = cp ? (cp->kmeans_sample == 0 ? n : std::min<int64_t>(cp->kmeans_sample, n)) : 0;
    if (cp && ncl > n_train)
        return fail(LIDER_EINVAL, "lider_build: n_clusters exceeds the rows k-means learns from");
    if (P->L < 1 || P->m < 1 || P->rmi_leaves < 1 || P->r0 < 1 || P->B < 1)
        return fail(LIDER_EINVAL, "lider_build: L, m, rmi_leaves, r0 and B must be >= 1");
    if (P->hash_kind != LIDER_HASH_PSTABLE && P->hash_kind != LIDER_HASH_HYPERPLANE)
        return fail(LIDER_EINVAL, "lider_build: unknown hash_kind");
    const bool hyper = P->hash_kind == LIDER_HASH_HYPERPLANE;
    if (!hyper && (!(P->W > 0.0) || !std::isfinite(P->W))) return fail(LIDER_EINVAL, "lider_build: W must be > 0");
    if (P->m > 64) return fail(LIDER_EINVAL, "lider_build: m must be <= 64");
    const int beta = hyper ? 1 : 64 / P->m;
    if ((int64_t)beta * P->B > 56)
        return fail(LIDER_EINVAL, "lider_build: (bits per element) * B must be <= 56 (p-stable: floor(64/m) bits)");
    if (P->route_kind != LIDER_ROUTE_EXACT && P->route_kind != LIDER_ROUTE_CORE)
        return fail(LIDER_EINVAL, "lider_build: unknown route_kind");
    if (P->raw_keys != 0 && P->raw_keys != 1) return fail(LIDER_EINVAL, "lider_build: raw_keys must be 0 or 1");
    if (P->route_kind == LIDER_ROUTE_CORE && ncl > kRouteCoreMaxClusters)
        return fail(LIDER_ELIMIT, "lider_build: LIDER_ROUTE_CORE supports n_clusters <= 8192");
    // hyperplane hashes take t = a.x: no offset, unit width
    const double W = hyper ? 1.0 : P->W;
    const bool raw = P->raw_keys != 0;
    if (P->L > LIDER_MAX_L) return fail(LIDER_ELIMIT, "lider_build: L exceeds LIDER_MAX_L");
    if (P->rmi_leaves > (1 << 24)) return fail(LIDER_ELIMIT, "lider_build: rmi_leaves too large");
    if (P->score_mode != LIDER_SCORE_TENSOR && P->score_mode != LIDER_SCORE_SIMT && P->score_mode != LIDER_SCORE_BF16 &&
        P->score_mode != LIDER_SCORE_F16 && P->score_mode != LIDER_SCORE_FP8)
        return fail(LIDER_EINVAL, "lider_build: unknown score_mode");
    if (P->score_mode != LIDER_SCORE_SIMT && P->L > 16)
        return fail(LIDER_ELIMIT, "lider_build: tensor-core scoring supports L <= 16 (use LIDER_SCORE_SIMT)");
    if ((P->score_mode == LIDER_SCORE_BF16 || P->score_mode == LIDER_SCORE_F16) && d % 8 != 0)
        return fail(LIDER_EINVAL, "lider_build: 16-bit tensor-core scoring needs d % 8 == 0");
    if (P->score_mode == LIDER_SCORE_FP8 && d % 16 != 0)
        return fail(LIDER_EINVAL, "lider_build: FP8 tensor-core scoring needs d % 16 == 0");
    if (P->rerank < 0 || P->rerank > 64) return fail(LIDER_EINVAL, "lider_build: rerank must be in [0, 64]");

    int dev = 0;
    LIDER_CUDA_TRY(cudaGetDevice(&dev));
    lider_index* ix = new lider_index();
    struct Guard {
        lider_index* ix;
        ~Guard() { if (ix) release(ix); }
    } guard{ix};
    ix->device = dev;
    ix->params = *P;
    if (ix->params.rerank == 0) ix->params.rerank = 4;
    LIDER_CUDA_TRY(cudaDeviceGetAttribute(&ix->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const int L = P->L, m = P->m, H = L * m, F = P->rmi_leaves;

    int rc;
#define ALLOC(ptr, bytes, what) \
    if ((rc = dev_alloc((void**)&(ptr), (bytes), what)) != LIDER_OK) return rc
    ALLOC(ix->X, (size_t)n * d * sizeof(float), "corpus");
    ALLOC(ix->orig_id, (size_t)n * sizeof(int64_t), "ids");
    ALLOC(ix->cl_off, (size_t)(ncl + 1) * sizeof(int64_t), "cluster offsets");
    ALLOC(ix->C, (size_t)ncl * d * sizeof(float), "centroids");
    ALLOC(ix->half_norm, (size_t)ncl * sizeof(double), "centroid norms");
    ALLOC(ix->A, (size_t)H * d * sizeof(float), "projections");
    ALLOC(ix->bproj, (size_t)H * sizeof(float), "offsets");
    ALLOC(ix->keys, (size_t)L * n * sizeof(uint64_t), "keys");
    ALLOC(ix->pos, (size_t)L * n * sizeof(int32_t), "positions");
    ALLOC(ix->root, (size_t)ncl * L * sizeof(RmiRoot), "rmi roots");
    ALLOC(ix->leaf, (size_t)ncl * L * F * sizeof(RmiLeaf), "rmi leaves");

    // scratch of the partition (and of k-means)
    const int64_t chunk = std::min<int64_t>(n, kRowChunk);
    DevBuf asg, asg_sorted, ids_in, tbuf, sbuf, errf;
    ALLOC(asg.p, (size_t)n * sizeof(int32_t), "assignment");
    ALLOC(asg_sorted.p, (size_t)n * sizeof(int32_t), "sorted assignment");
    ALLOC(ids_in.p, (size_t)n * sizeof(int64_t), "ids");
    ALLOC(sbuf.p, (size_t)chunk * std::max(ncl, H) * sizeof(double), "score chunk");
    ALLOC(errf.p, 64, "flags");
    LIDER_CUDA_TRY(cudaMemsetAsync(errf.p, 0, 64, st));

    if (cp) {
        // 0. k-means (Sec. 3.2); orig_id and cl_off serve as its scratch
        LIDER_CUDA_TRY(cudaStreamSynchronize(st));
        const auto t0 = clock::now();
        if ((rc = kmeans_run(corpus, n_train, d, ncl, cp->kmeans_iters, cp->seed, ix->C, ix->half_norm,
                             sbuf.as<double>(), std::min<int64_t>(n_train, kRowChunk), asg.as<int32_t>(),
                             asg_sorted.as<int32_t>(), ids_in.as<int64_t>(), ix->orig_id, ix->cl_off, st)))
            return rc;
        ix->kmeans_ms = std::chrono::duration<double, std::milli>(clock::now() - t0).count();
        ix->cluster = *cp;
        ix->clustered = true;
    } else {
        LIDER_CUDA_TRY(cudaMemcpyAsync(ix->C, centroids, (size_t)ncl * d * sizeof(float), cudaMemcpyDefault, st));
    }
    if (A) {
        LIDER_CUDA_TRY(cudaMemcpyAsync(ix->A, A, (size_t)H * d * sizeof(float), cudaMemcpyDefault, st));
        if (hyper) LIDER_CUDA_TRY(cudaMemsetAsync(ix->bproj, 0, (size_t)H * sizeof(float), st));
        else LIDER_CUDA_TRY(cudaMemcpyAsync(ix->bproj, b, (size_t)H * sizeof(float), cudaMemcpyDefault, st));
    } else {
        draw_projections_kernel<<<(unsigned)cdiv((int64_t)H * d, 256), 256, 0, st>>>(cp->seed, H, d, (float)P->W,
                                                                                  hyper, ix->A, ix->bproj);
        LIDER_LAUNCH_CHECK("draw_projections_kernel");
        ix->projections_drawn = true;
    }
    half_norm_kernel<<<(unsigned)cdiv(ncl, 128), 128, 0, st>>>(ix->C, ncl, d, ix->half_norm);
    LIDER_LAUNCH_CHECK("half_norm_kernel");
    if (P->score_mode != LIDER_SCORE_SIMT) {      // tensor-core hashing and routing
        // one front operand: the projections, zero rows up to a 256-row
        // boundary, then the centroids, each split into TF32 head and tail
        const int hp = (int)cdiv(H, 256) * 256;
        const int64_t frows = (int64_t)hp + ncl;
        ALLOC(ix->F_hi, (size_t)frows * d * sizeof(float), "front operand TF32 head");
        ALLOC(ix->F_lo, (size_t)frows * d * sizeof(float), "front operand TF32 tail");
        ix->front_hp = hp;
        LIDER_CUDA_TRY(cudaMemsetAsync(ix->F_hi, 0, (size_t)hp * d * sizeof(float), st));
        LIDER_CUDA_TRY(cudaMemsetAsync(ix->F_lo, 0, (size_t)hp * d * sizeof(float), st));
        if ((rc = launch_split_tf32(ix->A, (int64_t)H * d, ix->F_hi, ix->F_lo, st))) return rc;
        if ((rc = launch_split_tf32(ix->C, (int64_t)ncl * d, ix->F_hi + (int64_t)hp * d, ix->F_lo + (int64_t)hp * d,
                                    st)))
            return rc;
        if ((rc = make_tensor_map(&ix->map_fhi, ix->F_hi, frows, d, 256))) return rc;
        if ((rc = make_tensor_map(&ix->map_flo, ix->F_lo, frows, d, 256))) return rc;
        ALLOC(ix->a_norm, (size_t)H * sizeof(float), "projection norms");
        row_norms_kernel<<<(unsigned)cdiv((int64_t)H * 32, 256), 256, 0, st>>>(ix->A, H, d, ix->a_norm);
        LIDER_LAUNCH_CHECK("row_norms_kernel");
        std::vector<double> hn(ncl);
        LIDER_CUDA_TRY(cudaMemcpyAsync(hn.data(), ix->half_norm, ncl * sizeof(double), cudaMemcpyDeviceToHost, st));
        LIDER_CUDA_TRY(cudaStreamSynchronize(st));
        double mx = 0.0;
        for (double v : hn) mx = std::max(mx, std::sqrt(2.0 * v));
        ix->max_cnorm = (float)mx;
    }

    // 1. partition: nearest centroid of every point
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        if ((rc = launch_scores(corpus + r0 * d, rows, d, ix->C, ix->half_norm, ncl, sbuf.as<double>(), st)))
            return rc;
        argmax_rows_kernel<<<(unsigned)cdiv(rows * 32, 256), 256, 0, st>>>(sbuf.as<double>(), rows, ncl, r0,
                                                                          asg.as<int32_t>());
        LIDER_LAUNCH_CHECK("argmax_rows_kernel");
    }

    // 2. stable reorder by cluster (ids ascending inside each cluster)
    iota_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(ids_in.as<int64_t>(), n);
    LIDER_LAUNCH_CHECK("iota_kernel");
    int end_bit = 1;
    while ((1ll << end_bit) <= ncl) ++end_bit;
    {
        size_t tmp_bytes = 0;
        LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, asg.as<int32_t>(), asg_sorted.as<int32_t>(),
                                                       ids_in.as<int64_t>(), ix->orig_id, n, 0, end_bit, st));
        DevBuf tmp;
        ALLOC(tmp.p, tmp_bytes, "sort scratch");
        LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, asg.as<int32_t>(), asg_sorted.as<int32_t>(),
                                                       ids_in.as<int64_t>(), ix->orig_id, n, 0, end_bit, st));
    }
    cluster_offsets_kernel<<<(unsigned)cdiv(ncl + 1, 128), 128, 0, st>>>(asg_sorted.as<int32_t>(), n, ncl, ix->cl_off);
    LIDER_LAUNCH_CHECK("cluster_offsets_kernel");
    gather_rows_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(corpus, ix->orig_id, n, d, ix->X);
    LIDER_LAUNCH_CHECK("gather_rows_kernel");

    // 3. hash every point (shared projections), keys laid out [array][row]
    DevBuf keys_tmp, pos_tmp;
    ALLOC(keys_tmp.p, (size_t)L * n * sizeof(uint64_t), "key scratch");
    ALLOC(pos_tmp.p, (size_t)L * n * sizeof(int32_t), "position scratch");
    for (int64_t r0 = 0; r0 < n; r0 += chunk) {
        const int64_t rows = std::min(chunk, n - r0);
        if ((rc = launch_hash_t(ix->X + r0 * d, rows, d, ix->A, ix->bproj, H, W, sbuf.as<double>(), st))) return rc;
        if ((rc = launch_pack(sbuf.as<double>(), rows, L, m, beta, P->hash_kind, r0, 1, n, keys_tmp.as<uint64_t>(),
                              nullptr, nullptr, st)))
            return rc;
    }
    local_pos_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(asg_sorted.as<int32_t>(), ix->cl_off, n, L,
                                                           pos_tmp.as<int32_t>());
    LIDER_LAUNCH_CHECK("local_pos_kernel");

    // 4. sort every (cluster, array) segment by key; radix sort is stable, so
    //    equal keys stay in ascending position (= ascending id) order
    {
        size_t tmp_bytes = 0;
        LIDER_CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(
            nullptr, tmp_bytes, keys_tmp.as<uint64_t>(), ix->keys, pos_tmp.as<int32_t>(), ix->pos, n, ncl,
            ix->cl_off, ix->cl_off + 1, 0, 64, st));
        DevBuf tmp;
        ALLOC(tmp.p, tmp_bytes, "segmented sort scratch");
        for (int l = 0; l < L; ++l) {
            LIDER_CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(
                tmp.p, tmp_bytes, keys_tmp.as<uint64_t>() + (int64_t)l * n, ix->keys + (int64_t)l * n,
                pos_tmp.as<int32_t>() + (int64_t)l * n, ix->pos + (int64_t)l * n, n, ncl, ix->cl_off,
                ix->cl_off + 1, 0, 64, st));
        }
    }

    // tensor-core scoring: norms for the error guards, TF32 split (or 16-bit
    // copy) of the corpus, inverse ids, TMA maps
    if (P->score_mode != LIDER_SCORE_SIMT) {
        DevBuf mx;
        ALLOC(mx.p, 2 * sizeof(unsigned int), "norms");
        LIDER_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 2 * sizeof(unsigned int), st));
        max_norms_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(ix->X, n, d, mx.as<unsigned int>());
        LIDER_LAUNCH_CHECK("max_norms_kernel");
        unsigned int bits[2] = {0u, 0u};
        LIDER_CUDA_TRY(cudaMemcpyAsync(bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
        LIDER_CUDA_TRY(cudaStreamSynchronize(st));
        float norms[2];
        std::memcpy(norms, bits, sizeof(norms));
        ix->max_xnorm = norms[0];
        if (!std::isfinite(norms[0]))
            return fail(LIDER_EINVAL, "lider_build: corpus holds a non-finite value or a row norm overflows FP32");
        if (P->score_mode == LIDER_SCORE_TENSOR) {
            ALLOC(ix->X_hi, (size_t)n * d * sizeof(float), "corpus TF32 head");
            ALLOC(ix->X_lo, (size_t)n * d * sizeof(float), "corpus TF32 tail");
            if ((rc = launch_split_tf32(ix->X, n * d, ix->X_hi, ix->X_lo, st))) return rc;
            if ((rc = make_tensor_map(&ix->map_xhi, ix->X_hi, n, d, 256))) return rc;
            if ((rc = make_tensor_map(&ix->map_xlo, ix->X_lo, n, d, 256))) return rc;
        } else if (P->score_mode == LIDER_SCORE_FP8) {
            ALLOC(ix->X_f8, (size_t)n * d, "corpus FP8 copy");
            ALLOC(ix->x_rowscale, (size_t)n * sizeof(float), "corpus FP8 row scales");
            if ((rc = launch_to_f8_rows(ix->X, n, d, ix->x_rowscale, ix->X_f8, st))) return rc;
            if ((rc = make_tensor_map8(&ix->map_xf8, ix->X_f8, n, d, 256))) return rc;
        } else if (P->score_mode == LIDER_SCORE_BF16) {
            ALLOC(ix->X_h16, (size_t)n * d * sizeof(uint16_t), "corpus BF16 copy");
            if ((rc = launch_to_bf16(ix->X, n * d, ix->X_h16, st))) return rc;
            if ((rc = make_tensor_map(&ix->map_xh16, ix->X_h16, n, d, 256, true))) return rc;
        } else {
            ix->x_scale = f16_scale_host(norms[1]);
            LIDER_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 2 * sizeof(unsigned int), st));
            f16_residual_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(ix->X, n, d, ix->x_scale,
                                                                             mx.as<unsigned int>());
            LIDER_LAUNCH_CHECK("f16_residual_kernel");
            LIDER_CUDA_TRY(cudaMemcpyAsync(bits, mx.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
            LIDER_CUDA_TRY(cudaStreamSynchronize(st));
            std::memcpy(norms, bits, sizeof(norms));
            ix->xres_max = norms[0];
            ix->xhat_max = norms[1];
            ALLOC(ix->X_h16, (size_t)n * d * sizeof(uint16_t), "corpus FP16 copy");
            if ((rc = launch_to_f16(ix->X, n * d, ix->x_scale, ix->X_h16, st))) return rc;
            if ((rc = make_tensor_map(&ix->map_xh16, ix->X_h16, n, d, 256, true))) return rc;
        }
        ALLOC(ix->row_of, (size_t)n * sizeof(int32_t), "row of id");
        inverse_ids_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(ix->orig_id, n, ix->row_of);
        LIDER_LAUNCH_CHECK("inverse_ids_kernel");
    }

    // 5. RMI per (cluster, array)
    rmi_fit_kernel<<<dim3(ncl, L), 256, 0, st>>>(ix->keys, ix->cl_off, n, L, F, raw, ix->root, ix->leaf,
                                                errf.as<int>());
    LIDER_LAUNCH_CHECK("rmi_fit_kernel");

    // 6. Layer-1 centroids retriever (Sec. 3.2): a core model over the
    //    centroids with the same projections, laid out as one cluster
    std::vector<int32_t> h_cid;
    int64_t h_coff[2] = {0, ncl};
    DevBuf ct, ckt, cpt, coff;
    if (P->route_kind == LIDER_ROUTE_CORE) {
        ALLOC(ix->ckeys, (size_t)L * ncl * sizeof(uint64_t), "centroid keys");
        ALLOC(ix->cpos, (size_t)L * ncl * sizeof(int32_t), "centroid entries");
        ALLOC(ix->croot, (size_t)L * sizeof(RmiRoot), "centroid rmi roots");
        ALLOC(ix->cleaf, (size_t)L * F * sizeof(RmiLeaf), "centroid rmi leaves");
        ALLOC(ct.p, (size_t)ncl * H * sizeof(double), "centroid projections");
        ALLOC(ckt.p, (size_t)L * ncl * sizeof(uint64_t), "centroid key scratch");
        ALLOC(cpt.p, (size_t)L * ncl * sizeof(int32_t), "centroid entry scratch");
        ALLOC(coff.p, sizeof(h_coff), "centroid offsets");
        h_cid.resize((size_t)L * ncl);
        for (int l = 0; l < L; ++l)
            for (int j = 0; j < ncl; ++j) h_cid[(size_t)l * ncl + j] = j;
        LIDER_CUDA_TRY(cudaMemcpyAsync(cpt.p, h_cid.data(), h_cid.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        LIDER_CUDA_TRY(cudaMemcpyAsync(coff.p, h_coff, sizeof(h_coff), cudaMemcpyHostToDevice, st));
        if ((rc = launch_hash_t(ix->C, ncl, d, ix->A, ix->bproj, H, W, ct.as<double>(), st))) return rc;
        if ((rc = launch_pack(ct.as<double>(), ncl, L, m, beta, P->hash_kind, 0, 1, ncl, ckt.as<uint64_t>(), nullptr,
                              nullptr, st)))
            return rc;
        // stable radix sort: equal keys stay in ascending centroid order
        size_t tmp_bytes = 0;
        LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, ckt.as<uint64_t>(), ix->ckeys,
                                                       cpt.as<int32_t>(), ix->cpos, ncl, 0, 64, st));
        DevBuf tmp;
        ALLOC(tmp.p, tmp_bytes, "centroid sort scratch");
        for (int l = 0; l < L; ++l)
            LIDER_CUDA_TRY(cub::DeviceRadixSort::SortPairs(
                tmp.p, tmp_bytes, ckt.as<uint64_t>() + (int64_t)l * ncl, ix->ckeys + (int64_t)l * ncl,
                cpt.as<int32_t>() + (int64_t)l * ncl, ix->cpos + (int64_t)l * ncl, ncl, 0, 64, st));
        rmi_fit_kernel<<<dim3(1, L), 256, 0, st>>>(ix->ckeys, coff.as<int64_t>(), ncl, L, F, raw, ix->croot,
                                                  ix->cleaf, errf.as<int>());
        LIDER_LAUNCH_CHECK("rmi_fit_kernel<centroids>");
        LIDER_CUDA_TRY(cudaStreamSynchronize(st));   // the temporaries above are freed on return
    }

    ix->h_cl_off.resize(ncl + 1);
    LIDER_CUDA_TRY(cudaMemcpyAsync(ix->h_cl_off.data(), ix->cl_off, (ncl + 1) * sizeof(int64_t),
                                   cudaMemcpyDeviceToHost, st));
    int h_err = 0;
    LIDER_CUDA_TRY(cudaMemcpyAsync(&h_err, errf.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    LIDER_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return fail(LIDER_ECUDA, "lider_build: negative RMI root slope (unsorted segment)");

    // stream-ordered pool for search scratch; memory is kept between calls
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    LIDER_CUDA_TRY(cudaMemPoolCreate(&ix->pool, &props));
    uint64_t thr = UINT64_MAX;
    LIDER_CUDA_TRY(cudaMemPoolSetAttribute(ix->pool, cudaMemPoolAttrReleaseThreshold, &thr));

    Geometry& g = ix->g;
    g.n = n; g.d = d; g.ncl = ncl; g.L = L; g.m = m; g.F = F; g.beta = beta; g.B = P->B; g.H = H;
    g.W = W;
    g.hash_kind = P->hash_kind;
    g.raw_keys = P->raw_keys;
    g.X = ix->X; g.orig_id = ix->orig_id; g.cl_off = ix->cl_off; g.C = ix->C; g.half_norm = ix->half_norm;
    g.A = ix->A; g.bproj = ix->bproj; g.keys = ix->keys; g.pos = ix->pos; g.root = ix->root; g.leaf = ix->leaf;
    g.X_hi = ix->X_hi; g.X_lo = ix->X_lo; g.row_of = ix->row_of; g.X_h16 = ix->X_h16;
    int64_t max_nc = 0;
    for (int j = 0; j < ncl; ++j) max_nc = std::max(max_nc, ix->h_cl_off[j + 1] - ix->h_cl_off[j]);
    g.max_row_tiles = (int32_t)cdiv(max_nc, 256);
    {
        std::vector<int64_t> wv(ncl);
        for (int j = 0; j < ncl; ++j) wv[j] = cdiv(ix->h_cl_off[j + 1] - ix->h_cl_off[j], 32);
        std::sort(wv.begin(), wv.end(), std::greater<int64_t>());
        ix->top_words.assign(ncl + 1, 0);
        for (int j = 0; j < ncl; ++j) ix->top_words[j + 1] = ix->top_words[j] + wv[j];
    }
#undef ALLOC
    {
        // a pass's scratch stays within 48 GiB and 3/4 of the device memory
        // left free once the index is built
        size_t free_b = 0, total_b = 0;
        LIDER_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        ix->pass_budget = std::min<size_t>((size_t)48 << 30, free_b / 4 * 3);
    }
    LIDER_CUDA_TRY(cudaStreamCreateWithFlags(&ix->side, cudaStreamNonBlocking));
    ix->build_ms = std::chrono::duration<double, std::milli>(clock::now() - t_start).count();
    guard.ix = nullptr;
    *out = ix;
    return LIDER_OK;
}

}  // namespace

void destroy_index(lider_index* ix) { release(ix); }

int build_entry(const float* corpus, int64_t n, int32_t d, const float* centroids, int32_t ncl,
                const lider_cluster_params* cp, const float* A, const float* b, const lider_params* P, void* stream,
                lider_index** out) {
    return build_impl(corpus, n, d, centroids, ncl, cp, A, b, P, (cudaStream_t)stream, out);
}

}  // namespace lider
