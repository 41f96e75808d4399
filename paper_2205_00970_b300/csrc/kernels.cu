// Dense kernels shared by build and search: compensated (Dot2) tiled products
// for the LSH projections (Sec. 4.1) and the centroid scores (Sec. 3.2), and
// the packing of hash values into SK-LSH sortable keys (Sec. 4.2).
//
// Precision: hash values and cluster choices are integer decisions taken from
// floating point, and they must agree with an FP64 evaluation except within
// 1e-6 W of a bucket edge.  A plain FP32 dot of length 768 can be off by
// ~1e-5 there, so the products are accumulated with Dot2 (about 2x FP32
// precision) and finished in FP64.  This is SIMT FP32 work, not tensor-core
// work: tensor-core formats cannot carry that precision.
#include "lider_internal.cuh"

namespace lider {

namespace {

constexpr int TM = 64;   // rows of X per block
constexpr int TN = 64;   // rows of Y per block
constexpr int TK = 32;   // depth per shared-memory stage

enum { EPI_HASH = 0, EPI_SCORE = 1 };

// out[i][j] = epilogue(sum_k X[i][k] * Y[j][k]) over a TM x TN tile.
// Thread (tx, ty) owns rows ty + 16 a and columns tx + 16 b (a, b < 4).
template <int EPI>
__global__ void __launch_bounds__(256) dot2_tile_kernel(
        const float* __restrict__ X, int64_t n, int d,
        const float* __restrict__ Y, int ny,
        const float* __restrict__ bvec, double W,
        const double* __restrict__ half_norm,
        double* __restrict__ out) {
    __shared__ float Xs[TK][TM + 1];
    __shared__ float Ys[TK][TN + 1];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t row0 = (int64_t)blockIdx.x * TM;
    const int col0 = blockIdx.y * TN;

    Dot2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = Dot2{0.f, 0.f};

    for (int k0 = 0; k0 < d; k0 += TK) {
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int idx = tid + it * 256;          // 0..511: 64 rows x 8 float4
            const int r = idx >> 3, kq = (idx & 7) * 4;
            float4 vx = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 vy = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row0 + r < n && k0 + kq < d)
                vx = *reinterpret_cast<const float4*>(X + (row0 + r) * (int64_t)d + k0 + kq);
            if (col0 + r < ny && k0 + kq < d)
                vy = *reinterpret_cast<const float4*>(Y + (int64_t)(col0 + r) * d + k0 + kq);
            Xs[kq + 0][r] = vx.x; Xs[kq + 1][r] = vx.y; Xs[kq + 2][r] = vx.z; Xs[kq + 3][r] = vx.w;
            Ys[kq + 0][r] = vy.x; Ys[kq + 1][r] = vy.y; Ys[kq + 2][r] = vy.z; Ys[kq + 3][r] = vy.w;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < TK; ++kk) {
            float xa[4], yb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = Xs[kk][ty + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) yb[b] = Ys[kk][tx + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) dot2_step(acc[a][b], xa[a], yb[b]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t row = row0 + ty + 16 * a;
        if (row >= n) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int col = col0 + tx + 16 * b;
            if (col >= ny) continue;
            const double dot = dot2_value(acc[a][b]);
            double v;
            if (EPI == EPI_HASH)
                v = __ddiv_rn(__dadd_rn(dot, (double)bvec[col]), W);   // t = (a.x + b) / W
            else
                v = __dadd_rn(dot, -half_norm[col]);                   // x.mu - |mu|^2 / 2
            out[row * ny + col] = v;
        }
    }
}

// Pack the m hash values of (row, array l) into one key (Sec. 4.2 linear
// order; reading R2 for the element width) and count boundary/clamped values.
// p-stable: element floor(t) + 2^(beta-1), clamped; boundary when t lies
// within 1e-6 of an integer.  Hyperplane (t = a.x): element [t >= 0], one
// bit; boundary when |t| < 1e-6.
__global__ void pack_kernel(const double* __restrict__ t, int64_t n, int L, int m, int beta, int hash_kind,
                            int64_t row_offset, int64_t stride_row, int64_t stride_arr,
                            uint64_t* __restrict__ keys,
                            unsigned long long* n_boundary, unsigned long long* n_clamped) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned nb = 0, nc = 0;
    if (gid < n * L) {
        const int64_t row = gid / L;
        const int l = (int)(gid % L);
        const double* tr = t + row * (int64_t)(L * m) + (int64_t)l * m;
        const int64_t off = 1ll << (beta - 1);
        const int64_t vmax = (beta >= 63) ? INT64_MAX : ((1ll << beta) - 1);
        uint64_t key = 0;
        if (hash_kind == LIDER_HASH_HYPERPLANE) {
            for (int j = 0; j < m; ++j) {
                const double tj = tr[j];
                if (fabs(tj) < 1e-6) ++nb;
                key |= (uint64_t)(tj >= 0.0 ? 1u : 0u) << (m - 1 - j);
            }
            keys[(row_offset + row) * stride_row + (int64_t)l * stride_arr] = key;
        } else {
            for (int j = 0; j < m; ++j) {
                const double tj = tr[j];
                if (fabs(__dadd_rn(tj, -rint(tj))) < 1e-6) ++nb;
                double fl = floor(tj);
                fl = fmin(fmax(fl, -4.0e18), 4.0e18);
                int64_t v = (int64_t)fl + off;
                if (v < 0) { v = 0; ++nc; }
                if (v > vmax) { v = vmax; ++nc; }
                key |= (uint64_t)v << (beta * (m - 1 - j));
            }
            keys[(row_offset + row) * stride_row + (int64_t)l * stride_arr] = key;
        }
    }
    // warp-aggregated counters
    for (int o = 16; o > 0; o >>= 1) {
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
        nc += __shfl_xor_sync(0xffffffffu, nc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nb && n_boundary) atomicAdd(n_boundary, (unsigned long long)nb);
        if (nc && n_clamped) atomicAdd(n_clamped, (unsigned long long)nc);
    }
}

}  // namespace

int launch_hash_t(const float* X, int64_t n, int d, const float* A, const float* b, int H,
                  double W, double* t_out, cudaStream_t s) {
    if (n <= 0) return LIDER_OK;
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(H, TN));
    dot2_tile_kernel<EPI_HASH><<<grid, 256, 0, s>>>(X, n, d, A, H, b, W, nullptr, t_out);
    LIDER_LAUNCH_CHECK("dot2_tile_kernel<hash>");
    return LIDER_OK;
}

int launch_scores(const float* X, int64_t n, int d, const float* C, const double* half_norm,
                  int ncl, double* out, cudaStream_t s) {
    if (n <= 0) return LIDER_OK;
    dim3 grid((unsigned)cdiv(n, TM), (unsigned)cdiv(ncl, TN));
    dot2_tile_kernel<EPI_SCORE><<<grid, 256, 0, s>>>(X, n, d, C, ncl, nullptr, 1.0, half_norm, out);
    LIDER_LAUNCH_CHECK("dot2_tile_kernel<score>");
    return LIDER_OK;
}

int launch_pack(const double* t, int64_t n, int L, int m, int beta, int hash_kind, int64_t row_offset,
                int64_t stride_row, int64_t stride_arr, uint64_t* keys,
                unsigned long long* n_boundary, unsigned long long* n_clamped, cudaStream_t s) {
    if (n <= 0) return LIDER_OK;
    const int64_t total = n * L;
    pack_kernel<<<(unsigned)cdiv(total, 256), 256, 0, s>>>(t, n, L, m, beta, hash_kind, row_offset, stride_row,
                                                         stride_arr, keys, n_boundary, n_clamped);
    LIDER_LAUNCH_CHECK("pack_kernel");
    return LIDER_OK;
}

}  // namespace lider
