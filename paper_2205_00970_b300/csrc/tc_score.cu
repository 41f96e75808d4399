// Tensor-core candidate scoring support: the TF32 hi/lo split, TMA tensor
// maps, and a one-tile self-test of the tcgen05 engine (tc.cuh).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cmath>

#include <mutex>

#include "lider_internal.cuh"
#include "tc.cuh"

namespace lider {

namespace {

// x = hi + lo exactly: hi keeps sign, exponent and the top 10 mantissa bits
// (a TF32 value), lo = x - hi is exact in FP32.
__global__ void split_tf32_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ hi,
                                  float* __restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = x[i];
    const float h = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    hi[i] = h;
    lo[i] = __fsub_rn(v, h);
}

// Round scale * x to FP16 (nearest, ties to even); scale is a power of two,
// so the scaling itself is exact.
__global__ void to_f16_kernel(const float* __restrict__ x, int64_t n, float scale, uint16_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __half_as_ushort(__float2half_rn(x[i] * scale));
}

// FP8 e4m3 with one scale per row: s = max|x_row| / 448 (1 for a zero row),
// out = e4m3(x / s) (nearest, saturating to the finite range), so x ~ s * out.
// Warp per row.
__global__ void to_f8_rows_kernel(const float* __restrict__ x, int64_t n, int d, float* __restrict__ scale,
                                  uint8_t* __restrict__ out) {
    const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (row >= n) return;
    const float* xr = x + row * d;
    float amax = 0.f;
    for (int i = lane; i < d; i += 32) amax = fmaxf(amax, fabsf(xr[i]));
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const float inv = amax > 0.f ? 448.f / amax : 1.f;
    if (lane == 0) scale[row] = amax > 0.f ? amax / 448.f : 1.f;
    for (int i = lane; i < d; i += 32)
        out[row * d + i] = (uint8_t)__nv_cvt_float_to_fp8(xr[i] * inv, __NV_SATFINITE, __NV_E4M3);
}

// FP8 e4m3 without scaling (engine self-test).
__global__ void to_f8_kernel(const float* __restrict__ x, int64_t n, uint8_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = (uint8_t)__nv_cvt_float_to_fp8(x[i], __NV_SATFINITE, __NV_E4M3);
}

// Round to BF16 (nearest, ties to even).
__global__ void to_bf16_kernel(const float* __restrict__ x, int64_t n, uint16_t* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = __bfloat16_as_ushort(__float2bfloat16_rn(x[i]));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

int encode_fn(EncodeTiledFn* fn) {
    std::call_once(g_encode_once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (EncodeTiledFn)p;
        cudaGetLastError();
    });
    if (!g_encode) return fail(LIDER_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    *fn = g_encode;
    return LIDER_OK;
}

struct OneTile {
    __device__ int count() const { return 1; }
    __device__ void coords(int, int& a, int& b) const { a = 0; b = 0; }
};

struct WriteTile {
    float* out;
    int m, n;
    __device__ void operator()(int, int row, int col0, const uint32_t (&v)[32]) const {
        if (row >= m) return;
#pragma unroll
        for (int i = 0; i < 32; ++i)
            if (col0 + i < n) out[(int64_t)row * n + col0 + i] = __uint_as_float(v[i]);
    }
    __device__ void begin(int, int) const {}
    __device__ void done(int, int) const {}
};

template <class Kind>
__global__ void __launch_bounds__(tc::kThreads, 1)
    tc_tile_test_kernel(const __grid_constant__ CUtensorMap mAhi, const __grid_constant__ CUtensorMap mAlo,
                        const __grid_constant__ CUtensorMap mBhi, const __grid_constant__ CUtensorMap mBlo,
                        int kchunks, float* out, int m, int n, int* err, tc::WaitTest wt) {
    extern __shared__ unsigned char smem[];
    __shared__ tc::Ctl ctl;
    OneTile sched;
    WriteTile epi{out, m, n};
    tc::gemm_tiles<Kind>(&mAhi, &mAlo, &mBhi, &mBlo, kchunks, sched, epi, err, smem, ctl, wt);
}

}  // namespace

int launch_to_bf16(const float* x, int64_t n, uint16_t* out, cudaStream_t st) {
    if (n <= 0) return LIDER_OK;
    to_bf16_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(x, n, out);
    LIDER_LAUNCH_CHECK("to_bf16_kernel");
    return LIDER_OK;
}

int launch_to_f16(const float* x, int64_t n, float scale, uint16_t* out, cudaStream_t st) {
    if (n <= 0) return LIDER_OK;
    to_f16_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(x, n, scale, out);
    LIDER_LAUNCH_CHECK("to_f16_kernel");
    return LIDER_OK;
}

int launch_to_f8_rows(const float* x, int64_t n, int d, float* scale, uint8_t* out, cudaStream_t st) {
    if (n <= 0) return LIDER_OK;
    to_f8_rows_kernel<<<(unsigned)cdiv(n * 32, 256), 256, 0, st>>>(x, n, d, scale, out);
    LIDER_LAUNCH_CHECK("to_f8_rows_kernel");
    return LIDER_OK;
}

float f16_scale_host(float amax) {
    if (!(amax > 0.f) || !std::isfinite(amax)) return 1.f;
    int e = 0;
    std::frexp(amax, &e);                 // amax in [2^(e-1), 2^e)
    e = std::max(-100, std::min(e, 127));
    return std::ldexp(1.f, 14 - e);       // scaled max in [2^13, 2^14)
}

int launch_split_tf32(const float* x, int64_t n, float* hi, float* lo, cudaStream_t st) {
    if (n <= 0) return LIDER_OK;
    split_tf32_kernel<<<(unsigned)cdiv(n, 256), 256, 0, st>>>(x, n, hi, lo);
    LIDER_LAUNCH_CHECK("split_tf32_kernel");
    return LIDER_OK;
}

// 2-D tensor map over rows x d (row-major FP32, or BF16 when bf16), box of
// one 128-byte row of K (32 FP32 / 64 BF16) x box_rows, 128-byte swizzle.
// The same over 1-byte elements (FP8): box of one 128-byte row of K (128 elements).
int make_tensor_map8(CUtensorMap* map, const void* base, int64_t rows, int d, int box_rows) {
    EncodeTiledFn fn;
    int rc = encode_fn(&fn);
    if (rc) return rc;
    const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)d};
    const cuuint32_t box[2] = {(cuuint32_t)tc::kRowBytes, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void*)base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LIDER_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return LIDER_OK;
}

int make_tensor_map(CUtensorMap* map, const void* base, int64_t rows, int d, int box_rows, bool bf16) {
    EncodeTiledFn fn;
    int rc = encode_fn(&fn);
    if (rc) return rc;
    const int esz = bf16 ? 2 : 4;
    const cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)d * esz};
    const cuuint32_t box[2] = {(cuuint32_t)(tc::kRowBytes / esz), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                          (void*)base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LIDER_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return LIDER_OK;
}

}  // namespace lider

namespace lider {
namespace {

// Self-test of the tensor-core engine: out[m x n] = A[m x d] . B[n x d]^T with
// m <= 128, n <= 256, through the same TMA / tcgen05 / TMEM path as search;
// wt: the waits' limit and the test hook that leaves one stage unloaded.
int tc_tile_impl(const float* A, int32_t m, const float* B, int32_t n, int32_t d, int32_t kind, float* out,
                 tc::WaitTest wt, void* stream) {
    try {
        if (!A || !B || !out) return fail(LIDER_EINVAL, "lider_debug_tc_tile: NULL pointer");
        if (kind < 0 || kind > 3) return fail(LIDER_EINVAL, "lider_debug_tc_tile: kind must be 0, 1, 2 or 3");
        const int dmul = kind == 0 ? 4 : kind == 3 ? 16 : 8;
        if (m < 1 || m > tc::kBM || n < 1 || n > tc::kBN || d < dmul || d % dmul != 0)
            return fail(LIDER_EINVAL, "lider_debug_tc_tile: need 1<=m<=128, 1<=n<=256, d % 4 (16-bit: 8, FP8: 16) == 0");
        cudaStream_t st = (cudaStream_t)stream;
        float* buf = nullptr;
        const size_t na = (size_t)m * d, nb = (size_t)n * d;
        LIDER_CUDA_TRY(cudaMalloc(&buf, (2 * na + 2 * nb) * sizeof(float) + 64 * sizeof(int)));
        float *ahi = buf, *alo = buf + na, *bhi = buf + 2 * na, *blo = buf + 2 * na + nb;
        int* err = reinterpret_cast<int*>(buf + 2 * na + 2 * nb);
        int rc = LIDER_OK;
        CUtensorMap mah, mal, mbh, mbl;
        do {
            if (kind == 0) {
                if ((rc = launch_split_tf32(A, (int64_t)na, ahi, alo, st))) break;
                if ((rc = launch_split_tf32(B, (int64_t)nb, bhi, blo, st))) break;
                if ((rc = make_tensor_map(&mah, ahi, m, d, tc::kBM))) break;
                if ((rc = make_tensor_map(&mal, alo, m, d, tc::kBM))) break;
                if ((rc = make_tensor_map(&mbh, bhi, n, d, tc::kBN))) break;
                if ((rc = make_tensor_map(&mbl, blo, n, d, tc::kBN))) break;
            } else if (kind == 3) {
                uint8_t* a8 = reinterpret_cast<uint8_t*>(ahi);
                uint8_t* b8 = reinterpret_cast<uint8_t*>(bhi);
                to_f8_kernel<<<(unsigned)cdiv((int64_t)na, 256), 256, 0, st>>>(A, (int64_t)na, a8);
                to_f8_kernel<<<(unsigned)cdiv((int64_t)nb, 256), 256, 0, st>>>(B, (int64_t)nb, b8);
                if ((rc = make_tensor_map8(&mah, a8, m, d, tc::kBM))) break;
                if ((rc = make_tensor_map8(&mbh, b8, n, d, tc::kBN))) break;
                mal = mah;
                mbl = mbh;
            } else {
                uint16_t* a16 = reinterpret_cast<uint16_t*>(ahi);
                uint16_t* b16 = reinterpret_cast<uint16_t*>(bhi);
                if (kind == 1) {
                    if ((rc = launch_to_bf16(A, (int64_t)na, a16, st))) break;
                    if ((rc = launch_to_bf16(B, (int64_t)nb, b16, st))) break;
                } else {
                    if ((rc = launch_to_f16(A, (int64_t)na, 1.f, a16, st))) break;
                    if ((rc = launch_to_f16(B, (int64_t)nb, 1.f, b16, st))) break;
                }
                if ((rc = make_tensor_map(&mah, a16, m, d, tc::kBM, true))) break;
                if ((rc = make_tensor_map(&mbh, b16, n, d, tc::kBN, true))) break;
                mal = mah;
                mbl = mbh;
            }
            cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
            const void* kern = kind == 0   ? (const void*)tc_tile_test_kernel<tc::KindTf32x3>
                               : kind == 1 ? (const void*)tc_tile_test_kernel<tc::KindBf16>
                               : kind == 2 ? (const void*)tc_tile_test_kernel<tc::KindF16>
                                           : (const void*)tc_tile_test_kernel<tc::KindF8>;
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemBytes);
            if (e != cudaSuccess) { rc = cuda_fail(e, "cudaFuncSetAttribute"); break; }
            const int kbk = kind == 0 ? tc::KindTf32x3::kBK : kind == 3 ? tc::KindF8::kBK : tc::KindBf16::kBK;
            int kchunks = (d + kbk - 1) / kbk;
            void* args[] = {&mah, &mal, &mbh, &mbl, &kchunks, &out, &m, &n, &err, &wt};
            e = cudaLaunchKernel(kern, dim3(1), dim3(tc::kThreads), args, tc::kSmemBytes, st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "tc_tile_test_kernel launch"); break; }
            e = cudaGetLastError();
            if (e != cudaSuccess) { rc = cuda_fail(e, "tc_tile_test_kernel"); break; }
            int h_err = 0;
            e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "tc_tile_test_kernel sync"); break; }
            if (h_err) rc = fail(LIDER_ECUDA, "tc engine wait timed out (code " + std::to_string(h_err) + ")");
        } while (0);
        cudaFree(buf);
        return rc;
    } catch (...) {
        return fail(LIDER_ECUDA, "lider_debug_tc_tile: internal error");
    }
}

}  // namespace
}  // namespace lider

extern "C" int lider_debug_tc_tile(const float* A, int32_t m, const float* B, int32_t n, int32_t d, int32_t kind,
                                   float* out, void* stream) {
    return lider::tc_tile_impl(A, m, B, n, d, kind, out, lider::tc::WaitTest{}, stream);
}

extern "C" int lider_debug_tc_wait_expiry(const float* A, int32_t m, const float* B, int32_t n, int32_t d,
                                          int32_t kind, float* out, double limit_ms, void* stream) {
    if (!(limit_ms > 0.0) || limit_ms > 10000.0)
        return lider::fail(LIDER_EINVAL, "lider_debug_tc_wait_expiry: limit_ms must be in (0, 10000]");
    lider::tc::WaitTest wt;
    wt.timeout_ns = (uint64_t)(limit_ms * 1e6);
    wt.skip_first = true;
    return lider::tc_tile_impl(A, m, B, n, d, kind, out, wt, stream);
}
