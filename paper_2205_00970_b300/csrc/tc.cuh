// 5th-generation tensor-core (tcgen05) tile engine for sm_103a: TMA loads into
// 128-byte-swizzled shared memory, tcgen05.mma with the accumulator in TMEM,
// tcgen05.ld for the epilogue.  Used for the dense part of candidate scoring:
// D[128 x 256] = A[128 x d] . B[256 x d]^T in one of two kinds:
//   KindTf32x3: FP32 accuracy from three TF32 products (A_hi B_hi + A_hi B_lo +
//     A_lo B_hi; x = x_hi + x_lo with x_hi the TF32-representable head of x,
//     so the dropped A_lo B_lo term and the TF32 rounding of x_lo stay below
//     2^-21 relative); two stages of A_hi, A_lo, B_hi, B_lo;
//   KindBf16: one BF16 product per element pair (kind::f16, FP32
//     accumulation); four stages of A, B.
// Every shared-memory row is 128 bytes (32 FP32 or 64 BF16 elements of K) and
// every MMA consumes 32 bytes of K, four MMA steps per stage.
//
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lider {
namespace tc {

constexpr int kBM = 128;                       // MMA M = TMEM lanes
constexpr int kBN = 256;                       // MMA N = accumulator columns
constexpr int kRowBytes = 128;                 // K bytes per shared-memory row (one swizzle span)
constexpr int kTileA = kBM * kRowBytes;        // 16 KB
constexpr int kTileB = kBN * kRowBytes;        // 32 KB
constexpr int kMaxStages = 4;
constexpr int kSmemBytes = 2 * (2 * kTileA + 2 * kTileB) + 1024;  // both kinds: 192 KB + alignment slack
constexpr int kThreads = 192;       // producer + MMA warps + 4 epilogue warps
// threads of a block with kEpiWarps epilogue warps (4, 8 or 16)
constexpr int threads_for(int epi_warps) { return 64 + 32 * epi_warps; }
constexpr int kTmemCols = 2 * kBN;
constexpr uint64_t kTimeoutNs = 2000000000ull;

// instruction descriptors: D F32 (bits 4-5 = 1), A and B formats at bits 7-9
// and 10-12 (kind::tf32: 2 = TF32; kind::f16: 1 = BF16), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t idesc(uint32_t ab_format) {
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(kBN >> 3) << 17) |
           ((uint32_t)(kBM >> 4) << 24);
}

struct KindTf32x3 {
    static constexpr int kStages = 2;
    static constexpr int kOps = 2;                       // hi and lo buffers per operand
    static constexpr int kElemBytes = 4;
    static constexpr int kBK = kRowBytes / kElemBytes;   // 32 elements of K per stage
    static constexpr uint32_t kIdesc = idesc(2);
    static constexpr bool kF8 = false;
};

struct KindBf16 {
    static constexpr int kStages = 4;
    static constexpr int kOps = 1;
    static constexpr int kElemBytes = 2;
    static constexpr int kBK = kRowBytes / kElemBytes;   // 64 elements of K per stage
    static constexpr uint32_t kIdesc = idesc(1);
    static constexpr bool kF8 = false;
};

// FP8 e4m3 operands (kind::f8f6f4; a/b format code 0 = E4M3), 128 elements of
// K per 128-byte row, 32 per MMA (32 bytes, as the 16-bit kinds).
struct KindF8 {
    static constexpr int kStages = 4;
    static constexpr int kOps = 1;
    static constexpr int kElemBytes = 1;
    static constexpr int kBK = kRowBytes / kElemBytes;   // 128 elements of K per stage
    static constexpr uint32_t kIdesc = idesc(0);
    static constexpr bool kF8 = true;
};

struct KindF16 {
    static constexpr int kStages = 4;
    static constexpr int kOps = 1;
    static constexpr int kElemBytes = 2;
    static constexpr int kBK = kRowBytes / kElemBytes;   // 64 elements of K per stage
    static constexpr uint32_t kIdesc = idesc(0);
    static constexpr bool kF8 = false;
};

template <class Kind>
__host__ __device__ constexpr bool is_f8() {
    return Kind::kF8;
}

enum {
    TC_OK = 0,
    TC_TIMEOUT_EMPTY = 1,
    TC_TIMEOUT_FULL = 2,
    TC_TIMEOUT_TFULL = 3,
    TC_TIMEOUT_TEMPTY = 4,
    TC_TIMEOUT_DRAIN = 5,
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `parity` to complete; false on timeout (after
// timeout_ns) or abort.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          uint64_t timeout_ns = kTimeoutNs) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > timeout_ns) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every MMA issued so far by this thread has completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor for a K-major operand stored as rows of 128
// bytes with the 128-byte swizzle (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_128B): start address >> 4 in bits 0-13, leading byte
// offset (unused for this layout, 16 B) >> 4 at bit 16, stride byte offset
// between 8-row groups (1024 B) >> 4 at bit 32, descriptor version 1 at bit 46,
// layout type 2 (128-byte swizzle) at bit 61.  The tile base must be
// 1024-byte aligned; a K offset inside the 128-byte row is added to the start.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Shared state of one block.
struct Ctl {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint32_t tmem_base;
    int abort;
};

// Test hook of the bounded waits (engine self-test only): every wait gives up
// after timeout_ns, and with skip_first the producer leaves the first stage
// of the first tile unloaded, so the MMA warp's wait for it runs out.
struct WaitTest {
    uint64_t timeout_ns = kTimeoutNs;
    bool skip_first = false;
};

// One unit = one 128 x 256 tile: A rows [a_row, a_row+128), B rows
// [b_row, b_row+256), all of K.  Sched provides: int count() and
// void coords(int u, int& a_row, int& b_row).  Epi provides, called by every
// epilogue thread (row = its accumulator row, all 32 lanes of a warp
// together): void begin(int u, int row) before the tile's accumulator is
// waited for (it must not read TMEM; its loads overlap the tile's MMAs),
// void operator()(int u, int row, int col0, const uint32_t (&v)[32]) for
// columns col0..col0+31, and void done(int u, int row) after the last group.
// Each epilogue warp leaves its loop as a whole warp (Epi must not use
// barriers across warps); the warps of a tile need not run in step.
// mA0/mB0: the operands (KindTf32x3: their TF32 heads); mA1/mB1: the tails
// (KindTf32x3 only; ignored otherwise).  kchunks = ceil(d / Kind::kBK).
// kStagesUse: shared-memory stages of K (at most Kind::kStages, the plan the
// block's shared memory is sized for; a kernel with a larger epilogue can use
// fewer).
template <class Kind, class Sched, class Epi, int kEpiWarps = 4, int kStagesUse = Kind::kStages>
__device__ void gemm_tiles(const CUtensorMap* mAhi, const CUtensorMap* mAlo, const CUtensorMap* mBhi,
                           const CUtensorMap* mBlo, int kchunks, Sched& sched, Epi& epi, int* err,
                           unsigned char* smem_raw, Ctl& ctl, const WaitTest wt = WaitTest{}) {
    const uint64_t tmo = wt.timeout_ns;
    static_assert(kStagesUse >= 2 && kStagesUse <= Kind::kStages, "stages");
    constexpr int kStages = kStagesUse;
    constexpr int kStageBytes = Kind::kOps * (kTileA + kTileB);
    constexpr int kBK = Kind::kBK;
    static_assert(kStages * kStageBytes + 1024 <= kSmemBytes, "stages exceed the shared memory plan");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~(uintptr_t)1023);
    auto stage_ptr = [&](int s) { return smem + (size_t)s * kStageBytes; };
    volatile int* abort_flag = &ctl.abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&ctl.full[s], 1);
            mbar_init(&ctl.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&ctl.tfull[b], 1);
            mbar_init(&ctl.tempty[b], kEpiWarps);
        }
        ctl.abort = 0;
        fence_mbar_init();
    }
    if (warp == 0) {
        tmem_alloc(&ctl.tmem_base, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = ctl.tmem_base;
    const int nunits = sched.count();
    auto fail = [&](int code) {
        atomicCAS(err, 0, code);
        *abort_flag = 1;
    };

    if (warp == 0) {
        if (lane == 0) {                                         // TMA producer
            int it = 0;
            for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x) {
                int arow, brow;
                sched.coords(u, arow, brow);
                for (int kc = 0; kc < kchunks; ++kc, ++it) {
                    const int s = it % kStages;
                    const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                    if (!mbar_wait(&ctl.empty[s], ph ^ 1u, abort_flag, tmo)) { fail(TC_TIMEOUT_EMPTY); break; }
                    if (wt.skip_first && it == 0) continue;      // test hook: this stage never fills
                    unsigned char* st = stage_ptr(s);
                    mbar_expect_tx(&ctl.full[s], (uint32_t)kStageBytes);
                    const int k0 = kc * kBK;
                    tma_load_2d(st, mAhi, &ctl.full[s], k0, arow);
                    tma_load_2d(st + Kind::kOps * kTileA, mBhi, &ctl.full[s], k0, brow);
                    if constexpr (Kind::kOps == 2) {
                        tma_load_2d(st + kTileA, mAlo, &ctl.full[s], k0, arow);
                        tma_load_2d(st + 2 * kTileA + kTileB, mBlo, &ctl.full[s], k0, brow);
                    }
                }
            }
            // drain: wait until every issued stage has landed (bounded)
            const int issued = it;
            for (int j = (issued > kStages ? issued - kStages : 0); j < issued; ++j) {
                if (wt.skip_first && j == 0) continue;           // never issued
                const int s = j % kStages;
                const uint32_t ph = (uint32_t)(j / kStages) & 1u;
                const uint64_t t0 = globaltimer();
                while (!mbar_try(&ctl.full[s], ph)) {
                    if (globaltimer() - t0 > tmo) { atomicCAS(err, 0, TC_TIMEOUT_DRAIN); break; }
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {                                         // MMA issuer
            int it = 0, ui = 0;
            for (int u = blockIdx.x; u < nunits && !*abort_flag; u += gridDim.x, ++ui) {
                const int ab = ui & 1;
                const uint32_t aph = (uint32_t)(ui >> 1) & 1u;
                if (!mbar_wait(&ctl.tempty[ab], aph ^ 1u, abort_flag, tmo)) { fail(TC_TIMEOUT_TEMPTY); break; }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(ab * kBN);
                bool ok = true;
                for (int kc = 0; kc < kchunks; ++kc, ++it) {
                    const int s = it % kStages;
                    const uint32_t ph = (uint32_t)(it / kStages) & 1u;
                    if (!mbar_wait(&ctl.full[s], ph, abort_flag, tmo)) { fail(TC_TIMEOUT_FULL); ok = false; break; }
                    tc_fence_after();
                    const uint32_t sa = smem_u32(stage_ptr(s));
#pragma unroll
                    for (int kk = 0; kk < kRowBytes / 32; ++kk) {     // 32 bytes of K per MMA
                        const uint32_t off = (uint32_t)kk * 32u;
                        const uint32_t acc = (kc | kk) != 0 ? 1u : 0u;
                        if constexpr (Kind::kOps == 2) {
                            const uint32_t a_hi = sa, a_lo = sa + kTileA;
                            const uint32_t b_hi = sa + 2 * kTileA, b_lo = sa + 2 * kTileA + kTileB;
                            const uint64_t dah = sdesc_sw128(a_hi + off), dal = sdesc_sw128(a_lo + off);
                            const uint64_t dbh = sdesc_sw128(b_hi + off), dbl = sdesc_sw128(b_lo + off);
                            mma_tf32(d, dah, dbh, Kind::kIdesc, acc);
                            mma_tf32(d, dah, dbl, Kind::kIdesc, 1u);
                            mma_tf32(d, dal, dbh, Kind::kIdesc, 1u);
                        } else {
                            const uint64_t da = sdesc_sw128(sa + off), db = sdesc_sw128(sa + kTileA + off);
                            if constexpr (is_f8<Kind>()) mma_f8(d, da, db, Kind::kIdesc, acc);
                            else mma_f16(d, da, db, Kind::kIdesc, acc);
                        }
                    }
                    mma_commit(&ctl.empty[s]);                 // stage reusable once these finish
                }
                if (!ok) break;
                mma_commit(&ctl.tfull[ab]);                    // accumulator ready
            }
        }
    } else {                                                     // epilogue warps 2..
        // warp w reads TMEM lanes 32 (w % 4) ..; with more than 4 epilogue
        // warps, kEpiWarps / 4 of them share those lanes and split the 8
        // column groups (contiguous runs of kGroups, the last run shorter)
        static_assert(kEpiWarps % 4 == 0 && kEpiWarps >= 4 && kEpiWarps <= 32, "a multiple of 4 epilogue warps");
        constexpr int kWpq = kEpiWarps / 4;
        constexpr int kGroups = ((kBN / 32) + kWpq - 1) / kWpq;
        const int quarter = warp & 3;
        const int cb0 = ((warp - 2) >> 2) * kGroups;
        const int row = quarter * 32 + lane;
        int ui = 0;
        for (int u = blockIdx.x; u < nunits; u += gridDim.x, ++ui) {
            const int ab = ui & 1;
            const uint32_t aph = (uint32_t)(ui >> 1) & 1u;
            epi.begin(u, row);
            // the warp leaves as one (a timed-out wait on any lane), so its
            // .sync.aligned TMEM loads never see a partial warp; the other
            // warps' waits end by the abort flag or their own limit
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&ctl.tfull[ab], aph, abort_flag, tmo));
            if (!ok) {
                if (lane == 0) fail(TC_TIMEOUT_TFULL);
                break;
            }
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(ab * kBN);
#pragma unroll
            for (int g = 0; g < kGroups; ++g) {
                const int cb = cb0 + g;
                if (cb >= kBN / 32) break;               // the same in every lane
                uint32_t v[32];
                tmem_ld32(base + (uint32_t)(cb * 32), v);
                epi(u, row, cb * 32, v);
            }
            epi.done(u, row);
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl.tempty[ab]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kTmemCols);
}

}  // namespace tc
}  // namespace lider
