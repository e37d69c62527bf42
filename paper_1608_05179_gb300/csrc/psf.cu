// PSF matrix (§3 Eq. (10), arranged as A of Eq. (12)) on the 5th-generation
// tensor cores: the complex Gram product
//     G[n][s] = sum_m conj(L[n][m]) * R[s][m],   A[n][s] = scale * |G[n][s]|^2,
// diagonal stored as exactly 1, columns S..lda-1 zero.
//
// Real form: with L = Lr + i Li and R = Rr + i Ri,
//     Re G = Lr.Rr + Li.Ri,     Im G = Lr.Ri - Li.Rr,
// four real products over the microphones, each a K-major contraction.  FP32
// accuracy from TF32 tensor cores by the three-term split ("3xTF32"):
// x = x_hi + x_lo with x_hi = tf32(x), x_lo = tf32(x - x_hi), and
//     a.b ~ a_hi.b_hi + a_hi.b_lo + a_lo.b_hi     (dropped a_lo.b_lo ~ 2^-22 |a.b|),
// every product exact in FP32 and accumulated in FP32 in tensor memory.
//
// Two kernels.  psf_split_kernel turns the FP32 vector planes into operand
// planes H (hi) and Lo (lo), one row per point, laid out per chunk of 16
// microphones as [16 real parts | 16 imaginary parts] (128 bytes).
// psf_gram_tc_kernel is persistent and warp specialised, one CTA per SM over a
// list of 128 x 128 tiles of A (rows n, columns s):
//   TMA thread (warp 9)    loads the chunk's four operand boxes (A hi/lo, B
//                          hi/lo: 128 rows each; 128-byte swizzle) into a
//                          three-stage ring                   -> full[st]
//   MMA thread (warp 8)    24 tcgen05.mma.cta_group::1.kind::tf32 per chunk
//                          (M = 128, N = 128, K = 8; 3 split terms x 2 K slices
//                          x {Re G += Lr.Rr, Re G += Li.Ri, Im G += Lr.Ri,
//                          Im G -= Li.Rr via the negate-A bit}), accumulators
//                          Re G and Im G in 256 TMEM columns  -> empty[st];
//                          after a tile's last chunk            -> acc_full[a]
//   epilogue (warps 0-7)   waits acc_full[a], reads the accumulators 32 columns
//                          at a time with tcgen05.ld (thread = tile row),
//                          writes |G|^2                         -> acc_empty[a]
// TMEM holds two accumulator slots (a = tile parity, 2 x 256 = 512 columns), so
// the epilogue of one tile runs while the MMAs of the next fill the other slot.
// The epilogue writes 32 x 32 blocks.  FP32: the direct block A[n][s] and then
// its mirror A[s][n] as TMA stores of one per-warp staging tile in the tensor
// map's 128-byte swizzle (rows, then columns, of the lanes' values).  BF16: the
// mirror as 128-byte warp stores (lanes hold 32 consecutive n) and the direct
// block through a transpose buffer.  For symmetric A (L and
// R the same vectors, formulation E) only tiles that reach the upper triangle
// run, every value with s >= n is also written mirrored, and A is exactly
// symmetric.  Every wait is bounded by the global timer; a wait that runs out
// sets a CTA-wide abort flag, every role stops waiting, the remaining tiles
// are written as NaN, the operand loads already issued are let land, and the
// launch reports DAMAS_ETIMEDOUT in its status word, so a failure shows
// instead of hanging the device.
//
// Accuracy: FP32 accumulation in the tensor core truncates, so the result
// carries a small bias toward zero that grows with the number of MMAs per
// accumulator (measured against FP64: about -3e-6 relative in A at M = 128,
// -6e-6 at M = 256; max |error| 4e-6 and 8e-6 for entries in [0, 1]).
#include <cuda.h>

#include <mutex>
#include <type_traits>

#include "common.cuh"

namespace {

constexpr int BM = 128;           // tile rows (MMA M)
constexpr int BN = 128;           // tile columns (MMA N)
constexpr int KC = 16;            // complex microphones per chunk
constexpr int KR = 2 * KC;        // real K values per chunk: one 128-byte row
constexpr int A_TILE = BM * KR * 4;              // 16 KB
constexpr int B_TILE = BN * KR * 4;              // 16 KB
constexpr int STAGE = 2 * A_TILE + 2 * B_TILE;   // hi + lo of both operands: 64 KB
constexpr int NSTAGE = 3;
constexpr int EPI_WARPS = 8;                     // warps 0-7: epilogue, two per TMEM lane quarter
constexpr int MMA_WARP = EPI_WARPS;              // warp 8: TMEM owner and MMA issuer
constexpr int TMA_WARP = EPI_WARPS + 1;          // warp 9: operand loads
constexpr int THREADS = 32 * (EPI_WARPS + 2);
constexpr int TP_BYTES = EPI_WARPS * 32 * 32 * 4;  // per-warp 32 x 32 transpose buffers
constexpr int SMEM_BYTES = NSTAGE * STAGE + TP_BYTES;
constexpr int NACC = 2;                           // accumulator slots in TMEM
constexpr uint32_t ACC_COLS = 2 * BN;            // one slot: Re G in [0, BN), Im G in [BN, 2 BN)
constexpr uint32_t TMEM_COLS = NACC * ACC_COLS;  // 512
constexpr int TMA_BOX_ROWS = 128;
static_assert(BM == TMA_BOX_ROWS && BN == TMA_BOX_ROWS, "one TMA box per operand tile");
static_assert(SMEM_BYTES + 1024 <= 232448, "shared memory of one CTA");

// Test hook of the bounded waits: a launch with hold = 1 makes its operand
// loader first wait for this flag, which nothing ever sets, so that wait runs
// out and the launch takes its abort path (no GPU fault involved).
__device__ int psf_hold_flag;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// tcgen05 shared-memory matrix descriptor for a K-major operand with 128-byte
// swizzle: start address (16-byte units), leading offset unused (1), 8-row
// groups 1024 bytes apart, descriptor version 1 (bits 46-47), layout
// SWIZZLE_128B (2 in bits 61-63).  A K slice of 8 TF32 values starts 32 bytes
// further into the swizzled 128-byte row.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

// Instruction descriptor, kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (bits 7-9,
// 10-12 = 2), both K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28; bit 13
// negates A.
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
constexpr uint32_t IDESC_NEG_A = IDESC | (1u << 13);

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t addr, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(addr), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity; false when the deadline passed.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, unsigned long long deadline) {
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 15u) == 15u && now_ns() > deadline) return false;
    }
}

// 2-D TMA load of one box into shared memory, completion counted on mbar.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

template <typename OutT>
__device__ __forceinline__ void put(OutT *p, float v);
template <>
__device__ __forceinline__ void put<float>(float *p, float v) { *p = v; }
template <>
__device__ __forceinline__ void put<__nv_bfloat16>(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }

// Operand planes: H[p][32 c + k] = hi(Re v[p][16 c + k]), H[p][32 c + 16 + k] =
// hi(Im v[p][16 c + k]) for k < 16, and Lo likewise with the low parts.
__global__ void __launch_bounds__(256) psf_split_kernel(const float *__restrict__ Vre, const float *__restrict__ Vim,
                                                         int ldm, int S, float *__restrict__ H,
                                                         float *__restrict__ Lo) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)S * ldm) return;
    const size_t p = i / ldm;
    const int m = (int)(i - p * ldm);
    const float re = Vre[i], im = Vim[i];
    const float hr = to_tf32(re), hi = to_tf32(im);
    const size_t o = p * (size_t)(2 * ldm) + 32 * (m >> 4) + (m & 15);
    H[o] = hr;
    H[o + 16] = hi;
    Lo[o] = to_tf32(re - hr);
    Lo[o + 16] = to_tf32(im - hi);
}

// First column tile of row tile ty that reaches the upper triangle of a
// symmetric A: s0 + BN - 1 >= n0 for s0 = tx BN, n0 = ty BM.
__host__ __device__ __forceinline__ int first_upper_tile(int ty) { return ty * BM / BN; }

// Tile t of the launch's tile list -> (row tile, column tile).  Symmetric A runs
// only the tiles that reach the upper triangle.
__device__ __forceinline__ void tile_coords(int t, int ntx, int symmetric, int &ty, int &tx) {
    if (!symmetric) {
        ty = t / ntx;
        tx = t - ty * ntx;
        return;
    }
    ty = 0;
    for (;;) {
        const int cnt = ntx - first_upper_tile(ty);
        if (t < cnt) break;
        t -= cnt;
        ++ty;
    }
    tx = first_upper_tile(ty) + t;
}

struct GramMaps {
    CUtensorMap a_hi, a_lo, b_hi, b_lo;  // boxes of 32 values x 128 rows, 128-byte swizzle
    CUtensorMap out;                     // A (FP32 output only): boxes of 32 x 32, 128-byte swizzle
};

// 2-D TMA store of one 32 x 32 box from shared memory (bulk group of this thread).
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, uint32_t src, int x, int y) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <typename OutT>
__global__ void __launch_bounds__(THREADS, 1)
    psf_gram_tc_kernel(const __grid_constant__ GramMaps maps, int M, int S, float scale, OutT *__restrict__ A,
                       int lda, int symmetric, int ntx, int ntiles, unsigned long long timeout_ns, int *status,
                       int hold) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[NSTAGE], empty_bar[NSTAGE], acc_full[NACC], acc_empty[NACC],
        done_bar;
    __shared__ uint32_t tmem_holder;
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    float *tp_all = reinterpret_cast<float *>(smem_raw + (sbase - smem_u32(smem_raw)) + NSTAGE * STAGE);

    if (warp == MMA_WARP) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < NSTAGE; ++i) {
            mbar_init(smem_u32(&full_bar[i]), 1);
            mbar_init(smem_u32(&empty_bar[i]), 1);
        }
        for (int i = 0; i < NACC; ++i) {
            mbar_init(smem_u32(&acc_full[i]), 1);
            mbar_init(smem_u32(&acc_empty[i]), 32 * EPI_WARPS);
        }
        mbar_init(smem_u32(&done_bar), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tmem_holder;
    const int nchunk = (M + KC - 1) / KC;
    // a bounded wait that also gives up once another role has aborted
    auto wait = [&](uint32_t bar, uint32_t parity) -> bool {
        if (abort_flag) return false;
        if (mbar_wait(bar, parity, now_ns() + timeout_ns)) return true;
        abort_flag = 1;
        return false;
    };

    if (warp == TMA_WARP) {
        if (lane == 0) {
            if (hold) {
                // the test hook: a bounded wait for a flag that nothing sets
                const unsigned long long deadline = now_ns() + timeout_ns;
                while (*(volatile int *)&psf_hold_flag == 0 && !abort_flag)
                    if (now_ns() > deadline) abort_flag = 1;
            }
            // ring position: stage st in its use u (the u-th time it is filled);
            // last_fill[st]: the use of stage st whose loads were issued last
            int st = 0;
            uint32_t u = 0;
            int last_fill[NSTAGE];
            for (int i = 0; i < NSTAGE; ++i) last_fill[i] = -1;
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x) {
                int ty, tx;
                tile_coords(t, ntx, symmetric, ty, tx);
                const int n0 = ty * BM, s0 = tx * BN;
                bool ok = true;
                for (int c = 0; c < nchunk; ++c) {
                    // the MMAs of use u - 1 of this stage must have read it
                    if (u > 0 && !wait(smem_u32(&empty_bar[st]), (u - 1) & 1)) {
                        ok = false;
                        break;
                    }
                    const uint32_t stage = sbase + st * STAGE, bar = smem_u32(&full_bar[st]);
                    const int x = KR * c;
                    mbar_expect_tx(bar, STAGE);
                    tma_load_2d(stage, &maps.a_hi, x, n0, bar);
                    tma_load_2d(stage + A_TILE, &maps.a_lo, x, n0, bar);
                    tma_load_2d(stage + 2 * A_TILE, &maps.b_hi, x, s0, bar);
                    tma_load_2d(stage + 2 * A_TILE + B_TILE, &maps.b_lo, x, s0, bar);
                    last_fill[st] = (int)u;
                    if (++st == NSTAGE) {
                        st = 0;
                        ++u;
                    }
                }
                if (!ok) break;
            }
            if (abort_flag) {
                // another role gave up: let the loads already issued land before
                // the CTA exits (bounded; a completed fill's phase reads as done)
                for (int i = 0; i < NSTAGE; ++i)
                    if (last_fill[i] >= 0)
                        mbar_wait(smem_u32(&full_bar[i]), (uint32_t)last_fill[i] & 1u, now_ns() + timeout_ns);
            }
        }
        __syncwarp();
    } else if (warp == MMA_WARP) {
        if (lane == 0) {
            int st = 0;
            uint32_t u = 0, k = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < ntiles && !abort_flag; t += gridDim.x, ++k) {
                // slot a was last used by tile k - 2: its epilogue must have drained it
                const int a = k & 1;
                if (k >= NACC && !wait(smem_u32(&acc_empty[a]), ((k >> 1) - 1) & 1)) break;
                fence_after();
                const uint32_t d_re = tmem + a * ACC_COLS, d_im = d_re + BN;
                bool ok = true;
                for (int c = 0; c < nchunk; ++c) {
                    if (!wait(smem_u32(&full_bar[st]), u & 1)) {
                        ok = false;
                        break;
                    }
                    fence_after();
                    const uint32_t stage = sbase + st * STAGE;
                    const uint32_t a_hi = stage, a_lo = stage + A_TILE;
                    const uint32_t b_hi = stage + 2 * A_TILE, b_lo = b_hi + B_TILE;
                    const uint32_t a_ops[3] = {a_hi, a_hi, a_lo};
                    const uint32_t b_ops[3] = {b_hi, b_lo, b_hi};
                    // K slices of 8 values are 32 bytes: real parts at 0, 32; imaginary at 64, 96
#pragma unroll
                    for (int term = 0; term < 3; ++term) {
#pragma unroll
                        for (int j = 0; j < 2; ++j) {
                            const uint64_t are = smem_desc_sw128(a_ops[term] + 32 * j);
                            const uint64_t aim = smem_desc_sw128(a_ops[term] + 64 + 32 * j);
                            const uint64_t bre = smem_desc_sw128(b_ops[term] + 32 * j);
                            const uint64_t bim = smem_desc_sw128(b_ops[term] + 64 + 32 * j);
                            const uint32_t acc = (c == 0 && term == 0 && j == 0) ? 0u : 1u;
                            mma_tf32(d_re, are, bre, IDESC, acc);             // Re G += Lr.Rr
                            mma_tf32(d_re, aim, bim, IDESC, 1u);              // Re G += Li.Ri
                            mma_tf32(d_im, are, bim, IDESC, acc);             // Im G += Lr.Ri
                            mma_tf32(d_im, aim, bre, IDESC_NEG_A, 1u);        // Im G -= Li.Rr
                        }
                    }
                    mma_commit(smem_u32(&empty_bar[st]));
                    issued = true;
                    if (++st == NSTAGE) {
                        st = 0;
                        ++u;
                    }
                }
                if (!ok) break;
                mma_commit(smem_u32(&acc_full[a]));
            }
            // no MMA may still be running when TMEM is released
            if (issued) {
                mma_commit(smem_u32(&done_bar));
                mbar_wait(smem_u32(&done_bar), 0, now_ns() + timeout_ns);
            }
        }
        __syncwarp();
    } else {
        constexpr int CB = BN / 32 / 2;            // column blocks per warp
        const int q = warp & 3, half = warp >> 2;  // TMEM lane quarter, half of the column blocks
        // per-warp 32 x 32 buffer: the TMA staging tile of an FP32 output block, or
        // (BF16 output) a transpose buffer with element (r, c) at r * 32 + (c ^ r)
        float *tp = tp_all + warp * 32 * 32;
        const float nanv = __int_as_float(0x7fc00000);
        uint32_t k = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
            int ty, tx;
            tile_coords(t, ntx, symmetric, ty, tx);
            const int nb = ty * BM + 32 * q;   // first row of this warp's 32 x 32 blocks
            const int n = nb + lane;           // this thread's row
            const int a = k & 1;
            const bool ok = wait(smem_u32(&acc_full[a]), (k >> 1) & 1);
            fence_after();
#pragma unroll 1
            for (int cb = CB * half; cb < CB * half + CB; ++cb) {
                const int sb = tx * BN + 32 * cb;  // first column of the block
                if (sb >= lda) break;
                // symmetric A: blocks below the diagonal are written by their mirror
                if (symmetric && sb + 32 <= nb) continue;
                float v[32];
                if (ok) {
                    float gi[32];
                    const uint32_t taddr = tmem + a * ACC_COLS + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * cb);
                    tmem_ld32(taddr, v);
                    tmem_ld32(taddr + BN, gi);
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = scale * fmaf(v[j], v[j], gi[j] * gi[j]);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = nanv;
                }
                // columns >= S come out as exact zeros (their operands are zero)
                if (sb != nb) {
                    if constexpr (std::is_same<OutT, float>::value) {
                        // direct block A[n][sb..sb+31]: this lane's row into the staging
                        // tile (128-byte swizzle: 16-byte chunk c of row r at c ^ (r mod 8)),
                        // then one TMA store; rows past S are clipped by the tensor map.
                        // The warp's previous store must have read the tile first.
                        if (lane == 0) bulk_wait_read();
                        __syncwarp();
                        float4 *row = reinterpret_cast<float4 *>(tp + lane * 32);
#pragma unroll
                        for (int c4 = 0; c4 < 8; ++c4)
                            row[c4 ^ (lane & 7)] = make_float4(v[4 * c4], v[4 * c4 + 1], v[4 * c4 + 2], v[4 * c4 + 3]);
                        fence_proxy_async();
                        __syncwarp();
                        if (lane == 0 && nb < S) tma_store_2d(&maps.out, smem_u32(tp), sb, nb);
                        if (symmetric) {
                            // mirrored block A[sb + j][nb + lane]: the same values transposed
                            // into the tile (lane = column), once the direct store has read it
                            if (lane == 0) bulk_wait_read();
                            __syncwarp();
#pragma unroll
                            for (int j = 0; j < 32; ++j) tp[j * 32 + ((((lane >> 2) ^ (j & 7))) << 2) + (lane & 3)] = v[j];
                            fence_proxy_async();
                            __syncwarp();
                            if (lane == 0 && sb < S && nb < lda) tma_store_2d(&maps.out, smem_u32(tp), nb, sb);
                        }
                    } else {
                        if (symmetric) {
                            // mirrored block A[s][n], s = sb + j: lanes cover 32 consecutive n
                            OutT *p = A + (size_t)sb * lda + n;
                            const int jmax = S - sb < 32 ? S - sb : 32;
#pragma unroll
                            for (int j = 0; j < 32; ++j, p += lda)
                                if (j < jmax) put<OutT>(p, v[j]);
                        }
                        // direct block A[n][sb..sb+31] through the transpose buffer
#pragma unroll
                        for (int j = 0; j < 32; ++j) tp[lane * 32 + (j ^ lane)] = v[j];
                        __syncwarp();
                        const int imax = S - nb < 32 ? S - nb : 32;
                        OutT *p = A + (size_t)nb * lda + sb + lane;
#pragma unroll 8
                        for (int i = 0; i < 32; ++i, p += lda)
                            if (i < imax) put<OutT>(p, tp[i * 32 + (lane ^ i)]);
                        __syncwarp();
                    }
                } else {
                    // diagonal block: unit diagonal; symmetric A takes every pair
                    // from the value computed for s >= n
                    OutT *prow = A + (size_t)n * lda + sb, *pcol = A + (size_t)sb * lda + n;
#pragma unroll
                    for (int j = 0; j < 32; ++j, pcol += lda) {
                        const int s = sb + j;
                        if (n < S && (!symmetric || s >= n)) put<OutT>(prow + j, s == n ? 1.f : v[j]);
                        if (symmetric && s > n && s < S) put<OutT>(pcol, v[j]);
                    }
                }
            }
            fence_before();
            mbar_arrive(smem_u32(&acc_empty[a]));
        }
        if (std::is_same<OutT, float>::value && lane == 0) bulk_wait_all();  // staging tile read and written out
        __syncwarp();
    }
    fence_before();
    __syncthreads();
    // a wait that ran out anywhere in the CTA: report it (the launch's output is NaN there)
    if (threadIdx.x == 0 && abort_flag && status) atomicCAS(status, 0, (int)DAMAS_ETIMEDOUT);
    if (warp == MMA_WARP) {
        fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS)
                     : "memory");
    }
}

// BF16 copy of an FP32 matrix (round to nearest even, as the BF16 Gram epilogue
// stores), four entries a thread when both pointers allow vector access.
__global__ void __launch_bounds__(256) to_bf16_kernel(const float *__restrict__ src, __nv_bfloat16 *__restrict__ dst,
                                                      size_t n, int vec) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vec) {
        if (4 * t + 3 < n) {
            const float4 v = reinterpret_cast<const float4 *>(src)[t];
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            uint2 w;
            w.x = *reinterpret_cast<const uint32_t *>(&lo);
            w.y = *reinterpret_cast<const uint32_t *>(&hi);
            reinterpret_cast<uint2 *>(dst)[t] = w;
        }
    } else if (t < n) {
        dst[t] = __float2bfloat16_rn(src[t]);
    }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// Tensor map over an operand plane (S rows of 2 ldm floats): boxes of 32
// values x 128 rows with 128-byte swizzle; rows past S read as zeros.
// Tensor map over the FP32 output A (S rows of lda values): boxes of 32 x 32,
// 128-byte swizzle (the staging tiles' layout).
bool make_out_map(CUtensorMap *m, float *A, int lda, int S) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)lda, (cuuint64_t)S};
    const cuuint64_t strides[1] = {(cuuint64_t)lda * sizeof(float)};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, A, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

bool make_map(CUtensorMap *m, const float *plane, int ldm, int S) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * ldm), (cuuint64_t)S};
    const cuuint64_t strides[1] = {(cuuint64_t)(2 * ldm) * sizeof(float)};
    const cuuint32_t box[2] = {KR, TMA_BOX_ROWS};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(plane), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

static size_t psf_smem_bytes() { return SMEM_BYTES + 1024; }
size_t psf_work_floats(int S, int ldm, bool symmetric) { return (size_t)S * 2 * ldm * (symmetric ? 2 : 4); }

cudaError_t launch_psf_gram(const float *Lre, const float *Lim, const float *Rre, const float *Rim, int ldm, int M,
                               int S, float scale, void *A, int lda, int a_dtype, float *work, int *status,
                               unsigned long long timeout_ns, int hold, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    if (ldm % KC || !work) return cudaErrorInvalidValue;
    const bool symmetric = Lre == Rre && Lim == Rim;
    const size_t plane = (size_t)S * 2 * ldm;
    float *LH = work, *LL = work + plane;
    float *RH = symmetric ? LH : work + 2 * plane, *RL = symmetric ? LL : work + 3 * plane;
    const size_t n_el = (size_t)S * ldm;
    const unsigned split_blocks = (unsigned)((n_el + 255) / 256);
    psf_split_kernel<<<split_blocks, 256, 0, st>>>(Lre, Lim, ldm, S, LH, LL);
    if (!symmetric) psf_split_kernel<<<split_blocks, 256, 0, st>>>(Rre, Rim, ldm, S, RH, RL);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    GramMaps maps;
    if (!make_map(&maps.a_hi, LH, ldm, S) || !make_map(&maps.a_lo, LL, ldm, S) || !make_map(&maps.b_hi, RH, ldm, S) ||
        !make_map(&maps.b_lo, RL, ldm, S))
        return cudaErrorInvalidValue;
    memset(&maps.out, 0, sizeof(maps.out));
    if (a_dtype != DAMAS_BF16 && !make_out_map(&maps.out, (float *)A, lda, S)) return cudaErrorInvalidValue;

    const int ntx = (lda + BN - 1) / BN, nty = (S + BM - 1) / BM;
    long long ntiles = 0;
    if (symmetric)
        for (int ty = 0; ty < nty; ++ty) ntiles += ntx - first_upper_tile(ty) > 0 ? ntx - first_upper_tile(ty) : 0;
    else
        ntiles = (long long)ntx * nty;
    if (ntiles <= 0) return cudaSuccess;
    if (ntiles > INT32_MAX) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    const size_t smem = psf_smem_bytes();
    if (a_dtype == DAMAS_BF16) {
        e = cudaFuncSetAttribute(psf_gram_tc_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        psf_gram_tc_kernel<__nv_bfloat16><<<grid, THREADS, smem, st>>>(
            maps, M, S, scale, (__nv_bfloat16 *)A, lda, symmetric ? 1 : 0, ntx, (int)ntiles, timeout_ns, status,
            hold);
    } else {
        e = cudaFuncSetAttribute(psf_gram_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        psf_gram_tc_kernel<float><<<grid, THREADS, smem, st>>>(maps, M, S, scale, (float *)A, lda,
                                                               symmetric ? 1 : 0, ntx, (int)ntiles, timeout_ns,
                                                               status, hold);
    }
    return cudaGetLastError();
}

cudaError_t launch_to_bf16(const float *src, void *dst, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int vec = n % 4 == 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0 && reinterpret_cast<uintptr_t>(dst) % 8 == 0;
    const size_t work = vec ? n / 4 : n;
    to_bf16_kernel<<<(unsigned)((work + 255) / 256), 256, 0, st>>>(src, (__nv_bfloat16 *)dst, n, vec);
    return cudaGetLastError();
}
