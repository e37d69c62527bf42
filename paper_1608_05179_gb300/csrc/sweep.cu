// DAMAS Gauss-Seidel iteration with the non-negativity clamp (§3, Eq. (13)-(14)),
// one persistent launch over a batch of independent systems, in two forms with
// bit-identical results: teams of CTAs (below) and one CTA per system (the
// single-CTA form, further down).
//
// Rows are cut into blocks of 32 in the paper's order (block J = rows
// 32J..32J+31) and processed as the sequence of steps G = t*nb + J (sweep t,
// block J).  A team of CTAs serves one system: CTA c owns a contiguous range of
// blocks and keeps x and the residual r = A x - b of its rows in shared memory
// (r as an unevaluated FP32 pair hi + lo), plus its rows of A when they fit
// ("resident"); otherwise A is read from global memory (L2/HBM), and the two
// chain tiles of each own block (its diagonal block and the block of columns
// J-1) are copied into shared memory ahead of their solve: all of them once
// when the CTA owns at most four blocks, else through a four-slot ring filled
// three own blocks ahead.
//
// Step G, in every CTA of the team (one CTA barrier per step):
//  - warp 0, if the CTA owns block J, solves its rows in order.  With
//    w = -r, row j gives dx_j = max(w_j, -x_j) (x_j + dx_j = max(x_j - r_j, 0),
//    Eq. (14) with A_jj = 1) and every later row i takes w_i -= A_ij dx_j.  A row
//    with x_j = 0 and w_j + sum_{k<j} A_jk x_k <= 0 cannot move (the earlier rows
//    of the block can raise w_j by at most that sum, since PSF entries are >= 0
//    and x_k + dx_k >= 0), so only the remaining "candidate" rows enter the
//    chain: the lane of row j broadcasts w_j by shuffle and every lane applies
//    A_kj dx_j.  dx_J is then published as 32 mailbox words
//    (epoch << 32 | bits(dx)), which carry their own readiness.  Otherwise
//    warp 0 polls the mailbox of block J (bounded wait).
//  - warps 1-3 and 5-7, concurrently, fold dx of step G-1 into the residual of
//    every own row: r_k += sum over the nonzero dx_c of A_kc dx_c, one thread
//    per row, with error-free transformations (TwoProduct by FMA, TwoSum) so the
//    residual does not drift over thousands of sweeps.  Entries A_kc of a column
//    c are read as row c of the transpose (A itself when symmetric), so a warp
//    reads contiguous memory.  The rows of block J are left alone while warp 0
//    solves them: warp 0 adds dx_{J-1} to its w itself (a plain FP32 partial
//    that only steers this block's decisions) and the stored residual of those
//    rows receives dx_{J-1} one step later, just before dx_J, so every row sees
//    every dx in step order.  Warp 4 only joins the barriers, leaving warp 0's
//    scheduler to it.
// Teams of equal size (2..16 CTAs) are launched as one thread-block cluster
// each, so each team runs on one die; otherwise the launch is cooperative.
// Systems of one block run the same steps without the overlap.  At the end x,
// the residual and the two dx blocks not yet folded into every row are written
// out, so a later call continues bit for bit.
#include <mutex>

#include "common.cuh"

#include "sweep.cuh"

namespace {

constexpr int SW_THREADS = 256;
constexpr int UPD_WARPS = 6;
constexpr int UPD_THREADS = 32 * UPD_WARPS;
constexpr unsigned FULL = 0xffffffffu;
constexpr int TSLOTS = 4;  // chain-tile slots of a streamed CTA (power of two)

__device__ __forceinline__ int upd_index(int warp) { return warp < 4 ? warp - 1 : warp - 2; }

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all but the N most recent copy groups of this thread have landed
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }
__device__ __forceinline__ float bf16_bits(unsigned short h) { return __uint_as_float((uint32_t)h << 16); }

struct Team {
    int S, R, nb, row0, nrows, jb0, jb1, lds_w, tile_ld;
};

// A[row0 + r][c] from the resident copy; the row stride lds_w is an odd number
// of 32-bit words, so a warp reading one column of 32 rows, or 32 columns of
// one row, touches 32 different banks.
template <bool F32>
__device__ __forceinline__ float res_at(const Team &T, const uint32_t *As, int r, int c) {
    if (F32) return __uint_as_float(As[r * T.lds_w + c]);
    const uint32_t w = As[r * T.lds_w + (c >> 1)];
    return (c & 1) ? bf16_hi(w) : bf16_lo(w);
}
// Chain tile of block J for column block X: tile[j][k] = At[32X + j][32J + k] = A[32J + k][32X + j].
template <bool F32>
__device__ __forceinline__ float tile_at(const Team &T, const char *tile, int j, int k) {
    if (F32) return ((const float *)(tile + j * T.tile_ld))[k];
    return bf16_bits(((const unsigned short *)(tile + j * T.tile_ld))[k]);
}
// A[i][col] read as At[col][i] from global memory.
template <bool F32>
__device__ __forceinline__ float col_at(const SweepSys &s, int col, int i) {
    const size_t o = (size_t)col * s.lda + i;
    if (F32) return ((const float *)s.At)[o];
    return bf16_bits(((const unsigned short *)s.At)[o]);
}

// Warp 0: copy the two chain tiles of own block J (diagonal block, and the
// block of columns J-1) into tile slot `buf`; rows beyond S are zero-filled.
template <bool F32>
__device__ __forceinline__ void prefetch_tiles(const SweepSys &s, const Team &T, char *buf, int J) {
    const int lane = threadIdx.x & 31;
    const int Jm1 = J == 0 ? T.nb - 1 : J - 1;
    const int elt = F32 ? 4 : 2;
    const int lg = F32 ? 3 : 2;  // 16-byte chunks per tile row
    for (int t = 0; t < 2; ++t) {
        const int X = t == 0 ? J : Jm1;
        char *tile = buf + t * 32 * T.tile_ld;
        for (int e = lane; e < (32 << lg); e += 32) {
            const int j = e >> lg, q = e & ((1 << lg) - 1);
            char *dst = tile + j * T.tile_ld + q * 16;
            const int row = X * 32 + j;
            if (row < T.S)
                cp_async16(dst, (const char *)s.At + ((size_t)row * s.lda + (size_t)J * 32) * elt + q * 16);
            else
                *(uint4 *)dst = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    cp_async_commit();
}

// The nonzero entries of a 32-wide dx vector as a compact list (warp 0);
// returns their number.
__device__ __forceinline__ int make_list(float d, unsigned char *idx, int *cnt) {
    const int lane = threadIdx.x & 31;
    const unsigned m = __ballot_sync(FULL, d != 0.f);
    if (d != 0.f) idx[__popc(m & ((1u << lane) - 1u))] = (unsigned char)lane;
    if (lane == 0) *cnt = __popc(m);
    return __popc(m);
}

// Compensated sum over the listed columns c of A[row0 + r][c0 + c] * d[c], in
// list order.  Eight terms at a time, with their loads issued together.
template <bool F32, bool RES>
__device__ __forceinline__ void dot_list(const SweepSys &s, const Team &T, const uint32_t *As, int r, int c0,
                                         const float *d, const unsigned char *idx, int n, float &hi, float &lo) {
    hi = 0.f;
    lo = 0.f;
    for (int q0 = 0; q0 < n; q0 += 8) {
        int c[8];
        float a[8], dd[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = idx[q0 + u < n ? q0 + u : q0];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            dd[u] = d[c[u]];
            a[u] = RES ? res_at<F32>(T, As, r, c0 + c[u]) : col_at<F32>(s, c0 + c[u], T.row0 + r);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if (q0 + u < n) {
                float p, pe, t;
                two_prod(a[u], dd[u], p, pe);
                two_sum(hi, p, hi, t);
                lo = __fadd_rn(lo, __fadd_rn(t, pe));
            }
        }
    }
}

// dot_list for up to NR rows of one thread at once (rows[q] < 0: none), the
// loads of all rows issued together; each row's sum is formed exactly as by
// dot_list.
template <bool F32, bool RES, int NR>
__device__ __forceinline__ void dot_list_rows(const SweepSys &s, const Team &T, const uint32_t *As, const int (&rows)[NR],
                                              int c0, const float *d, const unsigned char *idx, int n, float (&hi)[NR],
                                              float (&lo)[NR]) {
#pragma unroll
    for (int q = 0; q < NR; ++q) hi[q] = lo[q] = 0.f;
    for (int q0 = 0; q0 < n; q0 += 8) {
        int c[8];
        float dd[8], a[NR][8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            c[u] = idx[q0 + u < n ? q0 + u : q0];
            dd[u] = d[c[u]];
        }
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int u = 0; u < 8; ++u)
                a[q][u] = rows[q] < 0 ? 0.f
                          : RES       ? res_at<F32>(T, As, rows[q], c0 + c[u])
                                      : col_at<F32>(s, c0 + c[u], T.row0 + rows[q]);
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (q0 + u < n) {
                    float p, pe, t;
                    two_prod(a[q][u], dd[u], p, pe);
                    two_sum(hi[q], p, hi[q], t);
                    lo[q] = __fadd_rn(lo[q], __fadd_rn(t, pe));
                }
            }
    }
}

// residual[r] += (hi + lo), kept as an unevaluated pair
__device__ __forceinline__ void fold(float *rh, float *rl, int r, float hi, float lo) {
    float h, t;
    two_sum(rh[r], hi, h, t);
    rh[r] = h;
    rl[r] = __fadd_rn(rl[r], __fadd_rn(lo, t));
}

// Warp 0 solves own block J.  dm1 (or nullptr) is dx of the previous step
// (columns of block Jm1), which the stored residual of these rows does not hold
// yet.  nonneg says that the CTA's diagonal blocks have no negative entry
// (checked once per launch), which is what lets rows that cannot move be
// skipped.  Each of the three parts (partial, bound, chain) runs as a dense
// loop over all 32 positions when many are needed, or walks only the needed
// ones otherwise (both with warp-uniform control flow).  Returns dx of the
// lane's row; writes x of the block's rows.
template <bool F32, bool RES>
__device__ __forceinline__ float solve_block(const Team &T, const uint32_t *As, const char *tiles, int J, int Jm1,
                                             float *xs, const float *rh, const float *rl, const float *dm1,
                                             bool nonneg) {
    const int k = threadIdx.x & 31;
    const int i = J * 32 + k, r = i - T.row0;
    const bool valid = i < T.S;
    const char *tdiag = tiles, *tpart = tiles + 32 * T.tile_ld;
    auto diag_at = [&](int j) -> float {
        return RES ? (valid ? res_at<F32>(T, As, r, J * 32 + j) : 0.f) : tile_at<F32>(T, tdiag, j, k);
    };
    auto part_at = [&](int c) -> float {
        return RES ? (valid ? res_at<F32>(T, As, r, Jm1 * 32 + c) : 0.f) : tile_at<F32>(T, tpart, c, k);
    };
    const float x_old = valid ? xs[r] : 0.f;
    float w = valid ? -__fadd_rn(rh[r], rl[r]) : 0.f;

    // dx of the previous step on this block's rows
    const unsigned m1 = dm1 ? __ballot_sync(FULL, dm1[k] != 0.f) : 0u;
    if (__popc(m1) > 6) {
        float a[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) a[c] = part_at(c);
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
            p0 = __fmaf_rn(a[c], dm1[c], p0);
            p1 = __fmaf_rn(a[c + 1], dm1[c + 1], p1);
            p2 = __fmaf_rn(a[c + 2], dm1[c + 2], p2);
            p3 = __fmaf_rn(a[c + 3], dm1[c + 3], p3);
        }
        w = __fsub_rn(w, __fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3)));
    } else if (m1) {
        float p0 = 0.f;
        unsigned m = m1;
        while (m) {
            const int c = __ffs(m) - 1;
            m &= m - 1u;
            p0 = __fmaf_rn(part_at(c), dm1[c], p0);
        }
        w = __fsub_rn(w, p0);
    }

    // which rows can move: x > 0, or w + (the most the block's earlier rows can
    // raise w: sum_{j<k} A_kj x_j) > 0
    const float *xb = xs + (J * 32 - T.row0);  // x of the block's rows (rows past S read as 0 below)
    unsigned mask;
    if (nonneg) {
        const unsigned mx = __ballot_sync(FULL, valid && x_old > 0.f);
        float bound = 0.f;
        if (__popc(mx) > 6) {
            float b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
                if (j < k) b0 = __fmaf_rn(diag_at(j), (mx >> j) & 1u ? xb[j] : 0.f, b0);
                if (j + 1 < k) b1 = __fmaf_rn(diag_at(j + 1), (mx >> (j + 1)) & 1u ? xb[j + 1] : 0.f, b1);
                if (j + 2 < k) b2 = __fmaf_rn(diag_at(j + 2), (mx >> (j + 2)) & 1u ? xb[j + 2] : 0.f, b2);
                if (j + 3 < k) b3 = __fmaf_rn(diag_at(j + 3), (mx >> (j + 3)) & 1u ? xb[j + 3] : 0.f, b3);
            }
            bound = __fadd_rn(__fadd_rn(b0, b1), __fadd_rn(b2, b3));
        } else {
            unsigned m = mx;
            while (m) {
                const int j = __ffs(m) - 1;
                m &= m - 1u;
                if (j < k) bound = __fmaf_rn(diag_at(j), xb[j], bound);
            }
        }
        const float margin = 3.8e-6f * (fabsf(w) + bound);
        mask = __ballot_sync(FULL, valid && (x_old > 0.f || __fadd_rn(w, bound) > -margin));
    } else {
        mask = __ballot_sync(FULL, valid);
    }

    // the rows that can move, in order
    float dchain = 0.f;
    if (__popc(mask) > 12) {
        float arow[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) arow[j] = diag_at(j);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float wj = __shfl_sync(FULL, w, j);
            const float xj = __shfl_sync(FULL, x_old, j);
            const float d = fmaxf(wj, -xj);
            w = __fmaf_rn(-arow[j], d, w);
            if (k == j) dchain = d;
        }
    } else {
        unsigned m = mask;
        while (m) {
            const int j = __ffs(m) - 1;
            m &= m - 1u;
            const float a = diag_at(j);
            const float wj = __shfl_sync(FULL, w, j);
            const float d = fmaxf(wj, -xb[j]);
            w = __fmaf_rn(-a, d, w);
            if (k == j) dchain = d;
        }
    }
    const float x_new = __fadd_rn(x_old, dchain);  // = max(x - r, 0)
    if (valid) xs[r] = x_new;
    return __fsub_rn(x_new, x_old);
}

// One warp: for the rows of own block Jb, bnd = sum over j < k of A_kj x_j with
// the block's current x.  x of a block changes only when the block is solved,
// so a bound computed after one solve serves the next one, off the critical
// path (see solve_block2).
template <bool F32, bool RES>
__device__ __forceinline__ void block_bound(const SweepSys &s, const Team &T, const uint32_t *As, int Jb,
                                            const float *xs, float *bnd) {
    const int k = threadIdx.x & 31;
    const int r = Jb * 32 - T.row0 + k;
    const bool valid = Jb * 32 + k < T.S;
    const float xk = valid ? xs[r] : 0.f;
    unsigned m = __ballot_sync(FULL, xk > 0.f);
    float b = 0.f;
    while (m) {
        int c[8], cnt = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = m ? __ffs(m) - 1 : 0;
            if (m) {
                m &= m - 1u;
                ++cnt;
            }
        }
        float a[8], xj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xj[q] = __shfl_sync(FULL, xk, c[q]);
            a[q] = !valid || q >= cnt ? 0.f
                   : RES                  ? res_at<F32>(T, As, r, Jb * 32 + c[q])
                                          : col_at<F32>(s, Jb * 32 + c[q], T.row0 + r);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < cnt && c[q] < k) b = __fmaf_rn(a[q], xj[q], b);
    }
    if (valid) bnd[r] = b;
}

// Warp 0 solves own block J: the same arithmetic as solve_block, arranged for
// latency.  The bound of each row comes from bnd (block_bound); dx of the
// previous step arrives in a register (dprev: this lane's entry) and is
// broadcast by shuffles.  The chain takes the candidate rows eight at a time:
// their positions are pulled from the mask and their coefficients loaded
// together before the dependent steps run (a dense pass over all 32 rows when
// more than 16 can move).
template <bool F32, bool RES>
__device__ __forceinline__ float solve_block2(const Team &T, const uint32_t *As, const char *tiles, int J, int Jm1,
                                              float *xs, const float *rh, const float *rl, const float *bnd,
                                              float dprev, bool have_prev, bool nonneg, int &ncand) {
    const int k = threadIdx.x & 31;
    const int i = J * 32 + k, r = i - T.row0;
    const bool valid = i < T.S;
    const char *tdiag = tiles, *tpart = tiles + 32 * T.tile_ld;
    // A[32J + row][32J + col] and A[32J + row][32 Jm1 + col], rows and columns within the blocks
    auto diag_rc = [&](int row, int col) -> float {
        return RES ? (J * 32 + row < T.S ? res_at<F32>(T, As, J * 32 + row - T.row0, J * 32 + col) : 0.f)
                   : tile_at<F32>(T, tdiag, col, row);
    };
    auto part_at = [&](int c) -> float {
        return RES ? (valid ? res_at<F32>(T, As, r, Jm1 * 32 + c) : 0.f) : tile_at<F32>(T, tpart, c, k);
    };
    const float x_old = valid ? xs[r] : 0.f;
    float w = valid ? -__fadd_rn(rh[r], rl[r]) : 0.f;
    const float bound = valid ? bnd[r] : 0.f;

    // dx of the previous step on this block's rows: one dense pass over the 32
    // columns whenever any of them is nonzero (cheaper than walking a short list
    // of positions: full grid -2.6%, compressed -0.4%)
    const unsigned m1 = have_prev ? __ballot_sync(FULL, dprev != 0.f) : 0u;
    if (m1) {
        float a[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) a[c] = part_at(c);
        float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
            p0 = __fmaf_rn(a[c], __shfl_sync(FULL, dprev, c), p0);
            p1 = __fmaf_rn(a[c + 1], __shfl_sync(FULL, dprev, c + 1), p1);
            p2 = __fmaf_rn(a[c + 2], __shfl_sync(FULL, dprev, c + 2), p2);
            p3 = __fmaf_rn(a[c + 3], __shfl_sync(FULL, dprev, c + 3), p3);
        }
        w = __fsub_rn(w, __fadd_rn(__fadd_rn(p0, p1), __fadd_rn(p2, p3)));
    }

    // which rows can move: x > 0, or w + (the most the block's earlier rows can
    // raise w) > 0
    unsigned mask;
    if (nonneg) {
        const float margin = 3.8e-6f * (fabsf(w) + bound);
        mask = __ballot_sync(FULL, valid && (x_old > 0.f || __fadd_rn(w, bound) > -margin));
    } else {
        mask = __ballot_sync(FULL, valid);
    }

    ncand = __popc(mask);
    const float xneg = -x_old;
    float dchain = 0.f;
    if (__popc(mask) > 16) {
        float arow[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) arow[j] = diag_rc(k, j);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float wj = __shfl_sync(FULL, w, j);
            const float d = fmaxf(wj, __shfl_sync(FULL, xneg, j));
            w = __fmaf_rn(-arow[j], d, w);
            if (k == j) dchain = d;
        }
    } else {
        unsigned m = mask;
        while (m) {
            int c[8], cnt = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                c[q] = m ? __ffs(m) - 1 : 0;
                if (m) {
                    m &= m - 1u;
                    ++cnt;
                }
            }
            float a[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) a[q] = diag_rc(k, c[q]);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                if (q >= cnt) break;
                const int j = c[q];
                const float wj = __shfl_sync(FULL, w, j);
                const float d = fmaxf(wj, __shfl_sync(FULL, xneg, j));
                w = __fmaf_rn(-a[q], d, w);
                if (k == j) dchain = d;
            }
        }
    }
    const float x_new = __fadd_rn(x_old, dchain);  // = max(x - r, 0)
    if (valid) xs[r] = x_new;
    return __fsub_rn(x_new, x_old);
}

template <bool F32, bool RES, bool STATS>
__device__ __forceinline__ void sweep_cta(const SweepParams &p, const SweepSys &s, float (*dring)[32],
                                          unsigned char (*nzidx)[32], int *nzcnt, int *s_abort_p, char *smem) {
    int &s_abort = *s_abort_p;
    Team T;
    T.S = s.S;
    T.R = s.rows_per_cta;
    T.nb = (s.S + 31) / 32;
    T.row0 = (blockIdx.x - s.cta0) * T.R;
    T.nrows = max(0, min(T.R, s.S - T.row0));
    T.jb0 = T.row0 / 32;
    T.jb1 = min(T.nb, (T.row0 + T.R) / 32);
    T.lds_w = (F32 ? s.lda : s.lda / 2) + 1;
    T.tile_ld = 32 * (F32 ? 4 : 2) + 16;
    const int S = T.S, nb = T.nb;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool pipelined = nb >= 2;
    const long long Gend = (long long)s.iters * nb;
    const int elt = F32 ? 4 : 2;
    bool nonneg_all = true;
    // warp 0: blocks solved, rows that entered the chain, nonzero dx (launch statistics)
    unsigned long long st_solves = 0, st_cand = 0, st_nnz = 0;

    float *rh = (float *)smem;
    float *rl = rh + T.R;
    float *xs = rl + T.R;
    float *bnd = xs + T.R;                   // per-row bound for candidate detection
    uint32_t *As = (uint32_t *)(bnd + T.R);  // resident rows of A
    char *tiles = (char *)(bnd + T.R);       // or: TSLOTS slots of two chain tiles
    const int slot_bytes = 2 * 32 * T.tile_ld;
    // Streamed A: the chain tiles of own blocks.  With at most TSLOTS own blocks
    // they are loaded once and stay; otherwise a ring of TSLOTS slots is filled
    // TSLOTS - 1 own blocks ahead, so a block's tiles have landed long before it
    // is solved (own solve number q uses slot q mod TSLOTS).
    const int nown = T.jb1 - T.jb0;
    const bool ring = nown > TSLOTS;

    // ---- prologue
    if (RES) {
        const int wpr = s.lda * elt / 4;  // 32-bit words per row of A
        for (int r = warp; r < T.R; r += SW_THREADS / 32) {
            const uint32_t *src = (const uint32_t *)((const char *)s.A + (size_t)(T.row0 + r) * s.lda * elt);
            for (int v = lane; v < wpr; v += 32) As[(size_t)r * T.lds_w + v] = r < T.nrows ? src[v] : 0u;
        }
    }
    int slot_q = 0;   // warp 0: slot of the next own solve
    int pf_slot = 0;  // slot and own index of the next ring prefetch
    int pf_k = 0;
    if (!RES && warp == 0 && pipelined) {
        const int first = ring ? TSLOTS - 1 : nown;
        for (int q = 0; q < first; ++q) prefetch_tiles<F32>(s, T, tiles + q * slot_bytes, T.jb0 + q);
        pf_slot = first & (TSLOTS - 1);
        pf_k = first;
    }
    for (int r = threadIdx.x; r < T.R; r += SW_THREADS) {
        const int i = T.row0 + r;
        const bool ok = r < T.nrows;
        xs[r] = (ok && s.init != DAMAS_INIT_ZERO) ? s.x[i] : 0.f;
        rh[r] = ok ? (s.init == DAMAS_INIT_STATE ? s.state[i] : (s.init == DAMAS_INIT_X ? 0.f : -s.b[i])) : 0.f;
        rl[r] = (ok && s.init == DAMAS_INIT_STATE) ? s.state[S + i] : 0.f;
    }
    if (warp == 0) {
        // slots 2 and 3: dx of steps -2 and -1, kept in the state of an earlier call
        const bool have = s.init == DAMAS_INIT_STATE && pipelined;
        for (int q = 0; q < 4; ++q) {
            const float d = (have && q >= 2) ? s.state[2 * S + (q - 2) * 32 + lane] : 0.f;
            dring[q][lane] = d;
            make_list(d, nzidx[q], &nzcnt[q]);
        }
        if (lane == 0) s_abort = 0;
    }
    __syncthreads();
    if (s.init == DAMAS_INIT_X) {
        // r_i = sum_j A_ij x_j - b_i, compensated; one warp per row
        for (int r = warp; r < T.nrows; r += SW_THREADS / 32) {
            float hi = 0.f, lo = 0.f;
            const char *Arow = (const char *)s.A + (size_t)(T.row0 + r) * s.lda * elt;
            for (int j = lane; j < S; j += 32) {
                const float a = F32 ? ((const float *)Arow)[j] : bf16_bits(((const unsigned short *)Arow)[j]);
                float pr, pe, t;
                two_prod(a, s.x[j], pr, pe);
                two_sum(hi, pr, hi, t);
                lo = __fadd_rn(lo, __fadd_rn(t, pe));
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float h2 = __shfl_xor_sync(FULL, hi, o), l2 = __shfl_xor_sync(FULL, lo, o);
                float t;
                two_sum(hi, h2, hi, t);
                lo = __fadd_rn(__fadd_rn(lo, l2), t);
            }
            if (lane == 0) {
                float h, t;
                two_sum(hi, -s.b[T.row0 + r], h, t);
                rh[r] = h;
                rl[r] = __fadd_rn(lo, t);
            }
        }
    }
    // PSF matrices have no negative entry; a CTA whose diagonal blocks do is
    // solved row by row without skipping
    {
        int negs = 0;
        const char *gA = (const char *)s.A;
        for (int e = threadIdx.x; e < T.nrows * 32; e += SW_THREADS) {
            const int r = e >> 5, c = (T.row0 + r) / 32 * 32 + (e & 31);
            if (c < S) {
                const size_t o = (size_t)(T.row0 + r) * s.lda + c;
                const float a = F32 ? ((const float *)gA)[o] : bf16_bits(((const unsigned short *)gA)[o]);
                negs |= a < 0.f;
            }
        }
        nonneg_all = !__syncthreads_or(negs);
    }
    if (pipelined)
        for (int Jb = T.jb0 + warp; Jb < T.jb1; Jb += SW_THREADS / 32) block_bound<F32, RES>(s, T, As, Jb, xs, bnd);
    if (warp == 0 && !RES && pipelined) cp_async_wait_all();
    __syncthreads();

    // ---- steps
    float dprev = dring[3][lane];  // warp 0: this lane's dx of the previous step
    int J = 0;
    unsigned epoch = s.epoch0 + 1u;
    for (long long G = 0; G < Gend; ++G) {
        const int Jm1 = J == 0 ? nb - 1 : J - 1;
        const int Jm2 = Jm1 == 0 ? nb - 1 : Jm1 - 1;
        const bool ownJ = J >= T.jb0 && J < T.jb1;
        const int gi = (int)(G & 3), g1 = (gi + 3) & 3, g2 = (gi + 2) & 3;

        if (!pipelined) {
            // a single block: solve, then fold its dx into its own residual
            if (warp == 0) {
                const float dk = solve_block<F32, RES>(T, As, tiles, 0, 0, xs, rh, rl, nullptr, nonneg_all);
                dring[gi][lane] = dk;
                const int nzk = make_list(dk, nzidx[gi], &nzcnt[gi]);
                if (STATS) {
                    st_nnz += nzk;
                    ++st_solves;
                }
            }
            __syncthreads();
            if (warp != 0 && warp != 4 && nzcnt[gi]) {
                const int u = upd_index(warp) * 32 + lane;
                if (u < T.nrows) {
                    float hi, lo;
                    dot_list<F32, RES>(s, T, As, u, 0, dring[gi], nzidx[gi], nzcnt[gi], hi, lo);
                    fold(rh, rl, u, hi, lo);
                }
            }
            __syncthreads();
            ++epoch;
            continue;
        }

        if (warp == 0) {
            if (ownJ) {
                const char *tl = tiles;
                if (!RES) {
                    tl = tiles + (ring ? slot_q : J - T.jb0) * slot_bytes;
                    if (ring) {
                        cp_async_wait_group<TSLOTS - 2>();  // this block's group; later ones may fly
                        __syncwarp();
                    }
                }
                int nc;
                const float dk =
                    solve_block2<F32, RES>(T, As, tl, J, Jm1, xs, rh, rl, bnd, dprev, true, nonneg_all, nc);
                dprev = dk;
                if (STATS) st_cand += nc;
                if (J != p.withhold_block)
                    st_relaxed_u64(s.mbox + (size_t)J * 32 + lane,
                                   ((unsigned long long)epoch << 32) | __float_as_uint(dk));
                dring[gi][lane] = dk;
                const int nzk = make_list(dk, nzidx[gi], &nzcnt[gi]);
                if (STATS) {
                    st_nnz += nzk;
                    ++st_solves;
                }
                if (!RES && ring) {
                    // the slot just used takes the own block TSLOTS - 1 solves ahead
                    __syncwarp();
                    prefetch_tiles<F32>(s, T, tiles + pf_slot * slot_bytes, T.jb0 + pf_k);
                    pf_slot = (pf_slot + 1) & (TSLOTS - 1);
                    if (++pf_k == nown) pf_k = 0;
                    slot_q = (slot_q + 1) & (TSLOTS - 1);
                }
            } else {
                const unsigned long long *mb = s.mbox + (size_t)J * 32 + lane;
                unsigned long long w = 0, t0 = 0;
                int iter = 0;
                for (;;) {
                    w = ld_relaxed_u64(mb);
                    if (__all_sync(FULL, (unsigned)(w >> 32) >= epoch)) break;
                    if ((++iter & 31) == 0) {
                        int bad = 0;
                        if (lane == 0) {
                            const unsigned long long now = global_ns();
                            if (t0 == 0) t0 = now;
                            if (now - t0 > p.timeout_ns) {
                                atomicCAS(p.status, 0, DAMAS_ETIMEDOUT);
                                bad = 1;
                            }
                            if (ld_volatile_i32(p.status) != 0) bad = 1;
                        }
                        if (__shfl_sync(FULL, bad, 0)) {
                            if (lane == 0) s_abort = 1;
                            break;
                        }
                    }
                }
                const float d = __uint_as_float((unsigned)w);
                dprev = d;
                dring[gi][lane] = d;
                make_list(d, nzidx[gi], &nzcnt[gi]);
            }
        } else if (warp != 4) {
            const int n1 = nzcnt[g1];
            const bool ownJm1 = Jm1 >= T.jb0 && Jm1 < T.jb1;
            const int n2 = ownJm1 ? nzcnt[g2] : 0;
            if (n1 || n2) {
                const int skip0 = ownJ ? J * 32 - T.row0 : -64;     // rows of block J: warp 0 has them
                const int def0 = ownJm1 ? Jm1 * 32 - T.row0 : -64;  // rows of block J-1: fold dx_{G-2} first
                if (F32 && !RES && T.nrows > UPD_THREADS) {
                    // many streamed FP32 rows per thread: rows of block J-1 take dx_{G-2}
                    // first, then dx_{G-1} goes into every own row but those of block J,
                    // four rows of a thread at a time so that their loads overlap (the
                    // band workload measured 13% faster; BF16 rows measured slower)
                    if (n2) {
                        const int r = def0 + lane;
                        if (upd_index(warp) == (def0 >> 5) % UPD_WARPS && r < T.nrows) {
                            float hi, lo;
                            dot_list<F32, RES>(s, T, As, r, Jm2 * 32, dring[g2], nzidx[g2], n2, hi, lo);
                            fold(rh, rl, r, hi, lo);
                        }
                    }
                    if (n1) {
                        constexpr int NR = 4;
                        for (int r0 = upd_index(warp) * 32 + lane; r0 < T.nrows; r0 += NR * UPD_THREADS) {
                            int rows[NR];
#pragma unroll
                            for (int q = 0; q < NR; ++q) {
                                const int r = r0 + q * UPD_THREADS;
                                rows[q] = (r < T.nrows && !(r >= skip0 && r < skip0 + 32)) ? r : -1;
                            }
                            float hi[NR], lo[NR];
                            dot_list_rows<F32, RES, NR>(s, T, As, rows, Jm1 * 32, dring[g1], nzidx[g1], n1, hi, lo);
#pragma unroll
                            for (int q = 0; q < NR; ++q)
                                if (rows[q] >= 0) fold(rh, rl, rows[q], hi[q], lo[q]);
                        }
                    }
                } else {
                    for (int r = upd_index(warp) * 32 + lane; r < T.nrows; r += UPD_THREADS) {
                        if (r >= skip0 && r < skip0 + 32) continue;
                        float hi, lo;
                        if (n2 && r >= def0 && r < def0 + 32) {
                            dot_list<F32, RES>(s, T, As, r, Jm2 * 32, dring[g2], nzidx[g2], n2, hi, lo);
                            fold(rh, rl, r, hi, lo);
                        }
                        if (n1) {
                            dot_list<F32, RES>(s, T, As, r, Jm1 * 32, dring[g1], nzidx[g1], n1, hi, lo);
                            fold(rh, rl, r, hi, lo);
                        }
                    }
                }
            }
            // block J-1 was solved in the previous step: its bound for the next sweep
            if (ownJm1 && Jm1 != J && upd_index(warp) == ((Jm1 * 32 - T.row0) >> 5) % UPD_WARPS)
                block_bound<F32, RES>(s, T, As, Jm1, xs, bnd);
        }
        __syncthreads();
        if (s_abort) {
            if (warp == 0 && !RES) cp_async_wait_all();  // no copy may land after exit
            return;
        }
        if (++J == nb) {
            J = 0;
            ++epoch;
        }
    }

    // ---- results: x, and the state a later call continues from
    for (int r = threadIdx.x; r < T.nrows; r += SW_THREADS) {
        s.x[T.row0 + r] = xs[r];
        if (s.state) {
            s.state[T.row0 + r] = rh[r];
            s.state[S + T.row0 + r] = rl[r];
        }
    }
    if (s.state && T.jb1 == nb && threadIdx.x < 64) {
        const long long G = Gend - 2 + (threadIdx.x >> 5);
        s.state[2 * S + threadIdx.x] = pipelined ? dring[G & 3][lane] : 0.f;
    }
    if (STATS && threadIdx.x == 0) {
        atomicAdd(p.stats, st_solves);
        atomicAdd(p.stats + 1, st_cand);
        atomicAdd(p.stats + 2, st_nnz);
    }
    if (warp == 0 && !RES) cp_async_wait_all();
}

// A build kernel of the context gave up a wait (so A may hold NaN): report it
// and leave x and the state untouched.  Read by one thread and shared, so every
// thread of the CTA takes the same branch.
__device__ __forceinline__ bool upstream_failed(const SweepParams &p) {
    __shared__ int s_up;
    if (threadIdx.x == 0) s_up = p.upstream ? ld_volatile_i32(p.upstream) : 0;
    __syncthreads();
    if (s_up == 0) return false;
    if (threadIdx.x == 0) atomicCAS(p.status, 0, (int)DAMAS_ETIMEDOUT);
    return true;
}

// At most 128 registers a thread, so that two CTAs of streamed teams fit on an SM
// (a batch of teams then runs side by side in one launch).
template <bool STATS>
__global__ void __launch_bounds__(SW_THREADS, 2) damas_sweep_kernel(const SweepParams p) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float dring[4][32];
    __shared__ unsigned char nzidx[4][32];
    __shared__ int nzcnt[4];
    __shared__ int s_abort;
    if (upstream_failed(p)) return;
    int si = 0;
    while (si + 1 < p.nsys && (int)blockIdx.x >= p.sys[si + 1].cta0) ++si;
    const SweepSys s = p.sys[si];
    // one specialised body per storage type and placement, chosen once per CTA
    if (s.dtype == DAMAS_F32) {
        if (s.resident)
            sweep_cta<true, true, STATS>(p, s, dring, nzidx, nzcnt, &s_abort, smem);
        else
            sweep_cta<true, false, STATS>(p, s, dring, nzidx, nzcnt, &s_abort, smem);
    } else {
        if (s.resident)
            sweep_cta<false, true, STATS>(p, s, dring, nzidx, nzcnt, &s_abort, smem);
        else
            sweep_cta<false, false, STATS>(p, s, dring, nzidx, nzcnt, &s_abort, smem);
    }
}

// ---------------------------------------------------------------- single-CTA form
// One CTA per system, A streamed from global memory: every block is the CTA's
// own, so there are no hand-overs and a step is the row chain plus one CTA
// barrier.  The rest of the step's work is arranged so that it finishes within
// the chain:
//  - one thread of warp 4 keeps a ring of tile slots filled SOLO_PD steps ahead
//    by TMA (four 32x32 boxes of At per step, completion counted on the slot's
//    mbarrier): the chain and partial tiles of block J for warp 0, and the tiles
//    of columns J-2 and J-1 over the rows of block J+1;
//  - the helper warp (1) folds dx_{G-2} and then dx_{G-1} into the rows of
//    block J+1 from those tiles, so that block is current through dx_{G-1} when
//    warp 0 solves it in step G+1 (adding dx_G itself, as in the team form);
//  - the updater warps (all but 0, 1, 4, 8 and 12) fold dx_{G-2} into every
//    row but those of blocks J and J+1, four rows per thread, reading the
//    entries of A from global memory (L2) as one vector per column and group
//    (staging them into shared memory a step ahead with asynchronous copies
//    measured slower: 17.5 against 16.8 ms on the compressed 81x81 system).
//    The last of them also forms the bound of block J-1 from that block's
//    diagonal tile (its own rows start at 1280, so it is otherwise idle on
//    compressed grids);
//  - warps 8 and 12, and the updater warps beyond the last row, have no part
//    in the steps and wait at the CTA barrier after them.
// Every row still receives every dx in step order through the same error-free
// fold arithmetic, and warp 0 solves from the same residual and partial, so the
// iterates are bit for bit those of the team form; so are the state written at
// the end and the state a call starts from.
constexpr int SOLO_SLOTS = 6;          // tile slots; the slot of step G+SOLO_PD is refilled in step G
constexpr int SOLO_PD = 4;             // (slots G-1 and G are read in step G: SOLO_SLOTS >= SOLO_PD + 2)
constexpr int SOLO_THREADS = 512;      // 16 warps
constexpr int SOLO_UPD_THREADS = 352;  // the updaters: every warp but 0, 1, 4, 8 and 12
static_assert(SOLO_SLOTS >= SOLO_PD + 2, "a slot must not be refilled while it is read");

__device__ __forceinline__ bool solo_updater(int warp) { return warp >= 2 && (warp & 3) != 0; }
// The per-step barrier of the warps that run the steps (named barrier 1; the
// whole warp converges first, as the aligned barrier instruction requires).
__device__ __forceinline__ void step_barrier(int nwarps) {
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"r"(32 * nwarps) : "memory");
}
__device__ __forceinline__ int solo_upd_index(int warp) { return warp - 2 - (warp >> 2); }

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void solo_mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void solo_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait for the completion of the mbarrier phase with the given parity.
__device__ __forceinline__ bool solo_mbar_wait(uint32_t bar, uint32_t parity, unsigned long long timeout_ns) {
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((i & 15u) == 15u) {
            const unsigned long long now = global_ns();
            if (t0 == 0) t0 = now;
            if (now - t0 > timeout_ns) return false;
        }
    }
}
// One 32 x 32 box of At (x = column, y = row; rows past S read as zeros).
__device__ __forceinline__ void solo_tma_box(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// The TMA thread (warp 4, lane 0): the four tiles of step G (block J) into one slot,
// tile(Y, X)[j][k] = At[32X + j][32Y + k]: (J, J) the chain, (J, J-1) warp 0's
// partial, (J+1, J-2) and (J+1, J-1) the helper's fold into block J+1.
__device__ __forceinline__ void solo_issue_tiles(const CUtensorMap *map, const Team &T, char *slot, uint32_t bar,
                                                 int J) {
    const int nb = T.nb;
    const int Jp1 = J + 1 == nb ? 0 : J + 1;
    const int Jm1 = J == 0 ? nb - 1 : J - 1;
    const int Jm2 = Jm1 == 0 ? nb - 1 : Jm1 - 1;
    const int tile_bytes = 32 * T.tile_ld;
    solo_expect_tx(bar, 4u * tile_bytes);
    solo_tma_box(smem_addr(slot), map, 32 * J, 32 * J, bar);
    solo_tma_box(smem_addr(slot + tile_bytes), map, 32 * J, 32 * Jm1, bar);
    solo_tma_box(smem_addr(slot + 2 * tile_bytes), map, 32 * Jp1, 32 * Jm2, bar);
    solo_tma_box(smem_addr(slot + 3 * tile_bytes), map, 32 * Jp1, 32 * Jm1, bar);
}

// Helper warp: fold dx list 2 (tile t2) and then dx list 1 (tile t1) into the
// rows of block Y (lane = row).  Each list's sum is formed exactly as by
// dot_list; the lists are short (a few nonzero dx per block), so they are walked
// two columns at a time, both lists together.
template <bool F32>
__device__ __forceinline__ void solo_tile_fold2(const Team &T, const char *t2, const char *t1, int Y, const float *d2,
                                                const unsigned char *idx2, int n2, const float *d1,
                                                const unsigned char *idx1, int n1, float *rh, float *rl) {
    const int k = threadIdx.x & 31, r = Y * 32 + k;
    if ((n1 == 0 && n2 == 0) || r >= T.S) return;
    float h2 = 0.f, l2 = 0.f, h1 = 0.f, l1 = 0.f;
    const int n = n1 > n2 ? n1 : n2;
    for (int q0 = 0; q0 < n; q0 += 2) {
        int c2[2], c1[2];
        float a2[2], a1[2], e2[2], e1[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            c2[u] = q0 + u < n2 ? idx2[q0 + u] : 0;
            c1[u] = q0 + u < n1 ? idx1[q0 + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            e2[u] = d2[c2[u]];
            a2[u] = tile_at<F32>(T, t2, c2[u], k);
            e1[u] = d1[c1[u]];
            a1[u] = tile_at<F32>(T, t1, c1[u], k);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            float p, pe, t;
            if (q0 + u < n2) {
                two_prod(a2[u], e2[u], p, pe);
                two_sum(h2, p, h2, t);
                l2 = __fadd_rn(l2, __fadd_rn(t, pe));
            }
            if (q0 + u < n1) {
                two_prod(a1[u], e1[u], p, pe);
                two_sum(h1, p, h1, t);
                l1 = __fadd_rn(l1, __fadd_rn(t, pe));
            }
        }
    }
    if (n2) fold(rh, rl, r, h2, l2);
    if (n1) fold(rh, rl, r, h1, l1);
}

// One warp: block_bound of block Jb from its diagonal tile (Jb, Jb).
template <bool F32>
__device__ __forceinline__ void solo_tile_bound(const Team &T, const char *tdiag, int Jb, const float *xs,
                                                float *bnd) {
    const int k = threadIdx.x & 31, r = Jb * 32 + k;
    const bool valid = r < T.S;
    const float xk = valid ? xs[r] : 0.f;
    unsigned m = __ballot_sync(FULL, xk > 0.f);
    float b = 0.f;
    while (m) {
        int c[8], cnt = 0;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            c[q] = m ? __ffs(m) - 1 : 0;
            if (m) {
                m &= m - 1u;
                ++cnt;
            }
        }
        float a[8], xj[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            xj[q] = __shfl_sync(FULL, xk, c[q]);
            a[q] = q < cnt ? tile_at<F32>(T, tdiag, c[q], k) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (q < cnt && c[q] < k) b = __fmaf_rn(a[q], xj[q], b);
    }
    if (valid) bnd[r] = b;
}

// Updater thread ut: fold the listed dx (columns c0 + idx[u]) into the rows of
// its groups of four: every block but skip1 and skip2, or only block `only`
// when it is >= 0.  The entries of a column over a group are one 16-byte
// (FP32) or 8-byte (BF16) load from global memory, two columns' loads issued
// together.  Each row's sum is formed exactly as by dot_list.
template <bool F32>
__device__ __forceinline__ void solo_fold(const SweepSys &s, const Team &T, int ut, int c0, const float *d,
                                          const unsigned char *idx, int n, int skip1, int skip2, int only, float *rh,
                                          float *rl) {
    if (n == 0) return;
    for (int g = ut; 4 * g < T.S; g += SOLO_UPD_THREADS) {
        const int blk = g >> 3;
        if (only >= 0 ? blk != only : (blk == skip1 || blk == skip2)) continue;
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        for (int u0 = 0; u0 < n; u0 += 2) {
            float a[2][4], dd[2];
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                const int u = u0 + v < n ? u0 + v : u0;
                const int c = idx[u];
                dd[v] = d[c];
                const size_t o = (size_t)(c0 + c) * s.lda + 4 * g;
                if (F32) {
                    const float4 w = *(const float4 *)((const float *)s.At + o);
                    a[v][0] = w.x;
                    a[v][1] = w.y;
                    a[v][2] = w.z;
                    a[v][3] = w.w;
                } else {
                    const uint2 w = *(const uint2 *)((const unsigned short *)s.At + o);
                    a[v][0] = bf16_lo(w.x);
                    a[v][1] = bf16_hi(w.x);
                    a[v][2] = bf16_lo(w.y);
                    a[v][3] = bf16_hi(w.y);
                }
            }
#pragma unroll
            for (int v = 0; v < 2; ++v)
                if (u0 + v < n) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float p, pe, t;
                        two_prod(a[v][q], dd[v], p, pe);
                        two_sum(hi[q], p, hi[q], t);
                        lo[q] = __fadd_rn(lo[q], __fadd_rn(t, pe));
                    }
                }
        }
        // fold() on the four rows, as one 16-byte access to each half of the pair
        float4 *ph = (float4 *)(rh + 4 * g), *pl = (float4 *)(rl + 4 * g);
        float4 h4 = *ph, l4 = *pl;
        float hh[4] = {h4.x, h4.y, h4.z, h4.w}, ll[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (4 * g + q < T.S) {
                float h, t;
                two_sum(hh[q], hi[q], h, t);
                hh[q] = h;
                ll[q] = __fadd_rn(ll[q], __fadd_rn(lo[q], t));
            }
        *ph = make_float4(hh[0], hh[1], hh[2], hh[3]);
        *pl = make_float4(ll[0], ll[1], ll[2], ll[3]);
    }
}

template <bool F32, bool STATS>
__device__ __forceinline__ void sweep_solo(const SweepParams &p, const SweepSys &s, const CUtensorMap *map,
                                           float (*dring)[32], unsigned char (*nzidx)[32], int *nzcnt,
                                           unsigned long long *tbar, int *s_abort_p, char *smem) {
    int &s_abort = *s_abort_p;
    Team T;
    T.S = s.S;
    T.nb = (s.S + 31) / 32;
    T.R = T.nb * 32;
    T.row0 = 0;
    T.nrows = s.S;
    T.jb0 = 0;
    T.jb1 = T.nb;
    T.lds_w = 0;
    T.tile_ld = 32 * (F32 ? 4 : 2);  // dense 32 x 32 boxes as TMA writes them
    const int S = T.S, nb = T.nb, R = T.R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long Gend = (long long)s.iters * nb;
    const int elt = F32 ? 4 : 2;
    const bool upd = solo_updater(warp);
    const int ut = upd ? solo_upd_index(warp) * 32 + lane : 0;
    // warp 0: blocks solved, rows that entered the chain, nonzero dx (launch statistics)
    unsigned long long st_solves = 0, st_cand = 0, st_nnz = 0;

    // tile slots first, 128-byte aligned for TMA; then the rows
    char *tiles = smem + ((128u - (smem_addr(smem) & 127u)) & 127u);
    const int slot_bytes = 4 * 32 * T.tile_ld;
    float *rh = (float *)(tiles + SOLO_SLOTS * slot_bytes);
    float *rl = rh + R;
    float *xs = rl + R;
    float *bnd = xs + R;

    // ---- prologue (as in the team form)
    if (threadIdx.x == 0) {
        for (int q = 0; q < SOLO_SLOTS; ++q) solo_mbar_init(smem_addr(&tbar[q]));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int r = threadIdx.x; r < R; r += SOLO_THREADS) {
        const bool ok = r < S;
        xs[r] = (ok && s.init != DAMAS_INIT_ZERO) ? s.x[r] : 0.f;
        rh[r] = ok ? (s.init == DAMAS_INIT_STATE ? s.state[r] : (s.init == DAMAS_INIT_X ? 0.f : -s.b[r])) : 0.f;
        rl[r] = (ok && s.init == DAMAS_INIT_STATE) ? s.state[S + r] : 0.f;
        bnd[r] = 0.f;
    }
    if (warp == 0) {
        const bool have = s.init == DAMAS_INIT_STATE;
        for (int q = 0; q < 4; ++q) {
            const float d = (have && q >= 2) ? s.state[2 * S + (q - 2) * 32 + lane] : 0.f;
            dring[q][lane] = d;
            make_list(d, nzidx[q], &nzcnt[q]);
        }
    }
    __syncthreads();
    // tile slots of steps 0 .. SOLO_PD-1 (the TMA thread); phase bit q: parity of
    // the next completion of slot q
    uint32_t phase = 0;
    if (warp == 4 && lane == 0)
        for (int q = 0; q < SOLO_PD && q < Gend; ++q)
            solo_issue_tiles(map, T, tiles + q * slot_bytes, smem_addr(&tbar[q]), q % nb);
    if (s.init == DAMAS_INIT_X) {
        for (int r = warp; r < S; r += SOLO_THREADS / 32) {
            float hi = 0.f, lo = 0.f;
            const char *Arow = (const char *)s.A + (size_t)r * s.lda * elt;
            for (int j = lane; j < S; j += 32) {
                const float a = F32 ? ((const float *)Arow)[j] : bf16_bits(((const unsigned short *)Arow)[j]);
                float pr, pe, t;
                two_prod(a, s.x[j], pr, pe);
                two_sum(hi, pr, hi, t);
                lo = __fadd_rn(lo, __fadd_rn(t, pe));
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float h2 = __shfl_xor_sync(FULL, hi, o), l2 = __shfl_xor_sync(FULL, lo, o);
                float t;
                two_sum(hi, h2, hi, t);
                lo = __fadd_rn(__fadd_rn(lo, l2), t);
            }
            if (lane == 0) {
                float h, t;
                two_sum(hi, -s.b[r], h, t);
                rh[r] = h;
                rl[r] = __fadd_rn(lo, t);
            }
        }
    }
    bool nonneg_all;
    {
        int negs = 0;
        const char *gA = (const char *)s.A;
        for (int e = threadIdx.x; e < S * 32; e += SOLO_THREADS) {
            const int r = e >> 5, c = r / 32 * 32 + (e & 31);
            if (c < S) {
                const size_t o = (size_t)r * s.lda + c;
                const float a = F32 ? ((const float *)gA)[o] : bf16_bits(((const unsigned short *)gA)[o]);
                negs |= a < 0.f;
            }
        }
        nonneg_all = !__syncthreads_or(negs);
    }
    for (int Jb = warp; Jb < nb; Jb += SOLO_THREADS / 32) block_bound<F32, false>(s, T, nullptr, Jb, xs, bnd);
    if (warp == 4 && lane == 0 && Gend > 0) {
        if (solo_mbar_wait(smem_addr(&tbar[0]), 0, p.timeout_ns)) {
            phase ^= 1u;
        } else {
            atomicCAS(p.status, 0, DAMAS_ETIMEDOUT);
            s_abort = 1;
        }
    }
    __syncthreads();

    // ---- steps
    float dprev = dring[3][lane];
    int J = 0, sl = 0, slm1 = SOLO_SLOTS - 1, pf_sl = SOLO_PD % SOLO_SLOTS, pf_J = SOLO_PD % nb;
    long long G = 0;
    // Only the warps with a part in the steps run them: warp 0, the helper, the
    // TMA warp, the updater warps that hold rows (thread ut holds rows 4ut..4ut+3)
    // and the last updater warp (the bound).  They meet at a named barrier sized
    // to them; the others wait at the CTA barrier after the loop (on the 81x81
    // compressed system, 10 warps of 16 step: 15.6 against 16.3 ms).
    const int n_upd_rows = min(SOLO_UPD_THREADS / 32, (S + 127) / 128);
    const int n_active = 3 + n_upd_rows + (n_upd_rows < SOLO_UPD_THREADS / 32 ? 1 : 0);
    const bool active = warp == 0 || warp == 1 || warp == 4 || warp == SOLO_THREADS / 32 - 1 ||
                        (upd && solo_upd_index(warp) < n_upd_rows);
    for (; active && G < Gend && !s_abort; ++G) {
        const int Jm1 = J == 0 ? nb - 1 : J - 1;
        const int Jm2 = Jm1 == 0 ? nb - 1 : Jm1 - 1;
        const int Jp1 = J + 1 == nb ? 0 : J + 1;
        const int gi = (int)(G & 3), g1 = (gi + 3) & 3, g2 = (gi + 2) & 3;
        const char *slot = tiles + sl * slot_bytes;
        if (warp == 0) {
            int nc;
            const float dk = solve_block2<F32, false>(T, nullptr, slot, J, Jm1, xs, rh, rl, bnd, dprev, true,
                                                      nonneg_all, nc);
            dprev = dk;
            dring[gi][lane] = dk;
            const int nzk = make_list(dk, nzidx[gi], &nzcnt[gi]);
            if (STATS) {
                st_nnz += nzk;
                st_cand += nc;
                ++st_solves;
            }
        } else if (warp == 1) {
            // block J+1: dx_{G-2} (which a call resumed from a state already folded
            // there), then dx_{G-1}
            const int tb = 32 * T.tile_ld;
            solo_tile_fold2<F32>(T, slot + 2 * tb, slot + 3 * tb, Jp1, dring[g2], nzidx[g2], G > 0 ? nzcnt[g2] : 0,
                                 dring[g1], nzidx[g1], nzcnt[g1], rh, rl);
        } else if (warp == 4) {
            // one thread: the tiles of step G+SOLO_PD, then the wait for those of step G+1
            if (lane == 0 && G + SOLO_PD < Gend)
                solo_issue_tiles(map, T, tiles + pf_sl * slot_bytes, smem_addr(&tbar[pf_sl]), pf_J);
            if (lane == 0 && G + 1 < Gend) {
                const int s1 = sl + 1 == SOLO_SLOTS ? 0 : sl + 1;
                if (solo_mbar_wait(smem_addr(&tbar[s1]), (phase >> s1) & 1u, p.timeout_ns)) {
                    phase ^= 1u << s1;
                } else {
                    atomicCAS(p.status, 0, DAMAS_ETIMEDOUT);
                    s_abort = 1;
                }
            }
        } else if (upd) {
            if (G == 0)  // a resumed state holds dx_{-2} everywhere but in block nb-1
                solo_fold<F32>(s, T, ut, Jm2 * 32, dring[g2], nzidx[g2], nzcnt[g2], -1, -1, Jm1, rh, rl);
            else
                solo_fold<F32>(s, T, ut, Jm2 * 32, dring[g2], nzidx[g2], nzcnt[g2], J, Jp1, -1, rh, rl);
            // the last updater warp (whose rows start at 1280): block J-1 was solved
            // in the previous step, its bound for the next solve
            if (warp == SOLO_THREADS / 32 - 1 && G > 0)
                solo_tile_bound<F32>(T, tiles + slm1 * slot_bytes, Jm1, xs, bnd);
        }
        step_barrier(n_active);
        J = Jp1;
        slm1 = sl;
        sl = sl + 1 == SOLO_SLOTS ? 0 : sl + 1;
        pf_sl = pf_sl + 1 == SOLO_SLOTS ? 0 : pf_sl + 1;
        pf_J = pf_J + 1 == nb ? 0 : pf_J + 1;
    }
    __syncthreads();  // every warp, in the steps or not, sees how they ended
    if (s_abort) {
        // a tile wait ran out (for step G): let the boxes still in flight, those of
        // steps G .. G+SOLO_PD-1, land (bounded), then stop
        if (warp == 4 && lane == 0)
            for (long long q = G; q < G + SOLO_PD && q < Gend; ++q) {
                const int sq = (int)(q % SOLO_SLOTS);
                if (solo_mbar_wait(smem_addr(&tbar[sq]), (phase >> sq) & 1u, p.timeout_ns)) phase ^= 1u << sq;
            }
        __syncthreads();
        return;
    }

    // ---- drain to the team form's final state: dx_{Gend-2} into every block
    // but 0 (the helper's) and nb-1 (which the team form also leaves without it)
    if (Gend > 0 && upd) {
        const int gq = (int)((Gend - 2) & 3);
        solo_fold<F32>(s, T, ut, (nb - 2) * 32, dring[gq], nzidx[gq], nzcnt[gq], 0, nb - 1, -1, rh, rl);
    }
    __syncthreads();

    // ---- results: x, and the state a later call continues from
    for (int r = threadIdx.x; r < S; r += SOLO_THREADS) {
        s.x[r] = xs[r];
        if (s.state) {
            s.state[r] = rh[r];
            s.state[S + r] = rl[r];
        }
    }
    if (s.state && threadIdx.x < 64) {
        const long long Gx = Gend - 2 + (threadIdx.x >> 5);
        s.state[2 * S + threadIdx.x] = dring[Gx & 3][lane];
    }
    if (STATS && threadIdx.x == 0) {
        atomicAdd(p.stats, st_solves);
        atomicAdd(p.stats + 1, st_cand);
        atomicAdd(p.stats + 2, st_nnz);
    }
}

template <bool STATS>
__global__ void __launch_bounds__(SOLO_THREADS, 1)
    damas_sweep_solo_kernel(const SweepParams p, const __grid_constant__ SoloMaps maps) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float dring[4][32];
    __shared__ unsigned char nzidx[4][32];
    __shared__ int nzcnt[4];
    __shared__ __align__(8) unsigned long long tbar[SOLO_SLOTS];
    __shared__ int s_abort;
    if (upstream_failed(p)) return;
    const SweepSys s = p.sys[blockIdx.x];
    if (s.dtype == DAMAS_F32)
        sweep_solo<true, STATS>(p, s, &maps.m[blockIdx.x], dring, nzidx, nzcnt, tbar, &s_abort, smem);
    else
        sweep_solo<false, STATS>(p, s, &maps.m[blockIdx.x], dring, nzidx, nzcnt, tbar, &s_abort, smem);
}

}  // namespace

size_t sweep_smem_bytes(int R, int lda, int dtype, bool resident) {
    const size_t elt = dtype == DAMAS_F32 ? 4 : 2;
    size_t b = (size_t)4 * R * sizeof(float);
    if (resident)
        b += (size_t)R * ((size_t)lda * elt / 4 + 1) * 4;
    else
        b += (size_t)TSLOTS * 2 * 32 * (32 * elt + 16);
    return b;
}

// The two instantiations (with and without launch statistics) have the same
// resources (at most 128 registers a thread): the occupancy of the plain one
// serves both.
cudaError_t sweep_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e =
        cudaFuncSetAttribute(damas_sweep_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, damas_sweep_kernel<false>, SW_THREADS, smem);
}

namespace {

template <bool STATS>
cudaError_t launch_sweep_t(const SweepParams &p, int grid, size_t smem, cudaStream_t st) {
    auto kern = damas_sweep_kernel<STATS>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // Teams only wait on their own members.  When every team has the same size
    // (2..16 CTAs) the launch is one thread-block cluster per team: a cluster is
    // co-scheduled on one GPC, so a team's hand-overs stay on one die (one-way
    // hand-overs between SMs of different dies take about 1.7 times as long).
    // Only when the device holds every cluster at once; otherwise the launch is
    // cooperative as below.
    bool same = p.nsys >= 1 && p.sys[0].ncta >= 2 && p.sys[0].ncta <= 16;
    for (int i = 1; same && i < p.nsys; ++i) same = p.sys[i].ncta == p.sys[0].ncta;
    if (same && grid == p.nsys * p.sys[0].ncta &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
        cudaLaunchConfig_t cc = {};
        cc.gridDim = dim3(grid);
        cc.blockDim = dim3(SW_THREADS);
        cc.dynamicSmemBytes = smem;
        cc.stream = st;
        cudaLaunchAttribute ca[1];
        ca[0].id = cudaLaunchAttributeClusterDimension;
        ca[0].val.clusterDim.x = p.sys[0].ncta;
        ca[0].val.clusterDim.y = 1;
        ca[0].val.clusterDim.z = 1;
        cc.attrs = ca;
        cc.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cc) == cudaSuccess && ncl >= p.nsys)
            return cudaLaunchKernelEx(&cc, kern, p);
        cudaGetLastError();  // a refused cluster query leaves no error behind
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SW_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, p);
}

template <bool STATS>
cudaError_t launch_sweep_solo_t(const SweepParams &p, const SoloMaps &maps, size_t smem, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(damas_sweep_solo_kernel<STATS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // no CTA waits on another: a plain launch, one CTA per system
    damas_sweep_solo_kernel<STATS><<<p.nsys, SOLO_THREADS, smem, st>>>(p, maps);
    return cudaGetLastError();
}

}  // namespace

// The statistics instantiation only when the caller asks for the counts.
cudaError_t launch_sweep(const SweepParams &p, int grid, size_t smem, cudaStream_t st) {
    return p.stats ? launch_sweep_t<true>(p, grid, smem, st) : launch_sweep_t<false>(p, grid, smem, st);
}

size_t sweep_solo_smem_bytes(int R, int dtype) {
    const size_t elt = dtype == DAMAS_F32 ? 4 : 2;
    return 128 + (size_t)SOLO_SLOTS * 4 * 32 * 32 * elt + (size_t)4 * R * sizeof(float);
}

// Tensor map over a system's At for the single-CTA form (FP32 or BF16, S rows of
// lda values): unswizzled 32 x 32 boxes; rows past S read as zeros.
bool make_sweep_tile_map(CUtensorMap *m, const void *At, int dtype, int lda, int S) {
    using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                     const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static std::once_flag once;
    static EncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(f);
    });
    if (!fn) return false;
    const size_t elt = dtype == DAMAS_F32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)lda, (cuuint64_t)S};
    const cuuint64_t strides[1] = {(cuuint64_t)lda * elt};
    const cuuint32_t box[2] = {32, 32};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, dtype == DAMAS_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
              const_cast<void *>(At), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

cudaError_t sweep_solo_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(damas_sweep_solo_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, damas_sweep_solo_kernel<false>, SOLO_THREADS,
                                                         smem);
}

cudaError_t launch_sweep_solo(const SweepParams &p, const SoloMaps &maps, size_t smem, cudaStream_t st) {
    return p.stats ? launch_sweep_solo_t<true>(p, maps, smem, st) : launch_sweep_solo_t<false>(p, maps, smem, st);
}
