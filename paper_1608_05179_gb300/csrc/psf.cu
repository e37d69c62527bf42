// PSF matrix (§3 Eq. (10), arranged as A of Eq. (12)): a complex Gram product
// with a |.|^2 epilogue,
//     A[n][s] = scale * | sum_m conj(L[n][m]) * R[s][m] |^2,
// diagonal stored as exactly 1, columns S..lda-1 zero.
//
// CUDA-core tiled kernel: 64 x 64 output tile per CTA, 256 threads each
// holding a 4 x 4 tile of complex accumulators (FP32), K (= microphones)
// staged through shared memory in chunks of 16.  The contraction is short
// (K = M <= 256) so for the library's sizes the kernel is bound by the A write
// and the CUDA-core FMA rate.  When L and R are the same vectors (formulation
// E) A is symmetric: only tiles on or above the diagonal are computed and each
// is also written mirrored (through shared memory, so both writes are
// coalesced), which makes A exactly symmetric in FP32 and halves the work.
#include "common.cuh"

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

template <typename OutT>
__device__ __forceinline__ void store_elem(OutT *A, size_t off, float v);
template <>
__device__ __forceinline__ void store_elem<float>(float *A, size_t off, float v) { A[off] = v; }
template <>
__device__ __forceinline__ void store_elem<__nv_bfloat16>(__nv_bfloat16 *A, size_t off, float v) {
    A[off] = __float2bfloat16_rn(v);
}

template <typename OutT>
__global__ void __launch_bounds__(256) psf_gram_kernel(const float *__restrict__ Lre, const float *__restrict__ Lim,
                                                       const float *__restrict__ Rre, const float *__restrict__ Rim,
                                                       int ldm, int M, int S, float scale, OutT *__restrict__ A,
                                                       int lda, int sym_nt) {
    // staging for the K chunks; reused for the output tile in the epilogue
    __shared__ float sbuf[4 * TK * (TM + 4)];
    float(*sLr)[TM + 4] = reinterpret_cast<float(*)[TM + 4]>(sbuf);
    float(*sLi)[TM + 4] = reinterpret_cast<float(*)[TM + 4]>(sbuf + TK * (TM + 4));
    float(*sRr)[TN + 4] = reinterpret_cast<float(*)[TN + 4]>(sbuf + 2 * TK * (TM + 4));
    float(*sRi)[TN + 4] = reinterpret_cast<float(*)[TN + 4]>(sbuf + 3 * TK * (TM + 4));
    static_assert(4 * TK * (TM + 4) >= TM * (TN + 1), "output tile must fit the staging buffer");
    const bool sym = sym_nt > 0;
    int ty = blockIdx.y, tx = blockIdx.x;
    if (sym) {
        // blockIdx.x enumerates the tiles (ty <= tx) of the upper triangle row by row
        const int nt = sym_nt;
        int t = blockIdx.x;
        ty = 0;
        while (t >= nt - ty) {
            t -= nt - ty;
            ++ty;
        }
        tx = ty + t;
    }
    const int n0 = ty * TM, s0 = tx * TN;
    const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    float gr[4][4], gi[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) gr[i][j] = gi[i][j] = 0.f;

    for (int m0 = 0; m0 < M; m0 += TK) {
        // stage L[n0..n0+63][m0..m0+15] and R[s0..][..] transposed to [m][n]
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int r = e / TK, k = e % TK;
            const int n = n0 + r, s = s0 + r, m = m0 + k;
            const bool okm = m < M;
            sLr[k][r] = (okm && n < S) ? Lre[(size_t)n * ldm + m] : 0.f;
            sLi[k][r] = (okm && n < S) ? Lim[(size_t)n * ldm + m] : 0.f;
            sRr[k][r] = (okm && s < S) ? Rre[(size_t)s * ldm + m] : 0.f;
            sRi[k][r] = (okm && s < S) ? Rim[(size_t)s * ldm + m] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            float ar[4], ai[4], br[4], bi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                ar[i] = sLr[k][ly + 16 * i];
                ai[i] = sLi[k][ly + 16 * i];
                br[i] = sRr[k][lx + 16 * i];
                bi[i] = sRi[k][lx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    // conj(a) * b = (ar br + ai bi) + j (ar bi - ai br)
                    gr[i][j] = fmaf(ar[i], br[j], gr[i][j]);
                    gr[i][j] = fmaf(ai[i], bi[j], gr[i][j]);
                    gi[i][j] = fmaf(ar[i], bi[j], gi[i][j]);
                    gi[i][j] = fmaf(-ai[i], br[j], gi[i][j]);
                }
        }
        __syncthreads();
    }
    float out[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = n0 + ly + 16 * i;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = s0 + lx + 16 * j;
            float v;
            if (s >= S || n >= S) v = 0.f;
            else if (s == n) v = 1.f;
            else v = scale * fmaf(gr[i][j], gr[i][j], gi[i][j] * gi[i][j]);
            out[i][j] = v;
        }
    }
    if (!sym) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int n = n0 + ly + 16 * i;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int s = s0 + lx + 16 * j;
                if (n < S && s < lda) store_elem<OutT>(A, (size_t)n * lda + s, out[i][j]);
            }
        }
        return;
    }
    // symmetric: every pair (n, s) gets the value computed for n <= s
    float(*sT)[TN + 1] = reinterpret_cast<float(*)[TN + 1]>(sbuf);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sT[ly + 16 * i][lx + 16 * j] = out[i][j];
    __syncthreads();
    const bool diag = tx == ty;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int rl = ly + 16 * i, n = n0 + rl;
        if (n >= S) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int cl = lx + 16 * j, s = s0 + cl;
            if (s >= lda) continue;
            const float v = (diag && cl < rl) ? sT[cl][rl] : sT[rl][cl];
            store_elem<OutT>(A, (size_t)n * lda + s, v);
        }
    }
    if (!diag) {
        // the mirrored tile: A[s][n] = A[n][s]
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int rl = ly + 16 * i, s = s0 + rl;  // row of the mirrored tile
            if (s >= S) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cl = lx + 16 * j, n = n0 + cl;
                if (n < lda) store_elem<OutT>(A, (size_t)s * lda + n, sT[cl][rl]);
            }
        }
    }
}

}  // namespace

cudaError_t launch_psf_gram(const float *Lre, const float *Lim, const float *Rre, const float *Rim, int ldm, int M,
                            int S, float scale, void *A, int lda, int a_dtype, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    const bool symmetric = Lre == Rre && Lim == Rim;
    int sym = 0;
    dim3 grid;
    if (symmetric) {
        sym = (lda + TN - 1) / TN;  // square tiling covers every column up to lda
        grid = dim3(sym * (sym + 1) / 2, 1);
    } else {
        grid = dim3((lda + TN - 1) / TN, (S + TM - 1) / TM);
    }
    if (a_dtype == DAMAS_BF16)
        psf_gram_kernel<__nv_bfloat16><<<grid, 256, 0, st>>>(Lre, Lim, Rre, Rim, ldm, M, S, scale,
                                                             (__nv_bfloat16 *)A, lda, sym);
    else
        psf_gram_kernel<float><<<grid, 256, 0, st>>>(Lre, Lim, Rre, Rim, ldm, M, S, scale, (float *)A, lda, sym);
    return cudaGetLastError();
}
