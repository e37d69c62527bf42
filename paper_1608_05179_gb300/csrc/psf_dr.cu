// Diagonal removal (§2: the auto-spectra on the CSM diagonal are dropped to
// suppress uncorrelated self-noise).  The PSF then leaves out the m = m'
// microphone pairs:
//     A_ns = scale * ( |sum_m conj(l_nm) r_sm|^2 - sum_m |l_nm|^2 |r_sm|^2 ),
// the first term being the PSF the tensor-core Gram already wrote.  Its
// diagonal d_n is not 1, so the matrix is rescaled to a unit diagonal,
// A'_ns = A_ns / (sqrt(d_n) sqrt(d_s)), which leaves the clamped iteration of
// Eq. (14) unchanged step for step (x = x' / sqrt(d)).
//
// dr_diag_kernel: one warp per point, d_n from the FP32 vectors as compensated
// FP32 sums (TwoProduct terms, TwoSum accumulation, pairs through the warp
// reduction; d_n is about 1 - 1/M, far from cancellation), out as sqrt(d_n).  dr_correct_kernel: the pair correction is a real Gram product of
// the squared magnitudes, 64 x 64 output tiles on CUDA cores (K = microphones
// staged through shared memory), fused with the rescaling and written in place;
// every entry is read and written by one thread, and the FMA order is the same
// for (n, s) and (s, n), so a symmetric A stays exactly symmetric.
#include "common.cuh"

namespace {

// (h, l) += a * b, error-free up to the final rounding of l
__device__ __forceinline__ void acc_prod(float &h, float &l, float a, float b) {
    float p, pe, t;
    two_prod(a, b, p, pe);
    two_sum(h, p, h, t);
    l = __fadd_rn(l, __fadd_rn(t, pe));
}

// (h, l) summed over the warp, returned as h + l on every lane
__device__ __forceinline__ float warp_pair_sum(float h, float l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
        float t;
        two_sum(h, h2, h, t);
        l = __fadd_rn(__fadd_rn(l, l2), t);
    }
    return __fadd_rn(h, l);
}

__global__ void __launch_bounds__(256) dr_diag_kernel(const float *__restrict__ Lre, const float *__restrict__ Lim,
                                                      const float *__restrict__ Rre, const float *__restrict__ Rim,
                                                      int ldm, int M, int S, float scale,
                                                      float *__restrict__ dscale) {
    const int lane = threadIdx.x & 31;
    const int n = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (n >= S) return;
    float grh = 0.f, grl = 0.f, gih = 0.f, gil = 0.f, th = 0.f, tl = 0.f;
    for (int m = lane; m < M; m += 32) {
        const size_t o = (size_t)n * ldm + m;
        const float lr = Lre[o], li = Lim[o], rr = Rre[o], ri = Rim[o];
        acc_prod(grh, grl, lr, rr);  // Re conj(l) r = lr rr + li ri
        acc_prod(grh, grl, li, ri);
        acc_prod(gih, gil, lr, ri);  // Im conj(l) r = lr ri - li rr
        acc_prod(gih, gil, -li, rr);
        acc_prod(th, tl, __fmaf_rn(lr, lr, __fmul_rn(li, li)), __fmaf_rn(rr, rr, __fmul_rn(ri, ri)));
    }
    const float gr = warp_pair_sum(grh, grl), gi = warp_pair_sum(gih, gil), t = warp_pair_sum(th, tl);
    if (lane == 0) {
        // |G|^2 - t with the squares error-free and one compensated sum
        float p1, e1, p2, e2, s1, e3, s2, e4;
        two_prod(gr, gr, p1, e1);
        two_prod(gi, gi, p2, e2);
        two_sum(p1, p2, s1, e3);
        two_sum(s1, -t, s2, e4);
        const float d = __fadd_rn(s2, __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(e3, e4)));
        dscale[n] = __fsqrt_rn(fmaxf(__fmul_rn(scale, d), 0.f));
    }
}

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) dr_correct_kernel(const float *__restrict__ Lre, const float *__restrict__ Lim,
                                                         const float *__restrict__ Rre, const float *__restrict__ Rim,
                                                         int ldm, int M, int S, float scale,
                                                         const float *__restrict__ dscale, float *__restrict__ A,
                                                         int lda) {
    __shared__ float sP[TK][TM + 4], sQ[TK][TN + 4];
    const int n0 = blockIdx.y * TM, s0 = blockIdx.x * TN;
    const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int m0 = 0; m0 < M; m0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            const int r = e / TK, k = e % TK, m = m0 + k;
            const int n = n0 + r, s = s0 + r;
            float p = 0.f, q = 0.f;
            if (m < M && n < S) {
                const float a = Lre[(size_t)n * ldm + m], b = Lim[(size_t)n * ldm + m];
                p = fmaf(a, a, b * b);
            }
            if (m < M && s < S) {
                const float a = Rre[(size_t)s * ldm + m], b = Rim[(size_t)s * ldm + m];
                q = fmaf(a, a, b * b);
            }
            sP[k][r] = p;
            sQ[k][r] = q;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TK; ++k) {
            float p[4], q[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                p[i] = sP[k][ly + 16 * i];
                q[i] = sQ[k][lx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(p[i], q[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int n = n0 + ly + 16 * i;
        if (n >= S) continue;
        const float dn = dscale[n];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int s = s0 + lx + 16 * j;
            if (s >= S) continue;
            const size_t o = (size_t)n * lda + s;
            A[o] = s == n ? 1.f : (A[o] - scale * acc[i][j]) / (dn * dscale[s]);
        }
    }
}

__global__ void divide_kernel(float *__restrict__ v, const float *__restrict__ d, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = v[i] / d[i];
}

}  // namespace

cudaError_t launch_psf_dr(const float *Lre, const float *Lim, const float *Rre, const float *Rim, int ldm, int M,
                          int S, float scale, float *A, int lda, float *dscale, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    dr_diag_kernel<<<(unsigned)(((size_t)S * 32 + 255) / 256), 256, 0, st>>>(Lre, Lim, Rre, Rim, ldm, M, S,
                                                                             scale, dscale);
    const dim3 grid((S + TN - 1) / TN, (S + TM - 1) / TM);
    dr_correct_kernel<<<grid, 256, 0, st>>>(Lre, Lim, Rre, Rim, ldm, M, S, scale, dscale, A, lda);
    return cudaGetLastError();
}

cudaError_t launch_divide(float *v, const float *d, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    divide_kernel<<<(n + 255) / 256, 256, 0, st>>>(v, d, n);
    return cudaGetLastError();
}
