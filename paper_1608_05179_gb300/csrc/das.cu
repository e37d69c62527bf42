// Mean-square DAS map (§2 Eq. (2)): b_n = scale * Re(l_n^H C l_n); with diagonal
// removal (§2) the terms of the CSM diagonal are left out.
//
// Each warp takes PPW grid points: the points' vectors l_n are put in shared
// memory, lane p forms (C l_n)_p for p = lane, lane+32, ... from the CTA's copy
// of C (two interleaved partial sums per component to halve the dependent FMA
// chain), multiplies by conj(l_np) and the warp sums.  C is staged in chunks of
// rows so any M <= 256 fits in shared memory.  PPW is chosen so the grid has at
// least two CTAs per SM.  FP32 arithmetic.
#include "common.cuh"

namespace {

constexpr int DAS_THREADS = 256, DAS_WARPS = DAS_THREADS / 32, ROWS_PER_CHUNK = 64;

template <int PPW>
__global__ void __launch_bounds__(DAS_THREADS) das_kernel(const float *__restrict__ Lre, const float *__restrict__ Lim,
                                                          int ldm, int M, int S, const float2 *__restrict__ C,
                                                          float scale, float *__restrict__ b, int dr) {
    extern __shared__ float2 sm[];
    const int cstride = M + 1;                       // padded row stride of the C chunk (float2)
    float2 *sC = sm;                                 // ROWS_PER_CHUNK x cstride
    float2 *sl = sm + ROWS_PER_CHUNK * cstride;      // DAS_WARPS x PPW x M
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int base = (blockIdx.x * DAS_WARPS + warp) * PPW;

    // stage this warp's point vectors
#pragma unroll
    for (int q = 0; q < PPW; ++q) {
        const int n = base + q;
        float2 *dst = sl + (size_t)(warp * PPW + q) * M;
        for (int m = lane; m < M; m += 32)
            dst[m] = (n < S) ? make_float2(Lre[(size_t)n * ldm + m], Lim[(size_t)n * ldm + m]) : make_float2(0.f, 0.f);
    }
    float acc[PPW];
#pragma unroll
    for (int q = 0; q < PPW; ++q) acc[q] = 0.f;

    for (int p0 = 0; p0 < M; p0 += ROWS_PER_CHUNK) {
        const int rows = min(ROWS_PER_CHUNK, M - p0);
        __syncthreads();
        for (int e = threadIdx.x; e < rows * M; e += DAS_THREADS) {
            const int r = e / M, c = e % M;
            // diagonal removal: the CSM diagonal enters as zero
            sC[r * cstride + c] = (dr && c == p0 + r) ? make_float2(0.f, 0.f) : C[(size_t)(p0 + r) * M + c];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < PPW; ++q) {
            const float2 *l = sl + (size_t)(warp * PPW + q) * M;
            float a = acc[q];
            for (int r = lane; r < rows; r += 32) {
                const float2 *crow = sC + r * cstride;
                float yr0 = 0.f, yi0 = 0.f, yr1 = 0.f, yi1 = 0.f;
                int c = 0;
#pragma unroll 4
                for (; c + 1 < M; c += 2) {
                    const float2 cv0 = crow[c], lv0 = l[c], cv1 = crow[c + 1], lv1 = l[c + 1];
                    yr0 = fmaf(cv0.x, lv0.x, fmaf(-cv0.y, lv0.y, yr0));
                    yi0 = fmaf(cv0.x, lv0.y, fmaf(cv0.y, lv0.x, yi0));
                    yr1 = fmaf(cv1.x, lv1.x, fmaf(-cv1.y, lv1.y, yr1));
                    yi1 = fmaf(cv1.x, lv1.y, fmaf(cv1.y, lv1.x, yi1));
                }
                if (c < M) {
                    const float2 cv = crow[c], lv = l[c];
                    yr0 = fmaf(cv.x, lv.x, fmaf(-cv.y, lv.y, yr0));
                    yi0 = fmaf(cv.x, lv.y, fmaf(cv.y, lv.x, yi0));
                }
                const float yr = yr0 + yr1, yi = yi0 + yi1;
                const float2 lp = l[p0 + r];
                // Re(conj(l_p) * y_p) = lr*yr + li*yi
                a = fmaf(lp.x, yr, fmaf(lp.y, yi, a));
            }
            acc[q] = a;
        }
    }
#pragma unroll
    for (int q = 0; q < PPW; ++q) {
        float v = acc[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int n = base + q;
        if (lane == 0 && n < S) b[n] = scale * v;
    }
}

template <int PPW>
cudaError_t launch_das_ppw(const float *Lre, const float *Lim, int ldm, int M, int S, const float *C, float scale,
                           float *b, int dr, cudaStream_t st) {
    const size_t smem = sizeof(float2) * ((size_t)ROWS_PER_CHUNK * (M + 1) + (size_t)DAS_WARPS * PPW * M);
    cudaError_t e = cudaFuncSetAttribute(das_kernel<PPW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int pts_per_cta = DAS_WARPS * PPW;
    const int blocks = (S + pts_per_cta - 1) / pts_per_cta;
    das_kernel<PPW><<<blocks, DAS_THREADS, smem, st>>>(Lre, Lim, ldm, M, S, (const float2 *)C, scale, b, dr);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_das(const float *Lre, const float *Lim, int ldm, int M, int S, const float *C, float scale,
                       float *b, int dr, cudaStream_t st) {
    if (S <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    // the most points per warp that still gives two CTAs per SM
    const long long want = 2LL * sms * DAS_WARPS;
    if ((long long)S >= 4 * want) return launch_das_ppw<4>(Lre, Lim, ldm, M, S, C, scale, b, dr, st);
    if ((long long)S >= 2 * want) return launch_das_ppw<2>(Lre, Lim, ldm, M, S, C, scale, b, dr, st);
    return launch_das_ppw<1>(Lre, Lim, ldm, M, S, C, scale, b, dr, st);
}
