// Cross-spectral matrix (Eq. (1)) estimated from microphone time series: blocks
// of K samples every `hop` samples, periodic Hann window w, the DFT of the
// selected bins, averaged over the L blocks (Welch):
//     X_lf[m] = sum_t w(t) p[m][l*hop + t] exp(-2 pi i bin_f t / K)
//     C_f     = sum_l X_lf X_lf^H / (L * sum_t w(t)^2).
//
// csm_twiddle_kernel: the table tw[t][2f] = w(t) cos, tw[t][2f+1] = -w(t) sin of
// the angle 2 pi ((bin_f * t) mod K) / K, the product reduced exactly in
// integers to a fraction of a period in [-1/2, 1/2] before an FP32 sine/cosine
// of pi times twice that fraction.
// csm_dft_kernel: X = blocks x table as a real product - rows are (block,
// microphone) pairs read straight from the overlapping blocks of p, columns
// are (bin, re/im) - 64 x 64 tiles on CUDA cores, FP32 accumulation, X stored
// as [L][F][M] complex.
// csm_accum_kernel: for every bin, the Hermitian sum over blocks of X X^H,
// 32 x 32 tiles of the upper triangle staged through shared memory; each value
// is written at (m, m') and conjugated at (m', m), so C is exactly Hermitian.
#include "common.cuh"

namespace {

__global__ void csm_twiddle_kernel(const int32_t *__restrict__ bins, int F, int K, float *__restrict__ tw) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)K * F) return;
    const int t = (int)(e / F), f = (int)(e % F);
    const long long b = ((long long)bins[f] % K + K) % K;
    // angles reduced exactly in integers to 2 pi q with q = r / K in [-1/2, 1/2]
    // (r, K < 2^24 are exact in FP32; the quotient is rounded once), then FP32
    // sine and cosine of pi * 2q
    long long r = (b * t) % K;
    if (2 * r > K) r -= K;
    const long long tt = 2 * t > K ? t - K : t;
    float s, c;
    sincospif(2.0f * __fdiv_rn((float)r, (float)K), &s, &c);
    const float w = __fmul_rn(0.5f, __fsub_rn(1.0f, cospif(2.0f * __fdiv_rn((float)tt, (float)K))));
    tw[(size_t)t * 2 * F + 2 * f] = __fmul_rn(w, c);
    tw[(size_t)t * 2 * F + 2 * f + 1] = -__fmul_rn(w, s);
}

constexpr int TR = 64, TC = 64, TKC = 32;

__global__ void __launch_bounds__(256) csm_dft_kernel(const float *__restrict__ p, int M, long long T, int K, int hop,
                                                      int L, int F, const float *__restrict__ tw,
                                                      float2 *__restrict__ X) {
    // staging of samples and table; reused for the output tile
    constexpr int STAGE = TKC * (TR + 4) + TKC * (TC + 4);
    static_assert(STAGE >= TR * (TC + 1), "output tile must fit the staging buffer");
    __shared__ float sbuf[STAGE];
    float(*sP)[TR + 4] = reinterpret_cast<float(*)[TR + 4]>(sbuf);
    float(*sT)[TC + 4] = reinterpret_cast<float(*)[TC + 4]>(sbuf + TKC * (TR + 4));
    const int r0 = blockIdx.y * TR, c0 = blockIdx.x * TC;
    const int nrows = M * L, ncols = 2 * F;
    const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int t0 = 0; t0 < K; t0 += TKC) {
        for (int e = threadIdx.x; e < TR * TKC; e += 256) {
            const int rr = e / TKC, k = e % TKC, r = r0 + rr, t = t0 + k;
            float v = 0.f;
            if (r < nrows && t < K) {
                const int l = r / M, m = r - l * M;
                v = p[(size_t)m * T + (size_t)l * hop + t];
            }
            sP[k][rr] = v;
        }
        for (int e = threadIdx.x; e < TKC * TC; e += 256) {
            const int k = e / TC, cc = e % TC, t = t0 + k, col = c0 + cc;
            sT[k][cc] = (t < K && col < ncols) ? tw[(size_t)t * ncols + col] : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int k = 0; k < TKC; ++k) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = sP[k][ly + 16 * i];
                b[i] = sT[k][lx + 16 * i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    // columns 2f and 2f+1 of a row are the re and im of X: lx and lx+16*j pair up
    // through shared memory
    float(*sOut)[TC + 1] = reinterpret_cast<float(*)[TC + 1]>(sbuf);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sOut[ly + 16 * i][lx + 16 * j] = acc[i][j];
    __syncthreads();
    for (int e = threadIdx.x; e < TR * (TC / 2); e += 256) {
        const int rr = e / (TC / 2), fc = e % (TC / 2), r = r0 + rr, f = c0 / 2 + fc;
        if (r >= nrows || f >= F) continue;
        const int l = r / M, m = r - l * M;
        X[((size_t)l * F + f) * M + m] = make_float2(sOut[rr][2 * fc], sOut[rr][2 * fc + 1]);
    }
}

constexpr int TA = 32, LCH = 32;

__global__ void __launch_bounds__(256) csm_accum_kernel(const float2 *__restrict__ X, int M, int L, int F,
                                                        float scale, int ntile, float *__restrict__ C) {
    __shared__ float2 sA[LCH][TA + 1], sB[LCH][TA + 1];
    const int f = blockIdx.y;
    // blockIdx.x enumerates the tiles (ti <= tj) of the upper triangle row by row
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int m0 = ti * TA, n0 = tj * TA;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // column tx, rows ty + 8 i
    float ar[4] = {0.f, 0.f, 0.f, 0.f}, ai[4] = {0.f, 0.f, 0.f, 0.f};
    for (int l0 = 0; l0 < L; l0 += LCH) {
        for (int e = threadIdx.x; e < LCH * TA; e += 256) {
            const int ll = e / TA, k = e % TA, l = l0 + ll;
            const bool okl = l < L;
            sA[ll][k] = (okl && m0 + k < M) ? X[((size_t)l * F + f) * M + m0 + k] : make_float2(0.f, 0.f);
            sB[ll][k] = (okl && n0 + k < M) ? X[((size_t)l * F + f) * M + n0 + k] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int ll = 0; ll < LCH; ++ll) {
            const float2 b = sB[ll][tx];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float2 a = sA[ll][ty + 8 * i];
                // a * conj(b)
                ar[i] = fmaf(a.x, b.x, fmaf(a.y, b.y, ar[i]));
                ai[i] = fmaf(a.y, b.x, fmaf(-a.x, b.y, ai[i]));
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 8 * i, n = n0 + tx;
        if (m >= M || n >= M || n < m) continue;
        const float re = scale * ar[i], im = m == n ? 0.f : scale * ai[i];
        C[2 * ((size_t)f * M * M + (size_t)m * M + n)] = re;
        C[2 * ((size_t)f * M * M + (size_t)m * M + n) + 1] = im;
        if (n != m) {
            C[2 * ((size_t)f * M * M + (size_t)n * M + m)] = re;
            C[2 * ((size_t)f * M * M + (size_t)n * M + m) + 1] = -im;
        }
    }
}

}  // namespace

size_t csm_work_floats(int M, int L, int F, int K) { return (size_t)K * 2 * F + (size_t)L * F * M * 2; }

cudaError_t launch_csm(const float *p, int M, long long T, int K, int hop, const int32_t *bins, int F, float *C,
                       float *work, cudaStream_t st) {
    const int L = (int)((T - K) / hop + 1);
    float *tw = work;
    float2 *X = reinterpret_cast<float2 *>(work + (size_t)K * 2 * F);
    const long long ntw = (long long)K * F;
    csm_twiddle_kernel<<<(unsigned)((ntw + 255) / 256), 256, 0, st>>>(bins, F, K, tw);
    const dim3 g1((2 * F + TC - 1) / TC, (unsigned)(((long long)M * L + TR - 1) / TR));
    csm_dft_kernel<<<g1, 256, 0, st>>>(p, M, T, K, hop, L, F, tw, X);
    double w2 = 0.0;
    for (int t = 0; t < K; ++t) {
        const double w = 0.5 - 0.5 * cos(2.0 * acos(-1.0) * t / K);
        w2 += w * w;
    }
    const int ntile = (M + TA - 1) / TA;
    const dim3 g2(ntile * (ntile + 1) / 2, F);
    csm_accum_kernel<<<g2, 256, 0, st>>>(X, M, L, F, (float)(1.0 / ((double)L * w2)), ntile, C);
    return cudaGetLastError();
}
