// Steering / propagation vectors of scan-grid points (§2 Eq. (4), §3 Eq. (7)).
//
// One warp per point, lanes over microphones.  The distance d and the phase
// k*d are formed in FP64: d^2 from the FP64 coordinate differences, then
// 1/d from an FP32 reciprocal-square-root seed y refined by one Newton step
// for x^-1/2, y' = y (3/2 - d^2 y^2 / 2), which takes the seed's relative error
// e (a few 1e-7) to about 1.5 e^2 (below 2e-13), and d = d^2 y'.  The phase is
// reduced to the fraction of a period t = d*f/c - rint(d*f/c) before an FP32
// sin/cos of 2*pi*t, so the FP32 part only sees an argument in [-pi, pi].
// FP64 serves the distance and the phase only: the amplitude |r|/d = |r| y' is
// an FP32 product of |r| and y' (rounded once), and ||g||^2 = sum_m (|r|/d_m)^2
// is a compensated FP32 sum (TwoProduct per term, TwoSum accumulation, the
// pairs carried through the warp reduction), accurate to about one FP32 ulp.
// Time convention exp(+j w t): a wave travelling distance d picks up
// exp(-j k d).
#include "common.cuh"

namespace {

// (h, l) += a * a, error-free up to the final rounding of l
__device__ __forceinline__ void acc_square(float &h, float &l, float a) {
    float p, pe, t;
    two_prod(a, a, p, pe);
    two_sum(h, p, h, t);
    l = __fadd_rn(l, __fadd_rn(t, pe));
}

// warp-wide sum of (h, l) pairs; every lane returns h + l
__device__ __forceinline__ float warp_sum_pair(float h, float l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
        float t;
        two_sum(h, h2, h, t);
        l = __fadd_rn(__fadd_rn(l, l2), t);
    }
    return __fadd_rn(h, l);
}

// Microphone m seen from point (px, py, pz): cos and sin of the phase
// 2 pi (d f / c), the distance d and its reciprocal (FP64).
__device__ __forceinline__ void mic_term(const GeomK &g, int m, double px, double py, double pz, float &c, float &s,
                                         double &d, double &inv_d) {
    const double ddx = px - g.mic[3 * m], ddy = py - g.mic[3 * m + 1], ddz = pz - g.mic[3 * m + 2];
    const double d2 = fma(ddx, ddx, fma(ddy, ddy, ddz * ddz));
    const double y = (double)rsqrtf((float)d2);
    inv_d = fma(0.5 * y, fma(-d2 * y, y, 1.0), y);
    d = d2 > 0.0 ? d2 * inv_d : 0.0;
    double t = d * g.f_over_c;
    t -= rint(t);
    sincospif(2.0f * (float)t, &s, &c);
}

constexpr int MAX_CACHED = 8;  // microphone terms per lane kept in registers (M <= 256)

// kind: 0 = L = g/||g|| (formulation E), 1 = L = v only, 2 = L = v and R = g (formulation P)
__global__ void __launch_bounds__(256) steer_kernel(GeomK g, int kind, const int32_t *__restrict__ idx, int n_pts,
                                                    float *__restrict__ Lre, float *__restrict__ Lim,
                                                    float *__restrict__ Rre, float *__restrict__ Rim, int ldm,
                                                    float *__restrict__ gnorm2) {
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (warp >= n_pts) return;
    const int n = idx ? idx[warp] : warp;
    const int ix = n % g.nx, iy = n / g.nx;
    const double px = g.x0 + ix * g.dx, py = g.y0 + iy * g.dy, pz = g.z;
    const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
    const float rabs = __fsqrt_rn(__fmaf_rn(pxf, pxf, __fmaf_rn(pyf, pyf, __fmul_rn(pzf, pzf))));

    // ||g||^2 = sum_m (|r| / d_m)^2; the terms of the first MAX_CACHED
    // microphones of this lane stay in registers for the output pass
    // (q = |r| / d, and d as FP32)
    float cc[MAX_CACHED], ss[MAX_CACHED], qq[MAX_CACHED], dd[MAX_CACHED];
    float g2h = 0.f, g2l = 0.f;
#pragma unroll
    for (int j = 0; j < MAX_CACHED; ++j) {
        const int m = lane + 32 * j;
        if (m < g.M) {
            double d, inv_d;
            mic_term(g, m, px, py, pz, cc[j], ss[j], d, inv_d);
            const float a = __fmul_rn(rabs, (float)inv_d);
            acc_square(g2h, g2l, a);
            qq[j] = a;
            dd[j] = (float)d;
        }
    }
    for (int m = lane + 32 * MAX_CACHED; m < g.M; m += 32) {
        float c, s;
        double d, inv_d;
        mic_term(g, m, px, py, pz, c, s, d, inv_d);
        acc_square(g2h, g2l, __fmul_rn(rabs, (float)inv_d));
    }
    const float g2 = warp_sum_pair(g2h, g2l);
    const float inv_norm_f = __frsqrt_rn(g2), inv_rabs = __frcp_rn(rabs);
    if (gnorm2 && lane == 0) gnorm2[warp] = g2;

    const size_t row = (size_t)warp * ldm;
    // q = |r| / d, dfl = d
    auto put = [&](int m, float c, float s, float q, float dfl) {
        if (kind == 0) {
            const float amp = q * inv_norm_f;
            Lre[row + m] = amp * c;
            Lim[row + m] = -amp * s;
        } else {
            const float av = dfl * inv_rabs;
            Lre[row + m] = av * c;
            Lim[row + m] = -av * s;
            if (kind == 2) {
                Rre[row + m] = q * c;
                Rim[row + m] = -q * s;
            }
        }
    };
#pragma unroll
    for (int j = 0; j < MAX_CACHED; ++j) {
        const int m = lane + 32 * j;
        if (m < g.M) put(m, cc[j], ss[j], qq[j], dd[j]);
    }
    for (int m = lane + 32 * MAX_CACHED; m < g.M; m += 32) {
        float c, s;
        double d, inv_d;
        mic_term(g, m, px, py, pz, c, s, d, inv_d);
        put(m, c, s, __fmul_rn(rabs, (float)inv_d), (float)d);
    }
    // zero padding of the plane rows
    for (int m = g.M + lane; m < ldm; m += 32) {
        Lre[row + m] = 0.f;
        Lim[row + m] = 0.f;
        if (kind == 2) {
            Rre[row + m] = 0.f;
            Rim[row + m] = 0.f;
        }
    }
}

}  // namespace

cudaError_t launch_steer(const GeomK &g, int kind, const int32_t *idx, int n, float *Lre, float *Lim, float *Rre,
                         float *Rim, int ldm, float *gnorm2, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 256, warps = threads / 32;
    const int blocks = (n + warps - 1) / warps;
    steer_kernel<<<blocks, threads, 0, st>>>(g, kind, idx, n, Lre, Lim, Rre, Rim, ldm, gnorm2);
    return cudaGetLastError();
}
