// Steering / propagation vectors of scan-grid points (§2 Eq. (4), §3 Eq. (7)).
//
// One warp per point, lanes over microphones.  Distances and the phase k*d
// are formed in FP64; the phase is reduced to the fraction of a period
// t = d*f/c - rint(d*f/c) before an FP32 sin/cos of 2*pi*t, so the FP32 part
// only sees an argument in [-pi, pi].  Time convention exp(+j w t): a wave
// travelling distance d picks up exp(-j k d).
#include "common.cuh"

namespace {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

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
    const double rabs = sqrt(px * px + py * py + pz * pz);

    // ||g||^2 = sum_m (|r| / d_m)^2
    double g2 = 0.0;
    for (int m = lane; m < g.M; m += 32) {
        const double ddx = px - g.mic[3 * m], ddy = py - g.mic[3 * m + 1], ddz = pz - g.mic[3 * m + 2];
        const double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
        const double a = rabs / d;
        g2 += a * a;
    }
    g2 = warp_sum_d(g2);
    const double inv_norm = 1.0 / sqrt(g2);
    if (gnorm2 && lane == 0) gnorm2[warp] = (float)g2;

    const size_t row = (size_t)warp * ldm;
    for (int m = lane; m < ldm; m += 32) {
        if (m >= g.M) {  // zero padding of the plane rows
            Lre[row + m] = 0.f;
            Lim[row + m] = 0.f;
            if (kind == 2) {
                Rre[row + m] = 0.f;
                Rim[row + m] = 0.f;
            }
            continue;
        }
        const double ddx = px - g.mic[3 * m], ddy = py - g.mic[3 * m + 1], ddz = pz - g.mic[3 * m + 2];
        const double d = sqrt(ddx * ddx + ddy * ddy + ddz * ddz);
        double t = d * g.f_over_c;
        t -= rint(t);
        float s, c;
        sincospif(2.0f * (float)t, &s, &c);
        if (kind == 0) {
            const float amp = (float)((rabs / d) * inv_norm);
            Lre[row + m] = amp * c;
            Lim[row + m] = -amp * s;
        } else {
            const float av = (float)(d / rabs);
            Lre[row + m] = av * c;
            Lim[row + m] = -av * s;
            if (kind == 2) {
                const float ag = (float)(rabs / d);
                Rre[row + m] = ag * c;
                Rim[row + m] = -ag * s;
            }
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
