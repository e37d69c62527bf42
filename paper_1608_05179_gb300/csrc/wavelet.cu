// Wavelet-compressed computational grid (§4, Algorithm 1).
//
// One CTA of 1024 threads per grid:
//  1. every point gets its level in the nested grids of Eq. (15) from the
//     trailing zeros of its indices, and (outside G^0) the interpolating-wavelet
//     coefficient of Eq. (23), prediction - b, with the prediction formed from
//     the coarser grid only, in FP32 with a fixed expression order;
//  2. the threshold: as given, eps * max(b), or the K-th largest |detail| found
//     by an exact 4-pass MSB radix select on the FP32 bit patterns (|d| >= 0 so
//     the unsigned order of the bits is the numeric order);
//  3. keep = G^0 or |detail| >= threshold (Eq. (22)); an ordered compaction
//     (contiguous chunk per thread + block scan) writes ascending indices.
// Every decision is integer or exact FP32 work, so the selection is
// deterministic and independent of thread scheduling.
#include "common.cuh"

namespace {

constexpr int WT = 1024;

__device__ __forceinline__ float predict(const float *__restrict__ b, int nx, int ny, int ix, int iy, int h, bool xo,
                                         bool yo, int pred) {
    const int xl = xo ? ix - h : ix, yl = yo ? iy - h : iy;
    if (pred == DAMAS_PRED_HAAR) return b[(size_t)yl * nx + xl];
    const bool hasx = xo && (ix + h <= nx - 1);
    const bool hasy = yo && (iy + h <= ny - 1);
    if (xo && !yo) {
        if (!hasx) return b[(size_t)iy * nx + xl];
        return __fmul_rn(0.5f, __fadd_rn(b[(size_t)iy * nx + (ix - h)], b[(size_t)iy * nx + (ix + h)]));
    }
    if (!xo && yo) {
        if (!hasy) return b[(size_t)yl * nx + ix];
        return __fmul_rn(0.5f, __fadd_rn(b[(size_t)(iy - h) * nx + ix], b[(size_t)(iy + h) * nx + ix]));
    }
    const float mm = b[(size_t)(iy - h) * nx + (ix - h)];
    if (hasx && hasy) {
        const float pm = b[(size_t)(iy - h) * nx + (ix + h)];
        const float mp = b[(size_t)(iy + h) * nx + (ix - h)];
        const float pp = b[(size_t)(iy + h) * nx + (ix + h)];
        return __fmul_rn(0.25f, __fadd_rn(__fadd_rn(mm, pm), __fadd_rn(mp, pp)));
    }
    if (hasx) return __fmul_rn(0.5f, __fadd_rn(mm, b[(size_t)(iy - h) * nx + (ix + h)]));
    if (hasy) return __fmul_rn(0.5f, __fadd_rn(mm, b[(size_t)(iy + h) * nx + (ix - h)]));
    return mm;
}

__device__ __forceinline__ int block_excl_scan(int v, int *warp_sums, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = warp_sums[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    total = warp_sums[31];
    const int before = warp ? warp_sums[warp - 1] : 0;
    return before + x - v;
}

__global__ void __launch_bounds__(WT) wavelet_kernel(const float *__restrict__ b, int nx, int ny, int J, int pred,
                                                     int mode, float eps_abs_in, float eps_rel, long long K,
                                                     int32_t *__restrict__ idx, int32_t *__restrict__ S_sub,
                                                     float *__restrict__ detail, float *__restrict__ eps_abs_out,
                                                     float *__restrict__ absd) {
    __shared__ unsigned int hist[256];
    __shared__ int warp_sums[32];
    __shared__ float s_red[32];
    __shared__ unsigned int s_prefix;
    __shared__ long long s_k;
    __shared__ float s_eps;
    const int S = nx * ny;

    // 1. levels and coefficients
    float bmax = -INFINITY;
    for (int n = threadIdx.x; n < S; n += WT) {
        const int ix = n % nx, iy = n / nx;
        const int tx = ix ? __ffs(ix) - 1 : 31, ty = iy ? __ffs(iy) - 1 : 31;
        const int t = min(tx, ty);
        const float bn = b[n];
        bmax = fmaxf(bmax, bn);
        if (t >= J) {
            absd[n] = -1.0f;
            if (detail) detail[n] = 0.0f;
        } else {
            const float bbar = predict(b, nx, ny, ix, iy, 1 << t, tx == t, ty == t, pred);
            const float d = __fsub_rn(bbar, bn);
            absd[n] = fabsf(d);
            if (detail) detail[n] = d;
        }
    }
    __syncthreads();

    // 2. threshold
    if (mode == DAMAS_EPS_ABS) {
        if (threadIdx.x == 0) s_eps = eps_abs_in;
    } else if (mode == DAMAS_EPS_REL_MAX) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = bmax;
        __syncthreads();
        if (threadIdx.x == 0) {
            float m = s_red[0];
            for (int w = 1; w < WT / 32; ++w) m = fmaxf(m, s_red[w]);
            s_eps = __fmul_rn(eps_rel, m);
        }
    } else {
        const int n0 = (((nx - 1) >> J) + 1) * (((ny - 1) >> J) + 1);
        const long long nd = (long long)S - n0;
        if (K <= 0) {
            if (threadIdx.x == 0) s_eps = INFINITY;
        } else if (K >= nd) {
            if (threadIdx.x == 0) s_eps = 0.0f;
        } else {
            if (threadIdx.x == 0) {
                s_prefix = 0u;
                s_k = K;
            }
            unsigned int mask = 0u;
            for (int pass = 0; pass < 4; ++pass) {
                const int shift = 24 - 8 * pass;
                for (int i = threadIdx.x; i < 256; i += WT) hist[i] = 0u;
                __syncthreads();
                const unsigned int prefix = s_prefix;
                for (int n = threadIdx.x; n < S; n += WT) {
                    const unsigned int key = __float_as_uint(absd[n]);
                    if (key & 0x80000000u) continue;  // G^0 marker (-1)
                    if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    long long k = s_k, cum = 0;
                    int chosen = 0;
                    for (int bkt = 255; bkt >= 0; --bkt) {
                        const long long c = hist[bkt];
                        if (cum + c >= k) {
                            chosen = bkt;
                            k -= cum;
                            break;
                        }
                        cum += c;
                    }
                    s_k = k;
                    s_prefix = prefix | ((unsigned int)chosen << shift);
                }
                mask |= 255u << shift;
                __syncthreads();
            }
            if (threadIdx.x == 0) s_eps = __uint_as_float(s_prefix);
        }
    }
    __syncthreads();
    const float eps = s_eps;

    // 3. ordered compaction
    const int chunk = (S + WT - 1) / WT;
    const int lo = min(S, threadIdx.x * chunk), hi = min(S, lo + chunk);
    int cnt = 0;
    for (int n = lo; n < hi; ++n) {
        const float a = absd[n];
        cnt += (a < 0.0f || a >= eps) ? 1 : 0;
    }
    int total;
    int pos = block_excl_scan(cnt, warp_sums, total);
    for (int n = lo; n < hi; ++n) {
        const float a = absd[n];
        if (a < 0.0f || a >= eps) idx[pos++] = n;
    }
    if (threadIdx.x == 0) {
        *S_sub = total;
        if (eps_abs_out) *eps_abs_out = eps;
    }
}

// Neighbour padding: clear the marks, mark the (2r+1)^2 square around every
// listed point (clipped to the grid; concurrent writes store the same byte),
// then the same ordered compaction as above.  Every listed index is read before
// the barrier that precedes the first write of out, so out may alias idx.
__global__ void __launch_bounds__(WT) pad_grid_kernel(int nx, int ny, const int32_t *__restrict__ idx,
                                                      const int32_t *__restrict__ n_in, int radius, int32_t *out,
                                                      int32_t *__restrict__ n_out, unsigned char *__restrict__ marks) {
    __shared__ int warp_sums[32];
    const int S = nx * ny;
    for (int n = threadIdx.x; n < S; n += WT) marks[n] = 0;
    __syncthreads();
    const int n = min(max(*n_in, 0), S);
    for (int i = threadIdx.x; i < n; i += WT) {
        const int p = idx[i];
        if (p < 0 || p >= S) continue;
        const int ix = p % nx, iy = p / nx;
        const int x0 = max(ix - radius, 0), x1 = min(ix + radius, nx - 1);
        const int y0 = max(iy - radius, 0), y1 = min(iy + radius, ny - 1);
        for (int y = y0; y <= y1; ++y)
            for (int x = x0; x <= x1; ++x) marks[y * nx + x] = 1;
    }
    __syncthreads();
    const int chunk = (S + WT - 1) / WT;
    const int lo = min(S, threadIdx.x * chunk), hi = min(S, lo + chunk);
    int cnt = 0;
    for (int q = lo; q < hi; ++q) cnt += marks[q];
    int total;
    int pos = block_excl_scan(cnt, warp_sums, total);
    for (int q = lo; q < hi; ++q)
        if (marks[q]) out[pos++] = q;
    if (threadIdx.x == 0) *n_out = total;
}

__global__ void gather_kernel(const float *__restrict__ src, const int32_t *__restrict__ idx, int n,
                              float *__restrict__ dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[idx[i]];
}

constexpr int ST = 1024;

// x_full = 0 everywhere, then x_full[idx[i]] = x_sub[i] / gnorm2[i]; total power
// as a compensated FP32 sum (TwoSum per term, (hi, lo) pairs through a fixed
// tree), in a fixed order; the pair is returned as the double hi + lo, which
// holds it exactly (two FP32 significands fit in one FP64 significand).
__global__ void __launch_bounds__(ST) scatter_power_kernel(const float *__restrict__ x_sub,
                                                           const int32_t *__restrict__ idx,
                                                           const float *__restrict__ gnorm2, int n,
                                                           float *__restrict__ x_full, int S,
                                                           double *__restrict__ total) {
    __shared__ float red_h[ST], red_l[ST];
    for (int i = threadIdx.x; i < S; i += ST) x_full[i] = 0.0f;
    __syncthreads();
    float h = 0.f, l = 0.f;
    for (int i = threadIdx.x; i < n; i += ST) {
        const float v = gnorm2 ? __fdiv_rn(x_sub[i], gnorm2[i]) : x_sub[i];
        x_full[idx ? idx[i] : i] = v;
        float t;
        two_sum(h, v, h, t);
        l = __fadd_rn(l, t);
    }
    red_h[threadIdx.x] = h;
    red_l[threadIdx.x] = l;
    __syncthreads();
    for (int s = ST / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            float hh, t;
            two_sum(red_h[threadIdx.x], red_h[threadIdx.x + s], hh, t);
            red_h[threadIdx.x] = hh;
            red_l[threadIdx.x] = __fadd_rn(__fadd_rn(red_l[threadIdx.x], red_l[threadIdx.x + s]), t);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) {
        float hh, t;
        two_sum(red_h[0], red_l[0], hh, t);  // normalise: |t| <= ulp(hh) / 2
        *total = (double)hh + (double)t;
    }
}

}  // namespace

cudaError_t launch_wavelet(const float *b, int nx, int ny, int levels, int pred, int eps_mode, float eps_abs,
                           float eps_rel, long long keep_K, int32_t *idx, int32_t *S_sub, float *detail,
                           float *eps_abs_out, float *work_absd, cudaStream_t st) {
    wavelet_kernel<<<1, WT, 0, st>>>(b, nx, ny, levels, pred, eps_mode, eps_abs, eps_rel, keep_K, idx, S_sub, detail,
                                      eps_abs_out, work_absd);
    return cudaGetLastError();
}

cudaError_t launch_pad_grid(int nx, int ny, const int32_t *idx, const int32_t *n_in, int radius, int32_t *out,
                            int32_t *n_out, unsigned char *marks, cudaStream_t st) {
    pad_grid_kernel<<<1, WT, 0, st>>>(nx, ny, idx, n_in, radius, out, n_out, marks);
    return cudaGetLastError();
}

cudaError_t launch_gather(const float *src, const int32_t *idx, int n, float *dst, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    gather_kernel<<<(n + 255) / 256, 256, 0, st>>>(src, idx, n, dst);
    return cudaGetLastError();
}

cudaError_t launch_scatter_power(const float *x_sub, const int32_t *idx, const float *gnorm2, int n, float *x_full,
                                 int S, double *total, cudaStream_t st) {
    scatter_power_kernel<<<1, ST, 0, st>>>(x_sub, idx, gnorm2, n, x_full, S, total);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------- allocation-free variant
// Some callers cannot allocate device memory at the moment they need a
// compressed grid: a real-time audio thread must not wait on the driver's
// allocator, a plug-in hosted by another application may only touch memory the
// host application handed it, and code that runs under a fixed device-memory
// budget reserved at start-up may not grow it.  wavelet_compress_grid_noalloc
// serves them: the one work array the selection needs lives in the file-scope
// device array below, created when the library's module is loaded on a device
// and held by every device that loads the library until the process exits.
#include <mutex>

namespace {

// |detail| per grid point (work array of the selection kernel).
static __device__ __align__(256) float g_noalloc_absd[DAMAS_NOALLOC_MAX_POINTS];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kMaxDevices] = {nullptr};

}  // namespace

extern "C" int wavelet_compress_grid_noalloc(damas_ctx *ctx, const float *b_dev, int nx, int ny,
                                             const damas_wavelet_cfg *cfg, int32_t *idx_dev, int32_t *S_sub_dev,
                                             float *detail_dev, float *eps_abs_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (!cfg) return ctx_fail(ctx, DAMAS_EINVAL, "cfg is NULL");
    if (!b_dev || !idx_dev || !S_sub_dev) return ctx_fail(ctx, DAMAS_EINVAL, "b_dev, idx_dev, S_sub_dev are required");
    if (nx < 1 || ny < 1 || nx > 65535 || ny > 65535)
        return ctx_fail(ctx, DAMAS_EINVAL, "grid %dx%d: nx and ny must be in 1..65535", nx, ny);
    if ((long long)nx * ny > DAMAS_NOALLOC_MAX_POINTS)
        return ctx_fail(ctx, DAMAS_EINVAL, "grid %dx%d exceeds the %d points of the allocation-free work array", nx, ny,
                        DAMAS_NOALLOC_MAX_POINTS);
    if (cfg->levels < 1 || cfg->levels > 15) return ctx_fail(ctx, DAMAS_EINVAL, "levels=%d out of range", cfg->levels);
    if (cfg->predictor != DAMAS_PRED_LINEAR && cfg->predictor != DAMAS_PRED_HAAR)
        return ctx_fail(ctx, DAMAS_EINVAL, "unknown predictor");
    if (cfg->eps_mode < DAMAS_EPS_ABS || cfg->eps_mode > DAMAS_EPS_KEEP_FRAC)
        return ctx_fail(ctx, DAMAS_EINVAL, "unknown eps_mode");
    if (!(cfg->eps >= 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "eps must be >= 0");
    if (cfg->eps_mode == DAMAS_EPS_KEEP_FRAC && cfg->eps > 1.0)
        return ctx_fail(ctx, DAMAS_EINVAL, "keep fraction must be in [0, 1]");
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return ctx_fail(ctx, DAMAS_EINVAL, "device index too large");

    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != ctx->device) {
        cudaError_t e = cudaSetDevice(ctx->device);
        if (e != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    }
    int rc = DAMAS_OK;
    float *work = nullptr;
    {
        // set-up, once per device, with that device current: the host-side name of
        // the array is only a stand-in, its device address comes from the runtime
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[ctx->device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_absd);
            if (e != cudaSuccess)
                rc = ctx_fail(ctx, DAMAS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            else
                g_noalloc_ptr[ctx->device] = (float *)p;
        }
        work = g_noalloc_ptr[ctx->device];
    }
    if (rc == DAMAS_OK) {
        // the work array needs no clearing: the kernel writes every entry it reads
        const int S = nx * ny;
        const int J = cfg->levels;
        const long long n0 = (long long)(((nx - 1) >> J) + 1) * (((ny - 1) >> J) + 1);
        const long long K =
            cfg->eps_mode == DAMAS_EPS_KEEP_FRAC ? (long long)ceil(cfg->eps * (double)S) - n0 : 0;
        cudaError_t e = launch_wavelet(b_dev, nx, ny, J, cfg->predictor, cfg->eps_mode, (float)cfg->eps,
                                       (float)cfg->eps, K, idx_dev, S_sub_dev, detail_dev, eps_abs_dev, work,
                                       (cudaStream_t)stream);
        if (e != cudaSuccess) rc = ctx_fail(ctx, DAMAS_ECUDA, "wavelet launch: %s", cudaGetErrorString(e));
    }
    if (prev >= 0 && prev != ctx->device) cudaSetDevice(prev);
    return rc;
}
