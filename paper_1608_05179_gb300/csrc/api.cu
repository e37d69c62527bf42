// C ABI of libdamas.so: argument checks, scratch management and launches.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "common.cuh"
#include "sweep.cuh"

// ----------------------------------------------------------------------------- context helpers
int ctx_fail(damas_ctx *ctx, int code, const char *fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

// Device memory the context holds as scratch.
size_t ctx_scratch_bytes(const damas_ctx *ctx) {
    return ctx->planes.cap + ctx->wave.cap + ctx->solve.cap + ctx->status.cap + ctx->misc.cap + ctx->pad.cap +
           ctx->probe.cap + ctx->kstat.cap;
}

int ctx_ensure(damas_ctx *ctx, ScratchBuf &b, size_t bytes) {
    if (bytes <= b.cap) return DAMAS_OK;
    {
        const size_t cap = (std::max(bytes, (size_t)1 << 20) + 4095) / 4096 * 4096;
        const size_t others = ctx_scratch_bytes(ctx) - b.cap;
        if (ctx->hbm_budget && others + cap > ctx->hbm_budget)
            return ctx_fail(ctx, DAMAS_ENOMEM, "scratch of %zu bytes would take the context to %zu bytes, above its budget of %zu",
                            cap, others + cap, ctx->hbm_budget);
    }
    if (b.ptr) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "sync before scratch growth: %s", cudaGetErrorString(e));
        cudaFree(b.ptr);
        b.ptr = nullptr;
        b.cap = 0;
    }
    size_t cap = std::max(bytes, (size_t)1 << 20);
    cap = (cap + 4095) / 4096 * 4096;
    if (cudaMalloc(&b.ptr, cap) != cudaSuccess) {
        cudaGetLastError();
        return ctx_fail(ctx, DAMAS_ENOMEM, "scratch allocation of %zu bytes failed", cap);
    }
    b.cap = cap;
    return DAMAS_OK;
}

namespace {

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }


struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int check_geom(damas_ctx *ctx, const damas_geom *g) {
    if (!g) return ctx_fail(ctx, DAMAS_EINVAL, "geom is NULL");
    if (g->M < 1 || g->M > DAMAS_MAX_MICS) return ctx_fail(ctx, DAMAS_EINVAL, "M=%d out of range", g->M);
    if (!g->mic_xyz_dev) return ctx_fail(ctx, DAMAS_EINVAL, "mic_xyz_dev is NULL");
    if (g->nx < 1 || g->ny < 1 || (long long)g->nx * g->ny > (1ll << 26))
        return ctx_fail(ctx, DAMAS_EINVAL, "grid %dx%d out of range", g->nx, g->ny);
    if (!(g->c > 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "speed of sound must be positive");
    if (g->formulation != DAMAS_FORM_E && g->formulation != DAMAS_FORM_P)
        return ctx_fail(ctx, DAMAS_EINVAL, "unknown formulation %d", g->formulation);
    if (g->diag_removal != 0 && g->diag_removal != 1)
        return ctx_fail(ctx, DAMAS_EINVAL, "diag_removal must be 0 or 1");
    if (g->diag_removal && g->M < 2) return ctx_fail(ctx, DAMAS_EINVAL, "diagonal removal needs M >= 2");
    return DAMAS_OK;
}

GeomK to_kernel(const damas_geom *g, double f) {
    GeomK k;
    k.mic = g->mic_xyz_dev;
    k.M = g->M;
    k.nx = g->nx;
    k.ny = g->ny;
    k.x0 = g->x0;
    k.y0 = g->y0;
    k.dx = g->dx;
    k.dy = g->dy;
    k.z = g->z;
    k.f_over_c = f / g->c;
    k.form = g->formulation;
    return k;
}

inline int planes_ld(int M) { return round_up(M, 16); }  // whole 16-microphone chunks for the Gram

// The context's build status word (device int, zero until a build kernel's
// bounded wait runs out); allocated and cleared on first use.
int ctx_kstat(damas_ctx *ctx, int **out) {
    if (!ctx->kstat.ptr) {
        int rc = ctx_ensure(ctx, ctx->kstat, 256);
        if (rc) return rc;
        DAMAS_CUDA_TRY(ctx, cudaMemset(ctx->kstat.ptr, 0, ctx->kstat.cap));
    }
    *out = (int *)ctx->kstat.ptr;
    return DAMAS_OK;
}

}  // namespace

extern "C" {

int damas_create(damas_ctx **out, int device) {
    if (!out) return DAMAS_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return DAMAS_EINVAL;
    }
    damas_ctx *ctx = new damas_ctx();
    ctx->device = device;
    DeviceGuard dg(device);
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device);
    ctx->sm_count = v;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    ctx->smem_optin = (size_t)v;
    *out = ctx;
    return DAMAS_OK;
}

int damas_destroy(damas_ctx *ctx) {
    if (!ctx) return DAMAS_EINVAL;
    if (ctx->serve) serve_shutdown(ctx);
    {
        DeviceGuard dg(ctx->device);
        cudaDeviceSynchronize();
        for (ScratchBuf *b : {&ctx->planes, &ctx->wave, &ctx->solve, &ctx->status, &ctx->misc, &ctx->pad, &ctx->probe,
                              &ctx->kstat})
            if (b->ptr) cudaFree(b->ptr);
    }
    delete ctx;
    return DAMAS_OK;
}

const char *damas_last_error(const damas_ctx *ctx) { return ctx ? ctx->err : "no context"; }

int damas_set_option(damas_ctx *ctx, int option, long long value) {
    if (!ctx) return DAMAS_EINVAL;
    switch (option) {
        case DAMAS_OPT_BUILD_TIMEOUT_MS:
            if (value < 1 || value > 600000) return ctx_fail(ctx, DAMAS_EINVAL, "build timeout %lld ms", value);
            ctx->build_timeout_ms = (int)value;
            return DAMAS_OK;
        case DAMAS_OPT_HBM_BUDGET_BYTES:
            if (value < 0) return ctx_fail(ctx, DAMAS_EINVAL, "HBM budget %lld bytes", value);
            if (value > 0 && (size_t)value < ctx_scratch_bytes(ctx))
                return ctx_fail(ctx, DAMAS_EINVAL, "HBM budget %lld bytes is below the %zu the context already holds",
                                value, ctx_scratch_bytes(ctx));
            ctx->hbm_budget = (size_t)value;
            return DAMAS_OK;
        case DAMAS_OPT_TEST_HOLD_BUILD:
            if (value != 0 && value != 1) return ctx_fail(ctx, DAMAS_EINVAL, "test hold must be 0 or 1");
            ctx->test_hold = (int)value;
            return DAMAS_OK;
        default:
            return ctx_fail(ctx, DAMAS_EINVAL, "unknown option %d", option);
    }
}

int damas_check(damas_ctx *ctx, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    DAMAS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (!ctx->kstat.ptr) return DAMAS_OK;
    int h = 0;
    DAMAS_CUDA_TRY(ctx, cudaMemcpy(&h, ctx->kstat.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h == 0) return DAMAS_OK;
    DAMAS_CUDA_TRY(ctx, cudaMemset(ctx->kstat.ptr, 0, sizeof(int)));
    return ctx_fail(ctx, h, "a build kernel's device wait ran out (limit %d ms); its output holds NaN",
                    ctx->build_timeout_ms);
}

int damas_lda(int S) { return S <= 0 ? 0 : round_up(S, 32); }

int damas_state_floats(int S) { return S <= 0 ? 0 : 2 * S + 64; }

// ----------------------------------------------------------------------------- PSF matrix
int damas_build_psf(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev, int S_sub,
                    int a_dtype, void *A_dev, int lda, float *gnorm2_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    int rc = check_geom(ctx, geom);
    if (rc) return rc;
    const long long S = (long long)geom->nx * geom->ny;
    if (geom->diag_removal)
        return ctx_fail(ctx, DAMAS_EINVAL, "diagonal removal: the PSF comes from damas_build_psf_dr");
    if (!(freq_hz > 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "frequency must be positive");
    if (S_sub < 1 || S_sub > S) return ctx_fail(ctx, DAMAS_EINVAL, "S_sub=%d out of range", S_sub);
    if (!idx_dev && S_sub != S) return ctx_fail(ctx, DAMAS_EINVAL, "S_sub must equal nx*ny when idx is NULL");
    if (a_dtype != DAMAS_F32 && a_dtype != DAMAS_BF16) return ctx_fail(ctx, DAMAS_EINVAL, "bad a_dtype");
    if (!A_dev) return ctx_fail(ctx, DAMAS_EINVAL, "A_dev is NULL");
    if (!aligned(A_dev, 16)) return ctx_fail(ctx, DAMAS_EINVAL, "A_dev must be 16-byte aligned");
    if (gnorm2_dev && !aligned(gnorm2_dev, 4)) return ctx_fail(ctx, DAMAS_EINVAL, "gnorm2_dev must be float-aligned");
    if (lda < S_sub || lda % 32) return ctx_fail(ctx, DAMAS_EINVAL, "lda=%d must be a multiple of 32 and >= S_sub", lda);
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ldm = planes_ld(geom->M);
    const int nplanes = geom->formulation == DAMAS_FORM_P ? 4 : 2;
    const size_t plane = (size_t)S_sub * ldm;
    const size_t work = psf_work_floats(S_sub, ldm, nplanes == 2);
    rc = ctx_ensure(ctx, ctx->planes, (plane * nplanes + work) * sizeof(float));
    if (rc) return rc;
    float *base = (float *)ctx->planes.ptr;
    float *Lre = base, *Lim = base + plane;
    float *Rre = nplanes == 4 ? base + 2 * plane : Lre, *Rim = nplanes == 4 ? base + 3 * plane : Lim;
    GeomK gk = to_kernel(geom, freq_hz);
    const int kind = geom->formulation == DAMAS_FORM_P ? 2 : 0;
    DAMAS_CUDA_TRY(ctx, launch_steer(gk, kind, idx_dev, S_sub, Lre, Lim, Rre, Rim, ldm, gnorm2_dev, st));
    const float scale = geom->formulation == DAMAS_FORM_P ? (float)(1.0 / ((double)geom->M * geom->M)) : 1.0f;
    int *kst = nullptr;
    rc = ctx_kstat(ctx, &kst);
    if (rc) return rc;
    DAMAS_CUDA_TRY(ctx, launch_psf_gram(Lre, Lim, Rre, Rim, ldm, geom->M, S_sub, scale, A_dev, lda, a_dtype,
                                        base + plane * nplanes, kst, (unsigned long long)ctx->build_timeout_ms * 1000000ull,
                                        ctx->test_hold, st));
    return DAMAS_OK;
}

int damas_build_psf_f32_bf16(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev,
                             int S_sub, float *A_f32_dev, void *A_bf16_dev, int lda, float *gnorm2_dev,
                             damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (!A_bf16_dev) return ctx_fail(ctx, DAMAS_EINVAL, "A_bf16_dev is NULL");
    if (!aligned(A_bf16_dev, 16)) return ctx_fail(ctx, DAMAS_EINVAL, "A_bf16_dev must be 16-byte aligned");
    if (A_f32_dev && S_sub > 0 && lda > 0) {
        const uintptr_t f0 = (uintptr_t)A_f32_dev, f1 = f0 + (uintptr_t)S_sub * lda * 4;
        const uintptr_t b0 = (uintptr_t)A_bf16_dev, b1 = b0 + (uintptr_t)S_sub * lda * 2;
        if (f0 < b1 && b0 < f1) return ctx_fail(ctx, DAMAS_EINVAL, "the two outputs must not overlap");
    }
    int rc = damas_build_psf(ctx, geom, freq_hz, idx_dev, S_sub, DAMAS_F32, A_f32_dev, lda, gnorm2_dev, stream);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    DAMAS_CUDA_TRY(ctx, launch_to_bf16(A_f32_dev, A_bf16_dev, (size_t)S_sub * lda, (cudaStream_t)stream));
    return DAMAS_OK;
}

int damas_build_psf_dr(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev, int S_sub,
                       float *A_dev, int lda, float *gnorm2_dev, float *dscale_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    int rc = check_geom(ctx, geom);
    if (rc) return rc;
    if (!geom->diag_removal) return ctx_fail(ctx, DAMAS_EINVAL, "damas_build_psf_dr needs geom->diag_removal = 1");
    const long long S = (long long)geom->nx * geom->ny;
    if (!(freq_hz > 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "frequency must be positive");
    if (S_sub < 1 || S_sub > S) return ctx_fail(ctx, DAMAS_EINVAL, "S_sub=%d out of range", S_sub);
    if (!idx_dev && S_sub != S) return ctx_fail(ctx, DAMAS_EINVAL, "S_sub must equal nx*ny when idx is NULL");
    if (!A_dev || !dscale_dev) return ctx_fail(ctx, DAMAS_EINVAL, "A_dev and dscale_dev are required");
    if (lda < S_sub || lda % 32) return ctx_fail(ctx, DAMAS_EINVAL, "lda=%d must be a multiple of 32 and >= S_sub", lda);
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int ldm = planes_ld(geom->M);
    const int nplanes = geom->formulation == DAMAS_FORM_P ? 4 : 2;
    const size_t plane = (size_t)S_sub * ldm;
    const size_t work = psf_work_floats(S_sub, ldm, nplanes == 2);
    rc = ctx_ensure(ctx, ctx->planes, (plane * nplanes + work) * sizeof(float));
    if (rc) return rc;
    float *base = (float *)ctx->planes.ptr;
    float *Lre = base, *Lim = base + plane;
    float *Rre = nplanes == 4 ? base + 2 * plane : Lre, *Rim = nplanes == 4 ? base + 3 * plane : Lim;
    GeomK gk = to_kernel(geom, freq_hz);
    const int kind = geom->formulation == DAMAS_FORM_P ? 2 : 0;
    DAMAS_CUDA_TRY(ctx, launch_steer(gk, kind, idx_dev, S_sub, Lre, Lim, Rre, Rim, ldm, gnorm2_dev, st));
    const float scale = geom->formulation == DAMAS_FORM_P ? (float)(1.0 / ((double)geom->M * geom->M)) : 1.0f;
    int *kst = nullptr;
    rc = ctx_kstat(ctx, &kst);
    if (rc) return rc;
    DAMAS_CUDA_TRY(ctx, launch_psf_gram(Lre, Lim, Rre, Rim, ldm, geom->M, S_sub, scale, A_dev, lda, DAMAS_F32,
                                        base + plane * nplanes, kst, (unsigned long long)ctx->build_timeout_ms * 1000000ull,
                                        ctx->test_hold, st));
    DAMAS_CUDA_TRY(ctx, launch_psf_dr(Lre, Lim, Rre, Rim, ldm, geom->M, S_sub, scale, A_dev, lda, dscale_dev, st));
    return DAMAS_OK;
}

int damas_divide(damas_ctx *ctx, float *v_dev, const float *div_dev, int n, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (n < 0 || (n > 0 && (!v_dev || !div_dev))) return ctx_fail(ctx, DAMAS_EINVAL, "bad divide arguments");
    DeviceGuard dg(ctx->device);
    DAMAS_CUDA_TRY(ctx, launch_divide(v_dev, div_dev, n, (cudaStream_t)stream));
    return DAMAS_OK;
}

// ----------------------------------------------------------------------------- CSM from time series
int damas_csm(damas_ctx *ctx, const float *p_dev, int M, long long T, int K, int hop, const int32_t *bins_dev, int F,
              float *C_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (M < 1 || M > DAMAS_MAX_MICS) return ctx_fail(ctx, DAMAS_EINVAL, "M=%d out of range", M);
    if (K < 2 || K > (1 << 20)) return ctx_fail(ctx, DAMAS_EINVAL, "K=%d out of range", K);
    if (hop < 1) return ctx_fail(ctx, DAMAS_EINVAL, "hop must be >= 1");
    if (T < K) return ctx_fail(ctx, DAMAS_EINVAL, "T=%lld shorter than one block", T);
    if (F < 1 || F > 4096) return ctx_fail(ctx, DAMAS_EINVAL, "F=%d out of range", F);
    if (!p_dev || !bins_dev || !C_dev) return ctx_fail(ctx, DAMAS_EINVAL, "NULL pointer");
    if (!aligned(C_dev, 8) || !aligned(p_dev, 4) || !aligned(bins_dev, 4))
        return ctx_fail(ctx, DAMAS_EINVAL, "C_dev must be 8-byte aligned (complex), p_dev and bins_dev 4-byte");
    const long long L = (T - K) / hop + 1;
    if ((long long)M * L > 65535ll * 64) return ctx_fail(ctx, DAMAS_EINVAL, "M*L=%lld too large", (long long)M * L);
    DeviceGuard dg(ctx->device);
    const int rc = ctx_ensure(ctx, ctx->misc, csm_work_floats(M, (int)L, F, K) * sizeof(float));
    if (rc) return rc;
    DAMAS_CUDA_TRY(ctx, launch_csm(p_dev, M, T, K, hop, bins_dev, F, C_dev, (float *)ctx->misc.ptr,
                                   (cudaStream_t)stream));
    return DAMAS_OK;
}

// ----------------------------------------------------------------------------- DAS map
int das_map(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const float *C_dev, float *b_dev,
            damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    int rc = check_geom(ctx, geom);
    if (rc) return rc;
    if (!(freq_hz > 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "frequency must be positive");
    if (!C_dev || !b_dev) return ctx_fail(ctx, DAMAS_EINVAL, "C_dev and b_dev are required");
    if (!aligned(C_dev, 8) || !aligned(b_dev, 4))
        return ctx_fail(ctx, DAMAS_EINVAL, "C_dev must be 8-byte aligned (complex), b_dev 4-byte");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    const int S = geom->nx * geom->ny;
    const int ldm = planes_ld(geom->M);
    const size_t plane = (size_t)S * ldm;
    rc = ctx_ensure(ctx, ctx->planes, plane * 2 * sizeof(float));
    if (rc) return rc;
    float *Lre = (float *)ctx->planes.ptr, *Lim = Lre + plane;
    GeomK gk = to_kernel(geom, freq_hz);
    // the vector the map is steered with: e (E) or v (P)
    const int kind = geom->formulation == DAMAS_FORM_P ? 1 : 0;
    DAMAS_CUDA_TRY(ctx, launch_steer(gk, kind, nullptr, S, Lre, Lim, nullptr, nullptr, ldm, nullptr, st));
    const float scale = geom->formulation == DAMAS_FORM_P ? (float)(1.0 / ((double)geom->M * geom->M)) : 1.0f;
    DAMAS_CUDA_TRY(ctx, launch_das(Lre, Lim, ldm, geom->M, S, C_dev, scale, b_dev, geom->diag_removal, st));
    return DAMAS_OK;
}

// ----------------------------------------------------------------------------- compressed grid
int wavelet_compress_grid(damas_ctx *ctx, const float *b_dev, int nx, int ny, const damas_wavelet_cfg *cfg,
                          int32_t *idx_dev, int32_t *S_sub_dev, float *detail_dev, float *eps_abs_dev,
                          damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (!cfg) return ctx_fail(ctx, DAMAS_EINVAL, "cfg is NULL");
    if (!b_dev || !idx_dev || !S_sub_dev) return ctx_fail(ctx, DAMAS_EINVAL, "b_dev, idx_dev, S_sub_dev are required");
    if (nx < 1 || ny < 1 || nx > 65535 || ny > 65535 || (long long)nx * ny > 4194304)
        return ctx_fail(ctx, DAMAS_EINVAL, "grid %dx%d out of range", nx, ny);
    if (cfg->levels < 1 || cfg->levels > 15) return ctx_fail(ctx, DAMAS_EINVAL, "levels=%d out of range", cfg->levels);
    if (cfg->predictor != DAMAS_PRED_LINEAR && cfg->predictor != DAMAS_PRED_HAAR)
        return ctx_fail(ctx, DAMAS_EINVAL, "unknown predictor");
    if (cfg->eps_mode < DAMAS_EPS_ABS || cfg->eps_mode > DAMAS_EPS_KEEP_FRAC)
        return ctx_fail(ctx, DAMAS_EINVAL, "unknown eps_mode");
    if (!(cfg->eps >= 0.0)) return ctx_fail(ctx, DAMAS_EINVAL, "eps must be >= 0");
    if (cfg->eps_mode == DAMAS_EPS_KEEP_FRAC && cfg->eps > 1.0)
        return ctx_fail(ctx, DAMAS_EINVAL, "keep fraction must be in [0, 1]");
    DeviceGuard dg(ctx->device);
    const int S = nx * ny;
    int rc = ctx_ensure(ctx, ctx->wave, (size_t)S * sizeof(float));
    if (rc) return rc;
    const int J = cfg->levels;
    const long long n0 = (long long)(((nx - 1) >> J) + 1) * (((ny - 1) >> J) + 1);
    const long long K = cfg->eps_mode == DAMAS_EPS_KEEP_FRAC ? (long long)ceil(cfg->eps * (double)S) - n0 : 0;
    DAMAS_CUDA_TRY(ctx, launch_wavelet(b_dev, nx, ny, J, cfg->predictor, cfg->eps_mode, (float)cfg->eps, (float)cfg->eps,
                                       K, idx_dev, S_sub_dev, detail_dev, eps_abs_dev, (float *)ctx->wave.ptr,
                                       (cudaStream_t)stream));
    return DAMAS_OK;
}

int damas_pad_grid(damas_ctx *ctx, int nx, int ny, const int32_t *idx_dev, const int32_t *S_sub_dev, int radius,
                   int32_t *out_idx_dev, int32_t *out_S_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (!idx_dev || !S_sub_dev || !out_idx_dev || !out_S_dev)
        return ctx_fail(ctx, DAMAS_EINVAL, "idx_dev, S_sub_dev, out_idx_dev, out_S_dev are required");
    if (nx < 1 || ny < 1 || nx > 65535 || ny > 65535 || (long long)nx * ny > 4194304)
        return ctx_fail(ctx, DAMAS_EINVAL, "grid %dx%d out of range", nx, ny);
    if (radius < 0 || radius > 8) return ctx_fail(ctx, DAMAS_EINVAL, "radius=%d out of range", radius);
    DeviceGuard dg(ctx->device);
    const int rc = ctx_ensure(ctx, ctx->pad, (size_t)nx * ny);
    if (rc) return rc;
    DAMAS_CUDA_TRY(ctx, launch_pad_grid(nx, ny, idx_dev, S_sub_dev, radius, out_idx_dev, out_S_dev,
                                        (unsigned char *)ctx->pad.ptr, (cudaStream_t)stream));
    return DAMAS_OK;
}

// ----------------------------------------------------------------------------- gather / scatter
int damas_gather(damas_ctx *ctx, const float *src_dev, const int32_t *idx_dev, int n, float *dst_dev,
                 damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (n < 0 || (n > 0 && (!src_dev || !idx_dev || !dst_dev))) return ctx_fail(ctx, DAMAS_EINVAL, "bad gather arguments");
    DeviceGuard dg(ctx->device);
    DAMAS_CUDA_TRY(ctx, launch_gather(src_dev, idx_dev, n, dst_dev, (cudaStream_t)stream));
    return DAMAS_OK;
}

int damas_scatter_power(damas_ctx *ctx, const float *x_sub_dev, const int32_t *idx_dev, const float *gnorm2_dev,
                        int n, float *x_full_dev, int S, double *total_power_dev, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (S < 1 || n < 0 || n > S || !x_full_dev || (n > 0 && !x_sub_dev))
        return ctx_fail(ctx, DAMAS_EINVAL, "bad scatter arguments");
    if (!idx_dev && n != S) return ctx_fail(ctx, DAMAS_EINVAL, "n must equal S when idx is NULL");
    if (total_power_dev && !aligned(total_power_dev, 8))
        return ctx_fail(ctx, DAMAS_EINVAL, "total_power_dev must be 8-byte aligned");
    DeviceGuard dg(ctx->device);
    DAMAS_CUDA_TRY(ctx, launch_scatter_power(x_sub_dev, idx_dev, gnorm2_dev, n, x_full_dev, S, total_power_dev,
                                             (cudaStream_t)stream));
    return DAMAS_OK;
}

// ----------------------------------------------------------------------------- DAMAS iteration
namespace {

struct Plan {
    int ncta, R, resident, solo;
    size_t smem;
};

// Systems up to this many rows run the single-CTA form when no team size is asked
// for: on such systems its step (the row chain and one barrier) is no longer than
// a team's average step with its hand-overs between CTAs (FP32 A, 1000 sweeps:
// 11.9 / 17.4 / 25.8 ms at S = 441 / 657 / 985 against 12.8 / 18.3 / 26.2 ms for
// the best team; 37.8 against 34.0 ms at S = 1313), and a batch of them needs no
// co-residency.
constexpr int SOLO_AUTO_ROWS = 1024;

Plan plan_system(const damas_ctx *ctx, const damas_system &s, int forced, int placement, int cta_budget,
                 bool allow_solo = true) {
    const int nb = (s.S + 31) / 32;
    const size_t budget = ctx->smem_optin > 4096 ? ctx->smem_optin - 2048 : 0;
    Plan p{};
    auto finish = [&](int R, bool res) {
        p.R = R;
        p.ncta = (nb * 32 + R - 1) / R;
        p.resident = res ? 1 : 0;
        p.smem = sweep_smem_bytes(R, s.lda, s.a_dtype, res);
    };
    auto rows_for = [&](int P) { return (nb + P - 1) / P * 32; };
    // the most rows of A a CTA can hold next to its x and residual
    const size_t per_row = sweep_smem_bytes(1, s.lda, s.a_dtype, true);
    const int rmax_res = (int)std::min<size_t>(budget / per_row, (size_t)1 << 20) / 32 * 32;
    if (nb == 1) {  // a single block is always held in shared memory
        finish(32, true);
        return p;
    }
    // one CTA without hand-overs (asked for, or by default for small systems)
    const size_t solo_smem = sweep_solo_smem_bytes(nb * 32, s.a_dtype);
    if (allow_solo && nb >= 4 && placement != 1 && solo_smem <= budget &&
        (forced == 1 || (forced == 0 && s.S <= SOLO_AUTO_ROWS))) {
        p.ncta = 1;
        p.R = nb * 32;
        p.resident = 0;
        p.solo = 1;
        p.smem = solo_smem;
        return p;
    }
    if (forced > 0) {
        const int R = rows_for(std::min(forced, nb));
        finish(R, placement == 1 || (placement == 0 && R <= rmax_res));
        return p;
    }
    if (placement != 2 && rmax_res >= 32) {
        const int P = (nb * 32 + rmax_res - 1) / rmax_res;
        if (P <= std::min(cta_budget, 16) || placement == 1) {
            finish(rows_for(P), true);
            return p;
        }
    }
    // rows streamed from global memory: three blocks per CTA (full 81x81 grid,
    // 1000 sweeps: 129.9 ms with 69 CTAs against 134.5 ms with two blocks per
    // CTA and 130.6 ms with four; fewer CTAs mean fewer hand-overs, more rows
    // per CTA a longer per-step update next to the row chain)
    const int P = std::max(1, std::min(cta_budget, (nb + 2) / 3));
    finish(rows_for(P), false);
    return p;
}

struct Launch {
    std::vector<int> ids;
    size_t smem = 0;
    int ctas = 0;
    int max_iters = 0;
    int solo = 0;
};

// Plan every system of a damas_solve call, then pack them into launches that
// fit on the device at once (systems already validated).
int plan_solve(damas_ctx *ctx, const damas_system *sys, int nsys, int forced, int placement,
               std::vector<Plan> &plans, std::vector<Launch> &launches) {
    // plan every system, then pack them into launches that fit on the device at once
    plans.assign(nsys, Plan());
    for (int i = 0; i < nsys; ++i)
        plans[i] = plan_system(ctx, sys[i], sys[i].ctas > 0 ? sys[i].ctas : forced, placement, ctx->sm_count);
    {
        // The single-CTA form runs in a launch of its own.  A call that also holds
        // teams keeps every system in the teams' one launch (launches on a stream
        // run one after another), so there the single-CTA systems become one-CTA
        // teams.
        int nsolo = 0;
        for (const Plan &q : plans) nsolo += q.solo;
        if (nsolo > 0 && nsolo < nsys)
            for (int i = 0; i < nsys; ++i)
                if (plans[i].solo)
                    plans[i] = plan_system(ctx, sys[i], sys[i].ctas > 0 ? sys[i].ctas : forced, placement,
                                           ctx->sm_count, false);
    }
    if (placement == 0 && nsys > 1) {
        // A batch whose resident teams need more than one launch (a resident CTA
        // fills an SM) but whose streamed teams fit in one (two CTAs per SM) is
        // streamed: the teams then run side by side.  Results do not depend on the
        // placement.
        auto fits_once = [&](const std::vector<Plan> &pl) -> bool {
            size_t smem = 0;
            int ctas = 0;
            for (const Plan &q : pl) {
                smem = std::max(smem, q.smem);
                ctas += q.ncta;
            }
            int occ = 0;
            if (nsys > SWEEP_MAX_SYS || sweep_occupancy(smem, &occ) != cudaSuccess) return false;
            return ctas <= occ * ctx->sm_count;
        };
        bool any_res = false;
        for (const Plan &q : plans) any_res |= q.resident != 0;
        if (any_res && !fits_once(plans)) {
            std::vector<Plan> streamed(nsys);
            for (int i = 0; i < nsys; ++i)
                streamed[i] = plans[i].resident
                                  ? plan_system(ctx, sys[i], sys[i].ctas > 0 ? sys[i].ctas : forced, 2, ctx->sm_count,
                                                false)
                                  : plans[i];
            if (fits_once(streamed)) plans.swap(streamed);
        }
        cudaGetLastError();
    }
    for (int i = 0; i < nsys; ++i) {
        if (plans[i].smem > ctx->smem_optin - 1024)
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: %zu bytes of shared memory per CTA do not fit", i,
                            plans[i].smem);
        if (plans[i].solo) continue;
        int occ = 0;
        cudaError_t e = sweep_occupancy(plans[i].smem, &occ);
        if (e != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
        if (plans[i].ncta > occ * ctx->sm_count)
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d needs %d co-resident CTAs, the device holds %d", i,
                            plans[i].ncta, occ * ctx->sm_count);
    }
    launches.clear();
    {
        // a launch holds either single-CTA systems (any number of CTAs: none waits
        // on another) or teams (all co-resident)
        Launch cur;
        for (int i = 0; i < nsys; ++i) {
            const Plan &pl = plans[i];
            bool flush = !cur.ids.empty() && ((int)cur.ids.size() == SWEEP_MAX_SYS || cur.solo != pl.solo);
            if (!flush && !pl.solo && !cur.ids.empty()) {
                int occ = 0;
                cudaError_t e = sweep_occupancy(std::max(cur.smem, pl.smem), &occ);
                if (e != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
                flush = cur.ctas + pl.ncta > occ * ctx->sm_count;
            }
            if (flush) {
                launches.push_back(cur);
                cur = Launch();
            }
            cur.solo = pl.solo;
            cur.ids.push_back(i);
            cur.smem = std::max(cur.smem, pl.smem);
            cur.ctas += pl.ncta;
            cur.max_iters = std::max(cur.max_iters, sys[i].iters);
        }
        if (!cur.ids.empty()) launches.push_back(cur);
    }
    return DAMAS_OK;
}

}  // namespace

}  // extern "C"

int solve_half_sm_units(damas_ctx *ctx, const damas_system *sys, int nsys, int *units) {
    std::vector<Plan> plans;
    std::vector<Launch> launches;
    int rc = plan_solve(ctx, sys, nsys, 0, 0, plans, launches);
    if (rc) return rc;
    int most = 0;
    for (const Launch &L : launches) {
        int occ = 0;
        cudaError_t e = L.solo ? sweep_solo_occupancy(L.smem, &occ) : sweep_occupancy(L.smem, &occ);
        if (e != cudaSuccess) return ctx_fail(ctx, DAMAS_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
        const int per_cta = occ >= 2 ? 1 : 2;  // a CTA that fills its SM holds both halves
        most = std::max(most, L.ctas * per_cta);
    }
    *units = most;
    return DAMAS_OK;
}

extern "C" {

int damas_solve_plan(damas_ctx *ctx, int S, int lda, int a_dtype, int ctas, int a_placement, int *ncta_out,
                     int *rows_per_cta_out, int *resident_out) {
    if (!ctx) return DAMAS_EINVAL;
    if (S < 1 || lda < round_up(S, 32) || lda % 32) return ctx_fail(ctx, DAMAS_EINVAL, "S=%d, lda=%d", S, lda);
    if (a_dtype != DAMAS_F32 && a_dtype != DAMAS_BF16) return ctx_fail(ctx, DAMAS_EINVAL, "a_dtype");
    if (ctas < 0 || a_placement < 0 || a_placement > 2) return ctx_fail(ctx, DAMAS_EINVAL, "ctas or a_placement");
    damas_system s;
    memset(&s, 0, sizeof(s));
    s.S = S;
    s.lda = lda;
    s.a_dtype = a_dtype;
    const Plan pl = plan_system(ctx, s, ctas, a_placement, ctx->sm_count);
    if (ncta_out) *ncta_out = pl.ncta;
    if (rows_per_cta_out) *rows_per_cta_out = pl.R;
    if (resident_out) *resident_out = pl.resident;
    return DAMAS_OK;
}

int damas_handover_probe(damas_ctx *ctx, int rounds, int max_pairs, int timeout_us, double *ns_host, int *n_pairs,
                         damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (rounds < 1 || rounds > 100000 || max_pairs < 1 || timeout_us < 0 || !ns_host || !n_pairs)
        return ctx_fail(ctx, DAMAS_EINVAL, "bad probe arguments");
    DeviceGuard dg(ctx->device);
    const int npairs = std::min(max_pairs, ctx->sm_count - 1);
    if (npairs < 1) return ctx_fail(ctx, DAMAS_EINVAL, "the device has one SM");
    int rc = ctx_ensure(ctx, ctx->probe, handover_probe_bytes(npairs));
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *ns_dev = nullptr;
    int *status_dev = nullptr;
    const unsigned long long timeout_ns = (timeout_us > 0 ? (unsigned long long)timeout_us : 2000000ull) * 1000ull;
    DAMAS_CUDA_TRY(ctx, launch_handover_probe(ctx->probe.ptr, rounds, npairs, timeout_ns, st, &ns_dev, &status_dev));
    int status = 0;
    DAMAS_CUDA_TRY(ctx, cudaMemcpyAsync(ns_host, ns_dev, sizeof(double) * npairs, cudaMemcpyDeviceToHost, st));
    DAMAS_CUDA_TRY(ctx, cudaMemcpyAsync(&status, status_dev, sizeof(int), cudaMemcpyDeviceToHost, st));
    DAMAS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    *n_pairs = npairs;
    if (status != 0) return ctx_fail(ctx, DAMAS_ETIMEDOUT, "a hand-over wait ran out");
    return DAMAS_OK;
}

}  // extern "C"

namespace {

int check_systems(damas_ctx *ctx, const damas_system *sys, int nsys) {
    for (int i = 0; i < nsys; ++i) {
        const damas_system &s = sys[i];
        if (s.S < 1) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: S=%d", i, s.S);
        if (!s.A_dev || !s.b_dev || !s.x_dev) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: NULL pointer", i);
        // rows of A are read as 16-byte vectors and by TMA, whose base must be 16-byte aligned
        if (!aligned(s.A_dev, 16) || (s.At_dev && !aligned(s.At_dev, 16)))
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: A_dev and At_dev must be 16-byte aligned", i);
        if (!aligned(s.b_dev, 4) || !aligned(s.x_dev, 4) || (s.state_dev && !aligned(s.state_dev, 4)))
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: b_dev, x_dev and state_dev must be float-aligned", i);
        if (s.a_dtype != DAMAS_F32 && s.a_dtype != DAMAS_BF16) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: a_dtype", i);
        if (s.lda < round_up(s.S, 32) || s.lda % 32)
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: lda=%d must be a multiple of 32 and >= S rounded up to 32", i,
                            s.lda);
        if (s.init < DAMAS_INIT_ZERO || s.init > DAMAS_INIT_STATE) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: init", i);
        if (s.init == DAMAS_INIT_STATE && !s.state_dev)
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: INIT_STATE needs state_dev", i);
        if (s.iters < 0 || s.iters > (1 << 24)) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: iters=%d", i, s.iters);
        if (s.ctas < 0) return ctx_fail(ctx, DAMAS_EINVAL, "system %d: ctas=%d", i, s.ctas);
    }
    return DAMAS_OK;
}

// The body of damas_solve on validated systems.  clear_status: start the call's
// status word at DAMAS_OK (a later call of a sequence keeps an earlier error);
// finish: without cfg->status_dev, synchronise and return the status.
int solve_checked(damas_ctx *ctx, const damas_system *sys, int nsys, const damas_solve_cfg *cfg, cudaStream_t st,
                  bool clear_status, bool finish) {
    const int forced = cfg ? cfg->ctas_per_system : 0;
    const int placement = cfg ? cfg->a_placement : 0;
    if (placement < 0 || placement > 2) return ctx_fail(ctx, DAMAS_EINVAL, "a_placement=%d", placement);
    const long long timeout_ms = (cfg && cfg->timeout_ms > 0) ? cfg->timeout_ms : 2000;

    std::vector<Plan> plans;
    std::vector<Launch> launches;
    int prc = plan_solve(ctx, sys, nsys, forced, placement, plans, launches);
    if (prc) return prc;
    // exchange buffers: per system nb*32 mailbox words (epoch << 32 | bits(dx)),
    // sized for the largest launch.  The region only ever holds mailbox words,
    // and epochs grow from launch to launch, so stale words always read as old.
    size_t need = 0;
    for (const Launch &L : launches) {
        size_t m = 0;
        for (int i : L.ids) m += (size_t)((sys[i].S + 31) / 32) * 32 * sizeof(unsigned long long);
        need = std::max(need, m);
    }
    const bool grow = need > ctx->solve.cap;
    int rc = ctx_ensure(ctx, ctx->solve, need);
    if (rc) return rc;
    if (grow) {
        DAMAS_CUDA_TRY(ctx, cudaMemsetAsync(ctx->solve.ptr, 0, ctx->solve.cap, st));
        ctx->epoch = 0;
    }
    rc = ctx_ensure(ctx, ctx->status, 64);
    if (rc) return rc;
    int *status = cfg && cfg->status_dev ? cfg->status_dev : (int *)ctx->status.ptr;
    if (clear_status) DAMAS_CUDA_TRY(ctx, cudaMemsetAsync(status, 0, sizeof(int), st));

    // A launch recorded into a CUDA graph keeps the epoch it was recorded with, so
    // every replay would find the words of the previous replay already "new": the
    // recording clears the mailbox words first, and each replay starts from zero.
    cudaStreamCaptureStatus cap_status = cudaStreamCaptureStatusNone;
    DAMAS_CUDA_TRY(ctx, cudaStreamIsCapturing(st, &cap_status));
    const bool capturing = cap_status == cudaStreamCaptureStatusActive;
    for (const Launch &L : launches) {
        if ((unsigned long long)ctx->epoch + L.max_iters + 2 >= 0xffffffffull) {
            DAMAS_CUDA_TRY(ctx, cudaMemsetAsync(ctx->solve.ptr, 0, ctx->solve.cap, st));
            ctx->epoch = 0;
        }
        if (capturing) {
            size_t used = 0;
            for (int i : L.ids) used += (size_t)((sys[i].S + 31) / 32) * 32 * sizeof(unsigned long long);
            DAMAS_CUDA_TRY(ctx, cudaMemsetAsync(ctx->solve.ptr, 0, used, st));
        }
        SweepParams p;
        memset(&p, 0, sizeof(p));
        p.nsys = (int)L.ids.size();
        p.status = status;
        p.timeout_ns = (unsigned long long)timeout_ms * 1000000ull;
        p.withhold_block = (cfg && cfg->withhold_block > 0) ? cfg->withhold_block - 1 : -1;
        p.upstream = (const int *)ctx->kstat.ptr;
        p.stats = cfg ? (unsigned long long *)cfg->stats_dev : nullptr;
        unsigned long long *mb = (unsigned long long *)ctx->solve.ptr;
        int cta = 0;
        for (int q = 0; q < p.nsys; ++q) {
            const int i = L.ids[q];
            const damas_system &s = sys[i];
            const Plan &pl = plans[i];
            const int nb = (s.S + 31) / 32;
            SweepSys &d = p.sys[q];
            d.A = s.A_dev;
            d.At = s.At_dev ? s.At_dev : s.A_dev;
            d.b = s.b_dev;
            d.x = s.x_dev;
            d.state = s.state_dev;
            d.mbox = mb;
            mb += (size_t)nb * 32;
            d.lda = s.lda;
            d.S = s.S;
            d.dtype = s.a_dtype;
            d.init = s.init;
            d.iters = s.iters;
            d.cta0 = cta;
            d.ncta = pl.ncta;
            d.rows_per_cta = pl.R;
            d.resident = pl.resident;
            d.epoch0 = ctx->epoch;
            cta += pl.ncta;
        }
        if (L.solo) {
            std::unique_ptr<SoloMaps> maps(new SoloMaps());  // copied into the launch's parameters
            for (int q = 0; q < p.nsys; ++q)
                if (!make_sweep_tile_map(&maps->m[q], p.sys[q].At, p.sys[q].dtype, p.sys[q].lda, p.sys[q].S))
                    return ctx_fail(ctx, DAMAS_ECUDA, "tensor map for system %d", L.ids[q]);
            DAMAS_CUDA_TRY(ctx, launch_sweep_solo(p, *maps, L.smem, st));
        } else {
            DAMAS_CUDA_TRY(ctx, launch_sweep(p, cta, L.smem, st));
        }
        ctx->epoch += (unsigned)L.max_iters + 1u;
    }
    if (!finish || (cfg && cfg->status_dev)) return DAMAS_OK;
    int h = 0;
    DAMAS_CUDA_TRY(ctx, cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DAMAS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    if (h != 0)
        return ctx_fail(ctx, h,
                        "a device wait ran out: in the solve (limit %lld ms), or in a build kernel of this context "
                        "before it (damas_check reports and clears that)",
                        timeout_ms);
    return DAMAS_OK;
}

}  // namespace

extern "C" {

int damas_chain_probe(damas_ctx *ctx, int rounds, double *ns_host, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (rounds < 1 || rounds > 10000000 || !ns_host) return ctx_fail(ctx, DAMAS_EINVAL, "bad probe arguments");
    DeviceGuard dg(ctx->device);
    int rc = ctx_ensure(ctx, ctx->probe, 4096);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    double *out = (double *)ctx->probe.ptr;
    float *sink = (float *)((char *)ctx->probe.ptr + 256);
    DAMAS_CUDA_TRY(ctx, launch_chain_probe(rounds, out, sink, st));
    DAMAS_CUDA_TRY(ctx, cudaMemcpyAsync(ns_host, out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    DAMAS_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    return DAMAS_OK;
}

int damas_solve(damas_ctx *ctx, const damas_system *sys, int nsys, const damas_solve_cfg *cfg, damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (nsys < 0 || (nsys > 0 && !sys)) return ctx_fail(ctx, DAMAS_EINVAL, "bad system array");
    if (nsys == 0) return DAMAS_OK;
    int rc = check_systems(ctx, sys, nsys);
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    return solve_checked(ctx, sys, nsys, cfg, (cudaStream_t)stream, true, true);
}

int damas_solve_mixed(damas_ctx *ctx, const damas_mixed_system *msys, int nsys, const damas_solve_cfg *cfg,
                      damas_stream stream) {
    if (!ctx) return DAMAS_EINVAL;
    if (nsys < 0 || (nsys > 0 && !msys)) return ctx_fail(ctx, DAMAS_EINVAL, "bad system array");
    if (nsys == 0) return DAMAS_OK;
    if (cfg && cfg->withhold_block) return ctx_fail(ctx, DAMAS_EINVAL, "withhold_block is a damas_solve test hook");
    // the two phases as plain systems: BF16 from x = 0, then FP32 from the exact
    // residual of the bulk phase's x (or from x = 0 when there is no bulk phase)
    std::vector<damas_system> bulk, refine;
    for (int i = 0; i < nsys; ++i) {
        const damas_mixed_system &m = msys[i];
        if (m.iters_bulk < 0 || m.iters_refine < 0)
            return ctx_fail(ctx, DAMAS_EINVAL, "system %d: negative sweep count", i);
        damas_system s;
        memset(&s, 0, sizeof(s));
        s.lda = m.lda;
        s.S = m.S;
        s.b_dev = m.b_dev;
        s.x_dev = m.x_dev;
        s.ctas = m.ctas;
        if (m.iters_bulk > 0) {
            s.A_dev = m.A_bulk_dev;
            s.At_dev = m.At_bulk_dev;
            s.a_dtype = DAMAS_BF16;
            s.init = DAMAS_INIT_ZERO;
            s.iters = m.iters_bulk;
            bulk.push_back(s);
        }
        if (m.iters_refine > 0 || m.iters_bulk == 0) {
            s.A_dev = m.A_refine_dev;
            s.At_dev = m.At_refine_dev;
            s.a_dtype = DAMAS_F32;
            s.init = m.iters_bulk > 0 ? DAMAS_INIT_X : DAMAS_INIT_ZERO;
            s.iters = m.iters_refine;
            refine.push_back(s);
        }
    }
    int rc = check_systems(ctx, bulk.data(), (int)bulk.size());
    if (rc == DAMAS_OK) rc = check_systems(ctx, refine.data(), (int)refine.size());
    if (rc) return rc;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (!bulk.empty()) {
        rc = solve_checked(ctx, bulk.data(), (int)bulk.size(), cfg, st, true, refine.empty());
        if (rc) return rc;
    }
    if (!refine.empty()) return solve_checked(ctx, refine.data(), (int)refine.size(), cfg, st, bulk.empty(), true);
    return DAMAS_OK;
}

}  // extern "C"
