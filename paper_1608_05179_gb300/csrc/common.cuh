// Shared definitions of the DAMAS CUDA library (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "damas.h"

// ----------------------------------------------------------------------------- context
struct ScratchBuf {
    void *ptr = nullptr;
    size_t cap = 0;
};

struct damas_ctx {
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;  // max dynamic shared memory per block (opt-in)
    char err[512] = {0};
    // scratch, grown on demand
    ScratchBuf planes;   // steering / propagation vectors
    ScratchBuf wave;     // wavelet work arrays
    ScratchBuf solve;    // solver exchange buffers and flags
    ScratchBuf status;   // solver status words
    ScratchBuf misc;
    ScratchBuf pad;      // neighbour-padding marks
    ScratchBuf probe;    // hand-over probe words
    ScratchBuf kstat;    // build status word: DAMAS_ETIMEDOUT once a build kernel's wait ran out (sticky)
    int build_timeout_ms = 2000;  // bound on the build kernels' device waits
    size_t hbm_budget = 0;        // cap on the context's device memory (scratch, serving default); 0 = none
    int test_hold = 0;            // test hook of those waits (damas_set_option)
    unsigned int epoch = 0;      // mailbox epoch of the solver exchange buffers
    struct ServeState *serve = nullptr;  // serving loop, when started
};
void serve_shutdown(damas_ctx *ctx);

int ctx_fail(damas_ctx *ctx, int code, const char *fmt, ...);
// Half-SM units that a damas_solve call on these systems (default placement and
// team sizes, as given per system) occupies while its largest launch runs: a CTA
// that fills its SM (one CTA per SM) counts 2, one of a launch with two or more
// CTAs per SM counts 1.  The device has 2 * sm_count units.  The calling thread
// must have the context's device current.
int solve_half_sm_units(damas_ctx *ctx, const damas_system *sys, int nsys, int *units);
int ctx_ensure(damas_ctx *ctx, ScratchBuf &b, size_t bytes);

#define DAMAS_CUDA_TRY(ctx, call)                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return ctx_fail((ctx), DAMAS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

static inline int round_up(int v, int m) { return (v + m - 1) / m * m; }

// Geometry as the kernels see it.
struct GeomK {
    const double *mic;  // M x 3
    int M;
    int nx, ny;
    double x0, y0, dx, dy, z;
    double f_over_c;    // k / (2 pi): cycles per metre
    int form;
};

// ----------------------------------------------------------------------------- kernel launchers
// Vectors of n points (grid indices idx[i], or i when idx is NULL) as FP32
// planes [n][ldm].  kind 0: L = e (formulation E); 1: L = v; 2: L = v, R = g
// (formulation P).  gnorm2 (optional) receives ||g||^2.
cudaError_t launch_steer(const GeomK &g, int kind, const int32_t *idx, int n, float *Lre, float *Lim, float *Rre,
                         float *Rim, int ldm, float *gnorm2, cudaStream_t st);
// A[n][s] = scale * |sum_m conj(L_nm) R_sm|^2 with unit diagonal, zero padding to
// lda, on the tensor cores (tcgen05, 3xTF32); ldm must be a multiple of 16 and
// work must hold psf_work_floats() floats of device scratch.  Every device wait
// is bounded by timeout_ns; one that runs out writes DAMAS_ETIMEDOUT into
// *status (when status is given, only over 0).  hold = 1 is the test hook of
// those waits: the operand loader first waits for a flag that nothing sets.
cudaError_t launch_psf_gram(const float *Lre, const float *Lim, const float *Rre, const float *Rim, int ldm,
                            int M, int S, float scale, void *A, int lda, int a_dtype, float *work, int *status,
                            unsigned long long timeout_ns, int hold, cudaStream_t st);
size_t psf_work_floats(int S, int ldm, bool symmetric);
// dst[i] = bfloat16(src[i]) (round to nearest even), i < n.
cudaError_t launch_to_bf16(const float *src, void *dst, size_t n, cudaStream_t st);
// b_n = scale * Re(L_n^H C L_n) for n < S (dr: without the terms of C's diagonal).
cudaError_t launch_das(const float *Lre, const float *Lim, int ldm, int M, int S, const float *C, float scale,
                       float *b, int dr, cudaStream_t st);
// Diagonal removal on a PSF the Gram wrote: d_n into dscale (as sqrt), then A
// corrected and rescaled to a unit diagonal in place (FP32).
cudaError_t launch_psf_dr(const float *Lre, const float *Lim, const float *Rre, const float *Rim, int ldm, int M,
                          int S, float scale, float *A, int lda, float *dscale, cudaStream_t st);
cudaError_t launch_divide(float *v, const float *d, int n, cudaStream_t st);
// CSM of F bins from time series (Welch); work: csm_work_floats(M, L, F, K) floats.
size_t csm_work_floats(int M, int L, int F, int K);
cudaError_t launch_csm(const float *p, int M, long long T, int K, int hop, const int32_t *bins, int F, float *C,
                       float *work, cudaStream_t st);
// Hand-over latency probe: work must hold handover_probe_bytes(npairs) bytes
// of device memory; out_ns / status point into it (npairs doubles, one int).
size_t handover_probe_bytes(int npairs);
cudaError_t launch_handover_probe(void *work, int rounds, int npairs, unsigned long long timeout_ns, cudaStream_t st,
                                  double **out_ns, int **status);
// Row-chain latency probe: out_dev[0] ns per candidate update of a block
// solve, out_dev[1] ns per barrier step of a 512-thread CTA; sink_dev: 33 floats.
cudaError_t launch_chain_probe(int rounds, double *out_dev, float *sink_dev, cudaStream_t st);
// Neighbour padding of a grid-index set (one CTA): marks (bytes, S of them)
// is scratch.
cudaError_t launch_pad_grid(int nx, int ny, const int32_t *idx, const int32_t *n_in, int radius, int32_t *out,
                            int32_t *n_out, unsigned char *marks, cudaStream_t st);
cudaError_t launch_wavelet(const float *b, int nx, int ny, int levels, int pred, int eps_mode, float eps_abs,
                           float eps_rel, long long keep_K, int32_t *idx, int32_t *S_sub, float *detail,
                           float *eps_abs_out, float *work_absd, cudaStream_t st);
cudaError_t launch_gather(const float *src, const int32_t *idx, int n, float *dst, cudaStream_t st);
cudaError_t launch_scatter_power(const float *x_sub, const int32_t *idx, const float *gnorm2, int n,
                                 float *x_full, int S, double *total, cudaStream_t st);

// ----------------------------------------------------------------------------- device helpers
#ifdef __CUDACC__
// Error-free transformations (Knuth TwoSum, FMA-based TwoProduct), written with
// round-to-nearest intrinsics so that no contraction changes them.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}
#endif
