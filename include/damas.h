/*
 * damas.h - C ABI of the GB300 DAMAS library (libdamas.so).
 *
 * Hot path of Ma & Liu, "Improving the Efficiency of DAMAS for Sound Source
 * Localization via Wavelet Compression Computational Grid": steering vectors,
 * PSF matrix, DAS map, wavelet-compressed grid, and the DAMAS Gauss-Seidel
 * iteration, on the full scan grid or on the compressed one.
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: DAMAS_OK (0) or a negative code.
 *    damas_last_error() returns a message for the last failure on a context.
 *  - Buffers are owned by the caller.  Pointers named *_dev are device pointers
 *    on the context's device; every call enqueues its work on the given stream
 *    and returns without waiting, unless its comment says otherwise.  Device
 *    results are valid once the stream has reached the call.
 *  - Arguments are validated on the host before anything is enqueued; a bad
 *    argument returns DAMAS_EINVAL and enqueues nothing.
 *  - A context owns scratch device memory (grown on demand, outside any
 *    captured region) that calls on that context share: issue the calls of one
 *    context on one stream, or serialise them.
 *  - Calls may be recorded into a CUDA graph (stream capture) once an eager run
 *    of the same calls has sized the scratch.  A recorded damas_solve clears its
 *    exchange words at the start of every replay, so a graph can be replayed any
 *    number of times, between eager calls on the same context; a later call that
 *    needs more scratch reallocates it and the graph must be recorded again.
 *  - Scan grid (§2): nx x ny points at (x0 + ix*dx, y0 + iy*dy, z), index
 *    n = iy*nx + ix; the array centre is the origin.
 *  - Equation numbers follow the order of the paper's displayed equations:
 *    (2) DAS map, (4) steering v, (7) propagation g, (10) PSF, (12) Ax=b,
 *    (13)-(14) Gauss-Seidel with clamp, (15) nested grids, (22) compressed
 *    grid, (23) wavelet coefficient, (24) compressed system; Algorithm 1.
 */
#ifndef DAMAS_H
#define DAMAS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct damas_ctx damas_ctx;
/* A CUDA stream handle (cudaStream_t); NULL selects the legacy default stream. */
typedef void *damas_stream;

enum {
    DAMAS_OK = 0,
    DAMAS_EINVAL = -1,    /* invalid argument (nothing was enqueued) */
    DAMAS_ENOMEM = -2,    /* scratch allocation failed */
    DAMAS_ECUDA = -3,     /* a CUDA runtime call failed */
    DAMAS_ETIMEDOUT = -4, /* a bounded device-side wait gave up (see damas_solve) */
    DAMAS_EBUSY = -5,     /* resource busy (serving queue full) */
    DAMAS_ENOTFOUND = -6  /* unknown ticket */
};

/* PSF-matrix formulations.
 * E: e_n = g_n / ||g_n|| with g of Eq. (7); A_nm = |e_n^H e_m|^2, b_n = Re(e_n^H C e_n).
 *    A is symmetric, positive semi-definite, with unit diagonal.  The solution is
 *    x'_n = x_n ||g_n||^2; damas_scatter_power divides by ||g_n||^2.
 * P: the paper's literal v (Eq. (4)) and g (Eq. (7)): A_ns = PSF(r_n|r_s) =
 *    |v_n^H g_s|^2 / M^2 (Eq. (10)), b_n = Re(v_n^H C v_n) / M^2 (Eq. (2));
 *    unit diagonal, not symmetric; x is in power units directly. */
enum { DAMAS_FORM_E = 0, DAMAS_FORM_P = 1 };

/* Storage type of A. */
enum { DAMAS_F32 = 1, DAMAS_BF16 = 2 };

/* Interpolation used by the wavelet coefficient of Eq. (23):
 * LINEAR (edge: mean of the two coarse neighbours, centre: mean of the four
 * coarse corners) or HAAR (constant: the lower-left coarse neighbour). */
enum { DAMAS_PRED_LINEAR = 0, DAMAS_PRED_HAAR = 1 };

/* How the threshold eps of Eq. (22) is formed:
 * ABS       eps as given;
 * REL_MAX   eps * max_n b_n (FP32 product);
 * KEEP_FRAC eps is a fraction f: the threshold is the K-th largest |detail|
 *           outside G^0 with K = ceil(f * nx * ny) - |G^0| (K <= 0 keeps G^0
 *           only; ties at the threshold are all kept). */
enum { DAMAS_EPS_ABS = 0, DAMAS_EPS_REL_MAX = 1, DAMAS_EPS_KEEP_FRAC = 2 };

typedef struct {
    int M;                   /* number of microphones, 1..DAMAS_MAX_MICS */
    const double *mic_xyz_dev; /* device, M x 3 doubles (x, y, z) in metres, array plane z = 0 */
    int nx, ny;              /* scan grid size, S = nx * ny */
    double x0, y0, dx, dy, z; /* scan grid origin, spacing and plane distance (metres) */
    double c;                /* speed of sound c0 (m/s); k = 2 pi f / c0 (§2) */
    int formulation;         /* DAMAS_FORM_E or DAMAS_FORM_P */
    int diag_removal;        /* 1: the CSM diagonal (auto-spectra) is removed (§2): das_map and
                                damas_build_psf_dr drop the m = m' microphone pairs; 0: off */
} damas_geom;

#define DAMAS_MAX_MICS 256

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`.  Allocates nothing yet. */
int damas_create(damas_ctx **out, int device);
/* Free the context and its scratch memory (synchronises the device). */
int damas_destroy(damas_ctx *ctx);
/* Message of the last failed call on ctx (static storage owned by ctx). */
const char *damas_last_error(const damas_ctx *ctx);
/* Context options (damas_set_option). */
enum {
    /* Bound, in milliseconds (1..600000, default 2000), on every device-side wait
     * of the build kernels (the PSF Gram of damas_build_psf / damas_build_psf_dr). */
    DAMAS_OPT_BUILD_TIMEOUT_MS = 1,
    /* Test hook of those bounded waits, 0 in normal use: 1 makes every later PSF
     * Gram launch on the context first wait for a device flag that nothing sets,
     * so the wait runs out after the build timeout and the launch takes its abort
     * path (no GPU fault is involved).  Set it back to 0 to build normally. */
    DAMAS_OPT_TEST_HOLD_BUILD = 2,
    /* Cap, in bytes, on the device memory the context holds (0, the default: no
     * cap).  Scratch that would take the context above it is refused with
     * DAMAS_ENOMEM (nothing is freed or launched); it is also the serving loop's
     * request budget when damas_serve_cfg.hbm_budget_bytes is 0.  A cap below
     * what the context already holds is refused with DAMAS_EINVAL. */
    DAMAS_OPT_HBM_BUDGET_BYTES = 3
};
int damas_set_option(damas_ctx *ctx, int option, long long value);

/*
 * Synchronise `stream` and report whether a build kernel enqueued on this
 * context gave up a bounded device wait since the last damas_check:
 * DAMAS_ETIMEDOUT (the status is then cleared) or DAMAS_OK.  The build calls
 * (damas_build_psf, damas_build_psf_dr) return as soon as their kernels are
 * enqueued, so a wait that runs out inside them cannot be their return value:
 * the Gram writes NaN where it stopped, lets its in-flight loads land, and sets
 * the context's build status, which damas_check reads and every later
 * damas_solve on the context sees (it then reports DAMAS_ETIMEDOUT and leaves
 * x and the state untouched) until damas_check clears it.
 */
int damas_check(damas_ctx *ctx, damas_stream stream);

/* Row stride, in elements, that the library uses for an S x S matrix A:
 * S rounded up to a multiple of 32 (every row 128-byte aligned for FP32). */
int damas_lda(int S);

/* Floats of the optional solver state of a system with S unknowns (damas_system.state_dev):
 * the residual as an FP32 pair per row plus the two last blocks of dx not yet folded into
 * every row.  Returns 0 for S < 1. */
int damas_state_floats(int S);

/* ------------------------------------------------------------------ a1 + a4: PSF matrix */

/*
 * PSF matrix of Eq. (10) arranged as A of Eq. (12), restricted to a set of grid
 * points (Eq. (24)) when idx_dev is given.
 *   idx_dev   device int32[S_sub], ascending grid indices, or NULL for all
 *             S = nx*ny points in order (then S_sub must equal S).
 *   A_dev     device, S_sub x lda, row-major, lda = damas_lda(S_sub), 16-byte
 *             aligned (the solver reads its rows by TMA and 16-byte vectors); FP32 when
 *             a_dtype = DAMAS_F32, bfloat16 when DAMAS_BF16.  A[n][m] for the
 *             n-th and m-th selected points; the diagonal is stored as exactly 1;
 *             padding columns S_sub..lda-1 are written as 0.
 *   gnorm2_dev optional device float[S_sub]: ||g_n||^2 of the selected points
 *             (formulation E uses it to turn x' into power).
 * Steering and propagation vectors are formed with the distance and the phase
 * k*d in FP64, reduced to a fraction of a period before an FP32 sine/cosine;
 * amplitudes and ||g||^2 are FP32 (the latter a compensated sum); the complex
 * Gram products accumulate in FP32.  FP64 serves the phase argument only.  The Gram's device waits are bounded
 * (DAMAS_OPT_BUILD_TIMEOUT_MS); one that runs out is reported by damas_check
 * and by the next damas_solve on the context, not by this call.
 */
int damas_build_psf(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev,
                    int S_sub, int a_dtype, void *A_dev, int lda, float *gnorm2_dev, damas_stream stream);

/*
 * The same PSF matrix in both storage types at once, for the mixed-precision
 * schedule (damas_solve_mixed): one FP32 build as damas_build_psf, then its BF16
 * copy rounded to nearest even, which is bit for bit what damas_build_psf with
 * DAMAS_BF16 stores.  A_f32_dev: device float S_sub x lda; A_bf16_dev: device
 * bfloat16 S_sub x lda, 16-byte aligned, not overlapping A_f32_dev (DAMAS_EINVAL
 * otherwise); other arguments as damas_build_psf.
 */
int damas_build_psf_f32_bf16(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev,
                             int S_sub, float *A_f32_dev, void *A_bf16_dev, int lda, float *gnorm2_dev,
                             damas_stream stream);

/*
 * PSF with the CSM diagonal removed (§2), for geom->diag_removal = 1 (which
 * damas_build_psf rejects): the response at point n to a unit source at s
 * without the m = m' microphone pairs,
 *   A_ns = scale * ( |sum_m conj(l_nm) r_sm|^2 - sum_m |l_nm|^2 |r_sm|^2 ),
 * whose diagonal d_n is no longer 1 and which has negative entries.  Returned
 * rescaled to a unit diagonal, A'_ns = A_ns / (sqrt(d_n) sqrt(d_s)) (A'_nn = 1
 * exactly), the form the solver takes: the clamped iteration on (A', b') with
 * b'_n = b_n / sqrt(d_n) is, step for step, the one on (A, b) with
 * x_n = x'_n / sqrt(d_n) (Eq. (14): the division by A_ii becomes the scaling).
 *   A_dev       device float S_sub x lda (FP32 only).
 *   gnorm2_dev  optional device float[S_sub]: ||g_n||^2 as in damas_build_psf.
 *   dscale_dev  device float[S_sub]: sqrt(d_n).  damas_divide turns the
 *               restricted map into b' and the solution x' into x.
 */
int damas_build_psf_dr(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const int32_t *idx_dev, int S_sub,
                       float *A_dev, int lda, float *gnorm2_dev, float *dscale_dev, damas_stream stream);

/* v[i] = v[i] / div[i], i < n (device arrays). */
int damas_divide(damas_ctx *ctx, float *v_dev, const float *div_dev, int n, damas_stream stream);

/* ------------------------------------------------------------------ a2: DAS map */

/*
 * Mean-square DAS map of Eq. (2) on the full grid.
 *   C_dev  device, M x M complex cross-spectral matrix (Eq. (1)), row-major,
 *          interleaved (re, im) FP32 pairs, 8-byte aligned; assumed Hermitian.
 *   b_dev  device float[nx*ny] output, FP32, real part of v^H C v (scaled as
 *          the formulation says); with geom->diag_removal the terms of the CSM
 *          diagonal are left out.
 */
int das_map(damas_ctx *ctx, const damas_geom *geom, double freq_hz, const float *C_dev, float *b_dev,
            damas_stream stream);

/* ------------------------------------------------------------------ acquisition: CSM from time series */

/*
 * Cross-spectral matrix (Eq. (1)) of selected frequency bins estimated from
 * microphone time series (Welch): blocks of K samples every hop samples,
 * periodic Hann window w(t) = (1 - cos(2 pi t / K)) / 2, L = (T - K) / hop + 1
 * blocks,
 *   C_f = sum_l X_lf X_lf^H / (L * sum_t w(t)^2),
 *   X_lf[m] = sum_t w(t) p[m][l*hop + t] exp(-2 pi i bins[f] t / K),
 * so that a source of variance P per sample gives C = P a a^H for its transfer
 * vector a, the form das_map takes (the same exp(-j k d) convention).
 *   p_dev     device float[M][T] (row-major; T >= K).
 *   bins_dev  device int32[F]: DFT bin indices, 0..K/2 (bin f is bins[f] * fs / K Hz).
 *   C_dev     device float[F][M][M][2] output, interleaved (re, im), 8-byte aligned,
 *             exactly Hermitian.
 * Limits: M 1..DAMAS_MAX_MICS, K 2..1048576, hop >= 1, F 1..4096, M * L <= 4194240.
 * The DFT of the selected bins runs as a tiled product of the sample blocks
 * with a window-and-twiddle table (angles reduced exactly in integers to a
 * fraction of a period in [-1/2, 1/2], FP32 sine and cosine); products and sums
 * in FP32.
 */
int damas_csm(damas_ctx *ctx, const float *p_dev, int M, long long T, int K, int hop, const int32_t *bins_dev,
              int F, float *C_dev, damas_stream stream);

/* ------------------------------------------------------------------ a3: compressed grid */

typedef struct {
    int levels;     /* J of Algorithm 1: level-0 grid = multiples of 2^J on both axes; 1..15 */
    int predictor;  /* DAMAS_PRED_LINEAR or DAMAS_PRED_HAAR */
    int eps_mode;   /* DAMAS_EPS_ABS, DAMAS_EPS_REL_MAX or DAMAS_EPS_KEEP_FRAC */
    double eps;     /* threshold, or kept fraction for KEEP_FRAC */
} damas_wavelet_cfg;

/*
 * Algorithm 1: the wavelet-compressed computational grid of the map b.
 * For j = J-1 down to 0 every point of G^{j+1} \ G^j is kept when
 * |interpolated(b from G^j) - b| >= eps (Eq. (22)-(23)); G^0 is always kept;
 * the result is the union as ascending grid indices.  The interpolation, the
 * threshold and the comparison are evaluated in FP32 in a fixed order:
 * edge = 0.5f*(a + c), centre = 0.25f*((b(-,-) + b(+,-)) + (b(-,+) + b(+,+))),
 * detail = prediction - b.  Coarse neighbours beyond the last row or column do
 * not exist; the prediction then averages the neighbours that do.
 *   b_dev       device float[nx*ny] input map.
 *   idx_dev     device int32[nx*ny] (capacity) output, ascending.
 *   S_sub_dev   device int32[1] output: the number of kept points S~.
 *   detail_dev  optional device float[nx*ny]: prediction - b (0 on G^0).
 *   eps_abs_dev optional device float[1]: the absolute threshold used.
 * Limits: nx, ny in 1..65535, nx*ny <= 4194304.
 */
int wavelet_compress_grid(damas_ctx *ctx, const float *b_dev, int nx, int ny, const damas_wavelet_cfg *cfg,
                          int32_t *idx_dev, int32_t *S_sub_dev, float *detail_dev, float *eps_abs_dev,
                          damas_stream stream);

/*
 * wavelet_compress_grid without any device allocation.  The paper has no
 * counterpart: this is a service for callers that cannot allocate device memory
 * when they need a compressed grid (a real-time audio thread that must not wait
 * on the driver's allocator, a plug-in that may only use memory its host
 * application gave it, a process whose device-memory budget is fixed at
 * start-up).  It computes exactly what wavelet_compress_grid computes, from the
 * same arguments; the caller still provides every input and output buffer.
 *  - Its one work array is a file-scope device array of DAMAS_NOALLOC_MAX_POINTS
 *    floats (1 MiB) inside libdamas.so; every device that loads the library holds
 *    it until the process exits.  Grids with more than DAMAS_NOALLOC_MAX_POINTS
 *    points are rejected with DAMAS_EINVAL and nothing is enqueued.
 *  - The first call on a device looks up the array's device address (once per
 *    device, under a lock, with that device current); make that first call
 *    before any stream capture.  The address is kept for the life of the
 *    process: after a cudaDeviceReset (which also invalidates every context and
 *    its scratch) this entry point must not be used on that device again.
 *  - Limits are those of wavelet_compress_grid (nx, ny in 1..65535) and, in
 *    addition, nx*ny <= DAMAS_NOALLOC_MAX_POINTS.
 *  - Every call on a device uses the same array, which keeps whatever the last
 *    call left there (nothing in it has to start at zero: each call writes every
 *    entry it reads).  Calls whose work overlaps on the GPU (different streams,
 *    or different host threads) race on it: serialise them.
 *  - ctx supplies the device and receives the error message; no context scratch
 *    is used.
 */
#define DAMAS_NOALLOC_MAX_POINTS 262144
int wavelet_compress_grid_noalloc(damas_ctx *ctx, const float *b_dev, int nx, int ny, const damas_wavelet_cfg *cfg,
                                  int32_t *idx_dev, int32_t *S_sub_dev, float *detail_dev, float *eps_abs_dev,
                                  damas_stream stream);

/*
 * Neighbour padding of a compressed grid.  An extension, not part of
 * Algorithm 1: §5 reports that DAMAS on the compressed grid aliases more on an
 * extended source because kept points lie further apart there, and its remedy
 * is a smaller eps (a denser grid everywhere).  Padding instead adds every grid
 * point within Chebyshev distance `radius` of a kept point, which gives the
 * kept regions back their full spacing and leaves the rest of the grid sparse.
 *   idx_dev      device int32[*S_sub_dev]: grid indices (any order, repeats
 *                allowed; entries outside [0, nx*ny) are ignored).
 *   S_sub_dev    device int32[1]: their number (a value outside [0, nx*ny] is
 *                clamped to that range).
 *   radius       0..8; 0 returns the input set sorted without repeats.
 *   out_idx_dev  device int32[nx*ny] (capacity) output: the padded set, ascending.
 *                May be the same buffer as idx_dev.
 *   out_S_dev    device int32[1] output: its size.
 * Limits: nx, ny in 1..65535, nx*ny <= 4194304.  The selection is integer work
 * and deterministic.
 */
int damas_pad_grid(damas_ctx *ctx, int nx, int ny, const int32_t *idx_dev, const int32_t *S_sub_dev, int radius,
                   int32_t *out_idx_dev, int32_t *out_S_dev, damas_stream stream);

/* ------------------------------------------------------------------ a5, a7: restriction and scatter */

/* dst[i] = src[idx[i]], i < n (b~ of Eq. (24)). */
int damas_gather(damas_ctx *ctx, const float *src_dev, const int32_t *idx_dev, int n, float *dst_dev,
                 damas_stream stream);

/*
 * Compressed-grid solution back onto the full grid (§5: zero off the kept
 * points), converted to power units:
 *   x_full[idx[i]] = x_sub[i] / gnorm2[i]   (gnorm2_dev given, formulation E)
 *   x_full[idx[i]] = x_sub[i]               (gnorm2_dev NULL)
 * every other entry of x_full[S] is set to 0.  idx_dev NULL means the identity
 * (n == S).  total_power_dev (optional, device double[1]) receives the
 * integrated power sum_n x_full[n] (Table 1): a compensated FP32 sum in a fixed
 * order, returned exactly as the double value of its (hi, lo) pair.
 */
int damas_scatter_power(damas_ctx *ctx, const float *x_sub_dev, const int32_t *idx_dev, const float *gnorm2_dev,
                        int n, float *x_full_dev, int S, double *total_power_dev, damas_stream stream);

/* ------------------------------------------------------------------ a6: DAMAS iteration */

/* How a solve starts. */
enum {
    DAMAS_INIT_ZERO = 0,  /* x^0 = 0 (the paper's choice, §3); x_dev is overwritten */
    DAMAS_INIT_X = 1,     /* continue from x_dev: the residual A x - b is recomputed */
    DAMAS_INIT_STATE = 2  /* continue from x_dev and the residual kept in state_dev by
                             an earlier solve of the same system: bit-identical to one
                             longer solve */
};

typedef struct {
    const void *A_dev;  /* S x lda, row-major, FP32 or BF16 (a_dtype), unit diagonal,
                           16-byte aligned (as At_dev; b, x and state float-aligned);
                           entries >= 0 (PSF matrices are) let rows that cannot move be
                           skipped exactly; a block with a negative entry is solved in full */
    const void *At_dev; /* A transposed, same type and lda, or NULL when A is symmetric
                           (formulation E).  Read when A's rows are not held in shared
                           memory: column c of A is then read as row c of At */
    int a_dtype;        /* DAMAS_F32 or DAMAS_BF16 */
    int lda;            /* row stride in elements, multiple of 32, >= S (damas_lda) */
    int S;              /* number of unknowns, >= 1 */
    const float *b_dev; /* device float[S] */
    float *x_dev;       /* device float[S], in/out */
    float *state_dev;   /* optional device float[damas_state_floats(S)] (2*S + 64): the iteration's internal state
                           (residual as an FP32 pair hi/lo plus the last two blocks of
                           dx not yet folded into every row); opaque, written at the
                           end of every solve, read with DAMAS_INIT_STATE */
    int init;           /* DAMAS_INIT_* */
    int iters;          /* number of sweeps T >= 0 */
    int ctas;           /* CTAs in this system's team; 0 = cfg->ctas_per_system or automatic */
} damas_system;

typedef struct {
    int ctas_per_system;  /* 0 = automatic; otherwise the number of cooperating CTAs per system */
    int timeout_ms;       /* bound on every device-side wait, default (0) 2000 ms */
    int32_t *status_dev;  /* optional device int32[1]: receives DAMAS_OK or DAMAS_ETIMEDOUT;
                             when given the call does not synchronise */
    int a_placement;      /* 0 = automatic; 1 = keep each CTA's rows of A in shared memory
                             (DAMAS_EINVAL if they do not fit); 2 = stream A tiles from
                             global memory (L2/HBM) through a shared-memory ring */
    int withhold_block;   /* test hook for the bounded waits, 0 in normal use: when > 0 the
                             owner of row block (withhold_block - 1) never publishes it, so
                             the waits of the other CTAs for it run out */
    uint64_t *stats_dev;  /* optional device uint64[3], added to by the call: 32-row blocks
                             solved, rows that entered a block's chain (those that could
                             move; systems of one block leave this out), nonzero dx
                             entries.  For measurement: the sequential chain's length and
                             the columns of A the folds must read */
} damas_solve_cfg;

/*
 * DAMAS iteration, Eq. (13)-(14) (§3), for nsys independent systems in one
 * persistent launch: for each sweep, for i = 1..S in order,
 *   r_i = sum_{j<i} A_ij x_j^(n+1) + sum_{j>=i} A_ij x_j^(n) - b_i,
 *   x_i = max(x_i - r_i / A_ii, 0),  with A_ii = 1.
 * The row order is exactly the paper's.  Rows are processed in blocks of 32:
 * a block is solved sequentially on chip from its residual, and the change of
 * x is applied to the residual of every other row (A[:,J] dx_J) while the next
 * block is being solved.  The residual is carried as an FP32 (hi, lo) pair
 * updated with error-free transformations, so it does not drift over thousands
 * of sweeps.
 *   sys    host array of nsys descriptors (copied before the call returns).
 *   cfg    optional (NULL = defaults).
 * A system runs in one of two forms with bit-identical results (x and state):
 *  - single CTA: one CTA of 512 threads holds the whole system's x and
 *    residual, reads A from global memory (tiles a few steps ahead by TMA, the
 *    entries of each fold as vector loads) and hands nothing to other CTAs.  Used
 *    for a system of 97 or more rows whose rows fit the CTA's shared memory
 *    when it is asked for one CTA (ctas = 1) with a_placement 0 or 2, or, by
 *    default, when it has at most 1024 rows; and only when every system of the
 *    call takes this form (such a launch needs no co-residency, so any number
 *    of systems run in it);
 *  - team: CTAs that run concurrently (a cooperative launch, or one
 *    thread-block cluster per team when all teams are equal, 2-16 CTAs, and fit
 *    at once; every team must fit on the device at once) own contiguous row
 *    blocks and hand each block's dx on through global memory.
 * Every device-side wait is bounded by cfg->timeout_ms; a wait that runs out
 * makes the kernel stop and report DAMAS_ETIMEDOUT.  Without cfg->status_dev
 * the call synchronises the stream and returns that status; with it the call
 * returns at once and the status lands in *status_dev.
 */
int damas_solve(damas_ctx *ctx, const damas_system *sys, int nsys, const damas_solve_cfg *cfg,
                damas_stream stream);

/*
 * Mixed-precision schedule of the iteration (the precision study's form): for
 * each system, iters_bulk sweeps of Eq. (13)-(14) with A stored in BF16 (half
 * the bytes of A per sweep) from x^0 = 0, then iters_refine sweeps with A in
 * FP32 that restart from the exact FP32 residual A x - b of the bulk phase's x
 * (DAMAS_INIT_X), in one call.  iters_bulk = 0 solves with the FP32 A from
 * x^0 = 0; iters_refine = 0 stops after the bulk phase.  The result is bit for
 * bit that of the two damas_solve calls it stands for.
 *   A_bulk_dev / At_bulk_dev     BF16 A and its transpose (NULL: A symmetric)
 *   A_refine_dev / At_refine_dev FP32 A and its transpose (NULL: A symmetric)
 *   lda                          row stride of both, in elements (a multiple of 32)
 * cfg and the status follow damas_solve: the status reports the first wait that
 * ran out in either phase (withhold_block must be 0).  The two phases run as
 * two launches on the stream; without cfg->status_dev the call synchronises
 * once, at the end.
 */
typedef struct {
    const void *A_bulk_dev, *At_bulk_dev;
    const void *A_refine_dev, *At_refine_dev;
    int lda, S;
    const float *b_dev; /* device float[S] */
    float *x_dev;       /* device float[S], output */
    int iters_bulk, iters_refine;
    int ctas;           /* as damas_system.ctas */
} damas_mixed_system;
int damas_solve_mixed(damas_ctx *ctx, const damas_mixed_system *sys, int nsys, const damas_solve_cfg *cfg,
                      damas_stream stream);

/*
 * The plan damas_solve would choose for one system of S rows when it is the
 * only system of the call (host only; no device work): CTAs in its team, rows
 * per CTA, and whether the CTAs keep their rows of A in shared memory (1) or
 * stream them (0).  ctas and a_placement mean what damas_solve_cfg's
 * ctas_per_system and a_placement mean.  *ncta_out = 1 with S >= 97 is the
 * single-CTA form.  Blocks of 32 rows are owned contiguously, so one sweep hands
 * the iteration from CTA to CTA *ncta_out times when *ncta_out > 1.
 */
int damas_solve_plan(damas_ctx *ctx, int S, int lda, int a_dtype, int ctas, int a_placement, int *ncta_out,
                     int *rows_per_cta_out, int *resident_out);

/*
 * Measurement aid, not part of the method: the one-way latency of handing a
 * value from one CTA to another the way damas_solve's teams hand each block's dx
 * to the next owner (a relaxed 64-bit store to global memory, polled with
 * relaxed loads).  CTA 0 of a cooperative launch passes a counter back and forth
 * with each of CTAs 1..npairs in turn, `rounds` times.
 *   rounds     1..100000.
 *   max_pairs  pairs to measure, capped at the SM count - 1 (>= 1).
 *   timeout_us bound on every wait in microseconds (0: 2 s); a wait that runs out
 *              makes the call return DAMAS_ETIMEDOUT (the device stays usable).
 *   ns_host    host double[max_pairs] output: mean nanoseconds per one-way hand-over
 *              for each pair.
 *   n_pairs    host int output: pairs measured.
 * Synchronises the stream.
 */
int damas_handover_probe(damas_ctx *ctx, int rounds, int max_pairs, int timeout_us, double *ns_host, int *n_pairs,
                         damas_stream stream);

/*
 * Measurement aid, not part of the method: the latency of the row chain of a
 * block solve on this device.  One CTA of 512 threads: warp 0 runs `rounds`
 * dependent candidate updates as a block solve does them (broadcast of the
 * candidate's w by shuffle, the clamp as a max with -x, one FMA into every
 * lane's w), then all 16 warps run `rounds` CTA-barrier steps.
 *   rounds   1..10000000.
 *   ns_host  host double[2] output: ns per candidate update, ns per barrier step.
 * Synchronises the stream.  With the counts of damas_solve_cfg.stats_dev,
 * candidates x ns[0] + blocks x ns[1] is the time the sweep's sequential
 * dependence alone takes on one CTA.
 */
int damas_chain_probe(damas_ctx *ctx, int rounds, double *ns_host, damas_stream stream);

/* ------------------------------------------------------------------ serving */

/*
 * A request loop with continuous batching: requests arriving while others run
 * are admitted as device memory and SM slots free up, each in its own stream,
 * and their kernels overlap on the device.  Each request is one measurement
 * (one array, one grid, several frequency bins); each bin goes through the
 * method of §5: DAS map, compressed grid (Algorithm 1) unless wavelet.levels is
 * 0, PSF matrix, Gauss-Seidel from x = 0, power map.  The result of a request
 * does not depend on what else is in flight (bit for bit).
 */
/* Admission: a queued request starts (stage 1: uploads, DAS maps, compressed
 * grids) when a pool slot is free and its stage-1 memory plus the least its
 * stage 2 can need (every bin keeps at least G^0, and ceil(f S) points with a
 * keep fraction f) fit hbm_budget_bytes beside the requests in flight; its
 * matrices and solve (stage 2) are admitted when their memory fits the budget
 * and the solve's share of the SMs fits the free sm_slots.  A request that does
 * not fit even alone runs when nothing else is in flight, and stage 2 is always
 * granted when no other request is solving, so a small budget slows the loop
 * but never stalls it (the budget can then be exceeded by that one request). */
typedef struct {
    size_t hbm_budget_bytes; /* device memory the loop may hold for requests; 0 = the context's
                                DAMAS_OPT_HBM_BUDGET_BYTES if set, else half the free memory */
    int max_inflight;        /* requests on the device at once; 0 = 32 */
    int sm_slots;            /* half-SM units that concurrent solves may hold together; 0 = twice the SM
                                count (the whole device).  A solve is charged by the library's plan of
                                it: a CTA that fills its SM (one CTA per SM: the single-CTA form,
                                teams holding A in shared memory) counts 2, a CTA of a launch that
                                fits two or more per SM counts 1 */
    int rows_per_cta;        /* solver team size target, rows per CTA; 0 = 768 */
} damas_serve_cfg;

typedef struct {
    int M;                     /* microphones */
    const double *mic_xyz;     /* HOST, M x 3 (copied at submit) */
    int nx, ny;
    double x0, y0, dx, dy, z, c;
    int formulation;           /* DAMAS_FORM_E (the loop's PSF builds assume it) */
    int n_bins;
    const double *freqs;       /* HOST, n_bins frequencies (Hz) */
    const float *C;            /* HOST, n_bins x M x M x 2 interleaved complex CSMs */
    damas_wavelet_cfg wavelet; /* compression of every bin; levels = 0 solves the full grid */
    int iters;                 /* Gauss-Seidel sweeps per bin */
} damas_request;

typedef struct {
    int status;                /* DAMAS_OK when done, DAMAS_EBUSY while in flight, or an error */
    int n_bins, S;
    const float *x;            /* host, n_bins x S power maps (valid until the ticket is released) */
    const double *total_power; /* host, n_bins integrated powers */
    const int *S_sub;          /* host, n_bins compressed sizes */
    double t_submit, t_admit, t_done; /* seconds on the host steady clock: submitted, admitted
                                         (stage 1: uploads, DAS maps, compressed grids), done */
    double t_solve;            /* when its matrices and solve were admitted (stage 2) */
    size_t hbm_bytes;          /* device memory charged to the request against hbm_budget_bytes */
    int sm_units;              /* half-SM units its solve was charged (see damas_serve_cfg.sm_slots) */
} damas_result;

/* Start the loop's worker thread on ctx's device. */
int damas_serve_start(damas_ctx *ctx, const damas_serve_cfg *cfg);
/* Copy a request in and queue it; returns a ticket.  DAMAS_EBUSY when the loop is stopped. */
int damas_serve_submit(damas_ctx *ctx, const damas_request *req, uint64_t *ticket);
/* Non-blocking: fills *res; res->status is DAMAS_EBUSY until the request is done. */
int damas_serve_poll(damas_ctx *ctx, uint64_t ticket, damas_result *res);
/* Drop a finished request's host results. */
int damas_serve_release(damas_ctx *ctx, uint64_t ticket);
/* Finish the requests in flight and stop the worker. */
int damas_serve_stop(damas_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DAMAS_H */
