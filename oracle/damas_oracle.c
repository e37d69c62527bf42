/*
 * Oracle for the DAMAS-on-a-wavelet-compressed-grid hot path (Ma & Liu,
 * "Improving the Efficiency of DAMAS for Sound Source Localization via
 * Wavelet Compression Computational Grid").
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, obviously correct CPU
 * implementation used to check the CUDA library; it shares no code with it and
 * the product path never calls it.  Floating point is FP64 except where the
 * method turns floating point into an integer decision (the wavelet grid
 * selection), which is evaluated in FP32 with a fixed expression order so that
 * both sides take the same decision.  Build with -ffp-contract=off.
 *
 * Equation numbers follow the order of the paper's displayed equations:
 *   (1) CSM, (2) DAS map, (4) steering component v_m, (7) propagation g_m,
 *   (8) incoherent CSM, (10) PSF, (12) Ax=b, (13)-(14) Gauss-Seidel step,
 *   (15) nested grids, (20) Donoho bound, (21)-(22) compressed grid,
 *   (23) interpolating wavelet coefficient, (24) compressed system.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_VEC_G 0 /* propagation vector g(r), Eq. (7) */
#define ORC_VEC_V 1 /* steering vector v(r), Eq. (4) */
#define ORC_VEC_E 2 /* normalised propagation vector e = g / |g| */

/*
 * Vectors of S points (pts, S x 3) towards M microphones (mic, M x 3), wave
 * number k.  Output row n holds the M complex components (re, im planes, S x M).
 *   g_m(r) = |r| / |r - r_m| * exp(-j k |r - r_m|)      Eq. (7), exponent read as r_s
 *   v_m(r) = |r - r_m| / |r| * exp(-j k |r - r_m|)      Eq. (4)
 *   e(r)   = g(r) / ||g(r)||_2
 * gnorm2 (optional, length S) receives ||g(r)||_2^2.
 */
void orc_vectors(int M, const double *mic, int S, const double *pts, double k, int kind,
                 double *re, double *im, double *gnorm2)
{
    for (int n = 0; n < S; ++n) {
        const double *p = pts + 3 * (size_t)n;
        double rabs = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
        double g2 = 0.0;
        for (int m = 0; m < M; ++m) {
            double dx = p[0] - mic[3 * m + 0];
            double dy = p[1] - mic[3 * m + 1];
            double dz = p[2] - mic[3 * m + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double g_amp = rabs / d;
            g2 += g_amp * g_amp;
        }
        double inv_norm = 1.0 / sqrt(g2);
        if (gnorm2) gnorm2[n] = g2;
        for (int m = 0; m < M; ++m) {
            double dx = p[0] - mic[3 * m + 0];
            double dy = p[1] - mic[3 * m + 1];
            double dz = p[2] - mic[3 * m + 2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double amp;
            if (kind == ORC_VEC_G) amp = rabs / d;
            else if (kind == ORC_VEC_V) amp = d / rabs;
            else amp = (rabs / d) * inv_norm;
            double ph = -k * d;
            re[(size_t)n * M + m] = amp * cos(ph);
            im[(size_t)n * M + m] = amp * sin(ph);
        }
    }
}

/*
 * PSF matrix, Eq. (10) arranged column-wise into A (Eq. (12)):
 *   A[n][s] = scale * | sum_m conj(l_nm) * r_sm |^2
 * With l = v, r = g, scale = 1/M^2 this is PSF(r_n | r_s) (formulation P);
 * with l = r = e and scale = 1 it is |e_n^H e_s|^2 (formulation E).
 * The diagonal is 1 in exact arithmetic for both; it is stored as exactly 1.0
 * so that the division by A_ii in Eq. (14) is exact.
 * A is S x S, row-major, row stride lda (>= S).
 */
void orc_psf(int S, int M, const double *lre, const double *lim, const double *rre,
             const double *rim, double scale, double *A, int lda)
{
    for (int n = 0; n < S; ++n) {
        for (int s = 0; s < S; ++s) {
            double gr = 0.0, gi = 0.0;
            for (int m = 0; m < M; ++m) {
                double ar = lre[(size_t)n * M + m], ai = -lim[(size_t)n * M + m]; /* conj(l) */
                double br = rre[(size_t)s * M + m], bi = rim[(size_t)s * M + m];
                gr += ar * br - ai * bi;
                gi += ar * bi + ai * br;
            }
            A[(size_t)n * lda + s] = scale * (gr * gr + gi * gi);
        }
        A[(size_t)n * lda + n] = 1.0;
    }
}

/*
 * Mean-square DAS map, Eq. (2): b_n = scale * Re( l_n^H C l_n ),
 * C is M x M complex, row-major, interleaved (re, im).  scale = 1/M^2 with l = v
 * (formulation P) or 1 with l = e (formulation E).  The imaginary part is zero
 * for Hermitian C up to rounding and is returned in bim (optional) for checking.
 */
void orc_das(int S, int M, const double *re, const double *im, const double *C, double scale,
             double *b, double *bim)
{
    for (int n = 0; n < S; ++n) {
        double sr = 0.0, si = 0.0;
        for (int p = 0; p < M; ++p) {
            /* (C l_n)_p */
            double yr = 0.0, yi = 0.0;
            for (int q = 0; q < M; ++q) {
                double cr = C[2 * ((size_t)p * M + q)], ci = C[2 * ((size_t)p * M + q) + 1];
                double lr = re[(size_t)n * M + q], li = im[(size_t)n * M + q];
                yr += cr * lr - ci * li;
                yi += cr * li + ci * lr;
            }
            double lr = re[(size_t)n * M + p], li = -im[(size_t)n * M + p]; /* conj(l_p) */
            sr += lr * yr - li * yi;
            si += lr * yi + li * yr;
        }
        b[n] = scale * sr;
        if (bim) bim[n] = scale * si;
    }
}

/*
 * Diagonal removal (§2: the auto-spectra on the CSM diagonal are dropped to
 * suppress uncorrelated microphone self-noise).  Both the map and the PSF then
 * exclude the m = m' terms of their double sums over microphone pairs:
 *   b_n  = scale * Re( sum_{p != q} conj(l_np) C_pq l_nq )
 *   A_ns = scale * sum_{m != m'} conj(l_nm) r_sm conj(r_sm') l_nm'
 * (the PSF is the map of a unit source at s, C = r_s r_s^H).  A_nn is no
 * longer 1; it is computed like every other entry.  Written as the plain
 * double sums: O(M^2) per entry.
 */
void orc_das_dr(int S, int M, const double *re, const double *im, const double *C, double scale, double *b)
{
    for (int n = 0; n < S; ++n) {
        double sr = 0.0;
        for (int p = 0; p < M; ++p) {
            double lpr = re[(size_t)n * M + p], lpi = -im[(size_t)n * M + p]; /* conj(l_p) */
            for (int q = 0; q < M; ++q) {
                if (q == p) continue;
                double cr = C[2 * ((size_t)p * M + q)], ci = C[2 * ((size_t)p * M + q) + 1];
                double lqr = re[(size_t)n * M + q], lqi = im[(size_t)n * M + q];
                /* conj(l_p) * C_pq * l_q, real part */
                double tr = lpr * cr - lpi * ci, ti = lpr * ci + lpi * cr;
                sr += tr * lqr - ti * lqi;
            }
        }
        b[n] = scale * sr;
    }
}

void orc_psf_dr(int S, int M, const double *lre, const double *lim, const double *rre, const double *rim,
                double scale, double *A, int lda)
{
    for (int n = 0; n < S; ++n) {
        for (int s = 0; s < S; ++s) {
            double acc = 0.0;
            for (int m = 0; m < M; ++m) {
                /* u = conj(l_nm) * r_sm */
                double ur = lre[(size_t)n * M + m] * rre[(size_t)s * M + m] + lim[(size_t)n * M + m] * rim[(size_t)s * M + m];
                double ui = lre[(size_t)n * M + m] * rim[(size_t)s * M + m] - lim[(size_t)n * M + m] * rre[(size_t)s * M + m];
                for (int mp = 0; mp < M; ++mp) {
                    if (mp == m) continue;
                    /* w = conj(r_sm') * l_nm' ; term = u * w, real part */
                    double wr = rre[(size_t)s * M + mp] * lre[(size_t)n * M + mp] + rim[(size_t)s * M + mp] * lim[(size_t)n * M + mp];
                    double wi = rre[(size_t)s * M + mp] * lim[(size_t)n * M + mp] - rim[(size_t)s * M + mp] * lre[(size_t)n * M + mp];
                    acc += ur * wr - ui * wi;
                }
            }
            A[(size_t)n * lda + s] = scale * acc;
        }
    }
}

/*
 * DAMAS iteration, Eq. (13)-(14) (§3), x^0 given (the paper takes x^0 = 0):
 *   r_i = sum_{j<i} A_ij x_j^(n+1) + sum_{j>=i} A_ij x_j^(n) - b_i
 *   x_i^(n+1) = max(x_i^(n) - r_i / A_ii, 0),        i = 1..S in order.
 * x is updated in place, so x[j] already holds x_j^(n+1) for j < i and x_j^(n)
 * for j >= i when row i is processed.
 */
void orc_gauss_seidel(int S, const double *A, int lda, const double *b, double *x, int iters)
{
    for (int it = 0; it < iters; ++it) {
        for (int i = 0; i < S; ++i) {
            const double *Ai = A + (size_t)i * lda;
            double lower = 0.0, upper = 0.0;
            for (int j = 0; j < i; ++j) lower += Ai[j] * x[j];
            for (int j = i; j < S; ++j) upper += Ai[j] * x[j];
            double r = lower + upper - b[i];
            double xn = x[i] - r / Ai[i];
            x[i] = xn > 0.0 ? xn : 0.0;
        }
    }
}

/* ------------------------------------------------------------------ wavelet grid */
#define ORC_PRED_LINEAR 0
#define ORC_PRED_HAAR 1
#define ORC_EPS_ABS 0
#define ORC_EPS_REL_MAX 1
#define ORC_EPS_KEEP_FRAC 2

static int cmp_float_desc(const void *a, const void *b)
{
    float x = *(const float *)a, y = *(const float *)b;
    return (x < y) - (x > y);
}

/*
 * Interpolated value of b at grid point (ix, iy) of G^{j+1} \ G^j from the
 * points of the coarser grid G^j only (Eq. (23) and Algorithm 1, step
 * "interpolate b on G^j to G^{j+1} minus G^j").  h is the spacing of G^{j+1}
 * (the spacing of G^j is 2h).  Neighbours beyond the last row/column do not
 * exist; the average is then taken over the neighbours that do.
 * FP32 with a fixed expression order:
 *   edge:   0.5f * (left + right)
 *   centre: 0.25f * ((b(-,-) + b(+,-)) + (b(-,+) + b(+,+)))
 * HAAR (constant interpolation): the lower-left coarse neighbour.
 */
static float orc_predict(const float *b, int nx, int ny, int ix, int iy, int h, int pred)
{
    int xo = (ix / h) & 1; /* ix is an odd multiple of h */
    int yo = (iy / h) & 1;
    int xl = xo ? ix - h : ix, yl = yo ? iy - h : iy; /* lower-left coarse neighbour */
    if (pred == ORC_PRED_HAAR) return b[(size_t)yl * nx + xl];
    int hasx = xo && (ix + h <= nx - 1);
    int hasy = yo && (iy + h <= ny - 1);
    if (xo && !yo) { /* neighbours left and right */
        if (!hasx) return b[(size_t)iy * nx + xl];
        return 0.5f * (b[(size_t)iy * nx + (ix - h)] + b[(size_t)iy * nx + (ix + h)]);
    }
    if (!xo && yo) { /* neighbours below and above */
        if (!hasy) return b[(size_t)yl * nx + ix];
        return 0.5f * (b[(size_t)(iy - h) * nx + ix] + b[(size_t)(iy + h) * nx + ix]);
    }
    /* centre: four corners */
    float mm = b[(size_t)(iy - h) * nx + (ix - h)];
    if (hasx && hasy) {
        float pm = b[(size_t)(iy - h) * nx + (ix + h)];
        float mp = b[(size_t)(iy + h) * nx + (ix - h)];
        float pp = b[(size_t)(iy + h) * nx + (ix + h)];
        return 0.25f * ((mm + pm) + (mp + pp));
    }
    if (hasx) return 0.5f * (mm + b[(size_t)(iy - h) * nx + (ix + h)]);
    if (hasy) return 0.5f * (mm + b[(size_t)(iy + h) * nx + (ix - h)]);
    return mm;
}

/*
 * Algorithm 1 (§4): wavelet-compressed computational grid from the DAS map b
 * (nx x ny, FP32, n = iy*nx + ix).
 *   - nested grids G^j, j = 0..J: the points whose indices are multiples of
 *     2^(J-j) on both axes (Eq. (15));
 *   - for j = J-1 down to 0, every point of G^{j+1} \ G^j is kept when
 *     |interpolated(b) - b| >= eps (Eq. (22), "not less than eps", §4);
 *   - G^0 is always kept;
 *   - the compressed grid is the union, returned as ascending indices.
 * eps_mode: ABS (eps as given), REL_MAX (eps * max_n b_n, in FP32), KEEP_FRAC
 * (the threshold is the K-th largest |d| over points outside G^0, with
 * K = ceil(eps * S) - |G^0|; ties at the threshold are all kept).
 * Outputs: idx (capacity S), detail[n] = b_bar - b (0 on G^0), level[n]
 * (0 on G^0, j+1 on G^{j+1} \ G^j), *eps_abs_out.  Returns the count S~.
 */
int orc_wavelet_select(int nx, int ny, const float *b, int J, int pred, int eps_mode, double eps,
                       int32_t *idx, float *detail, int8_t *level, float *eps_abs_out)
{
    const int S = nx * ny;
    const int step0 = 1 << J;
    int n0 = 0;
    float *absdiff = (float *)malloc(sizeof(float) * (size_t)S);
    for (int n = 0; n < S; ++n) { absdiff[n] = -1.0f; detail[n] = 0.0f; level[n] = 0; }

    /* interpolation of every level from the next coarser one */
    for (int j = J - 1; j >= 0; --j) {
        int h = 1 << (J - j - 1); /* spacing of G^{j+1} */
        int H = 2 * h;           /* spacing of G^j */
        for (int iy = 0; iy < ny; iy += h) {
            for (int ix = 0; ix < nx; ix += h) {
                if (ix % H == 0 && iy % H == 0) continue; /* in G^j */
                float bbar = orc_predict(b, nx, ny, ix, iy, h, pred);
                float diff = bbar - b[(size_t)iy * nx + ix];
                detail[(size_t)iy * nx + ix] = diff;
                absdiff[(size_t)iy * nx + ix] = fabsf(diff);
                level[(size_t)iy * nx + ix] = (int8_t)(j + 1);
            }
        }
    }
    for (int iy = 0; iy < ny; iy += step0)
        for (int ix = 0; ix < nx; ix += step0) ++n0;

    float eps_abs;
    if (eps_mode == ORC_EPS_ABS) {
        eps_abs = (float)eps;
    } else if (eps_mode == ORC_EPS_REL_MAX) {
        float bmax = b[0];
        for (int n = 1; n < S; ++n) if (b[n] > bmax) bmax = b[n];
        eps_abs = (float)eps * bmax;
    } else {
        long K = (long)ceil(eps * (double)S) - n0;
        int nd = S - n0;
        if (K <= 0) eps_abs = INFINITY;
        else if (K >= nd) eps_abs = 0.0f;
        else {
            float *tmp = (float *)malloc(sizeof(float) * (size_t)nd);
            int t = 0;
            for (int n = 0; n < S; ++n) if (level[n] > 0) tmp[t++] = absdiff[n];
            qsort(tmp, (size_t)nd, sizeof(float), cmp_float_desc);
            eps_abs = tmp[K - 1];
            free(tmp);
        }
    }
    *eps_abs_out = eps_abs;

    int cnt = 0;
    for (int n = 0; n < S; ++n) {
        int keep = (level[n] == 0) || (absdiff[n] >= eps_abs);
        if (keep) idx[cnt++] = n;
    }
    free(absdiff);
    return cnt;
}
