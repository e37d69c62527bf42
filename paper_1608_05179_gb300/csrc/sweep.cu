// DAMAS Gauss-Seidel iteration with the non-negativity clamp (§3, Eq. (13)-(14)),
// as one persistent cooperative launch over a batch of independent systems.
//
// Layout: the rows of a system are cut into blocks of 32 (the paper's row order
// is kept: block J holds rows 32J..32J+31).  A team of `ncta` CTAs serves one
// system; CTA c owns a contiguous range of blocks (its rows) and keeps, in
// shared memory, x and the residual r = A x - b of those rows, and its rows of A
// when they fit (otherwise they are streamed from global memory).
//
// Sweep, block J in order:
//  - the owner's warp 0 solves the 32 rows one after another: lane k holds row
//    k's pending value v_k = x_k - r_k and row k of the 32 x 32 diagonal block of
//    A in registers; step j broadcasts lane j's v with a shuffle, forms
//    x_j' = max(v_j, 0) and dx_j = x_j' - x_j, and every lane applies
//    v_k -= A_kj dx_j (Eq. (13)-(14) with A_jj = 1);
//  - the owner publishes dx_J (32 floats) and a release flag tagged with the
//    sweep's epoch; every other CTA of the team waits for that flag (acquire);
//  - every CTA adds A[rows, J] dx_J to the residual of all of its rows.  The
//    residual is an unevaluated FP32 pair (hi, lo) and each product and sum goes
//    through error-free transformations (TwoProduct by FMA, TwoSum), so it does
//    not drift over thousands of sweeps; the in-block chain above only decides
//    x and is then discarded.
// A block whose rows all have x = 0 and r >= 0 cannot change (every step gives
// dx = 0), so it is skipped exactly, and the flag says so.
//
// Every wait is bounded (global timer); a wait that runs out sets the status
// word to DAMAS_ETIMEDOUT and the whole team returns.
#include "common.cuh"

#include "sweep.cuh"

namespace {

constexpr int SW_THREADS = 256;
constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ float ld_relaxed_f32(const float *p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int *p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Eight consecutive A entries A[row][col..col+7] as FP32 (col multiple of 8),
// from shared memory (resident rows) or global memory.  Columns >= S read as 0.
__device__ __forceinline__ void load8(const SweepSys &s, const char *As, int lds_bytes, bool resident, int row_g,
                                      int row_l, int col, float a[8]) {
    if (s.dtype == DAMAS_F32) {
        const float4 *p = resident ? (const float4 *)(As + (size_t)row_l * lds_bytes + (size_t)col * 4)
                                   : (const float4 *)((const float *)s.A + (size_t)row_g * s.lda + col);
        const float4 u = p[0], w = p[1];
        a[0] = u.x; a[1] = u.y; a[2] = u.z; a[3] = u.w;
        a[4] = w.x; a[5] = w.y; a[6] = w.z; a[7] = w.w;
    } else {
        const uint4 *p = resident ? (const uint4 *)(As + (size_t)row_l * lds_bytes + (size_t)col * 2)
                                  : (const uint4 *)((const __nv_bfloat16 *)s.A + (size_t)row_g * s.lda + col);
        const uint4 u = p[0];
        a[0] = bf16_lo(u.x); a[1] = bf16_hi(u.x); a[2] = bf16_lo(u.y); a[3] = bf16_hi(u.y);
        a[4] = bf16_lo(u.z); a[5] = bf16_hi(u.z); a[6] = bf16_lo(u.w); a[7] = bf16_hi(u.w);
    }
    if (col + 8 > s.S) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (col + q >= s.S) a[q] = 0.f;
    }
}

// r[rows] += A[rows, J0..J0+31] * d[0..31] with compensated accumulation.
// 4 threads per row, 8 columns each; all threads of the CTA take part.
__device__ void apply_update(const SweepSys &s, const char *As, int lds_bytes, bool resident, int row0, int nrows,
                             int J0, const float *dsh, float *rh, float *rl) {
    const int sub = threadIdx.x & 3;
    float d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) d[q] = dsh[sub * 8 + q];
    for (int rb = 0; rb < nrows; rb += SW_THREADS / 4) {
        const int r = rb + (threadIdx.x >> 2);
        float hi = 0.f, c = 0.f;
        if (r < nrows) {
            float a[8];
            load8(s, As, lds_bytes, resident, row0 + r, r, J0 + sub * 8, a);
            two_prod(a[0], d[0], hi, c);
#pragma unroll
            for (int q = 1; q < 8; ++q) {
                float p, pe, t;
                two_prod(a[q], d[q], p, pe);
                two_sum(hi, p, hi, t);
                c = __fadd_rn(c, __fadd_rn(t, pe));
            }
        }
#pragma unroll
        for (int o = 2; o >= 1; o >>= 1) {
            const float h2 = __shfl_xor_sync(FULL, hi, o), c2 = __shfl_xor_sync(FULL, c, o);
            float t;
            two_sum(hi, h2, hi, t);
            c = __fadd_rn(__fadd_rn(c, c2), t);
        }
        if (sub == 0 && r < nrows) {
            float h, t;
            two_sum(rh[r], hi, h, t);
            rh[r] = h;
            rl[r] = __fadd_rn(rl[r], __fadd_rn(c, t));
        }
    }
}

__global__ void __launch_bounds__(SW_THREADS, 1) damas_sweep_kernel(const SweepParams p) {
    extern __shared__ __align__(16) char smem[];
    __shared__ float dsh[32];
    __shared__ int s_ctrl[2];  // [0] abort, [1] active

    // which system / team rank
    int si = 0;
    while (si + 1 < p.nsys && (int)blockIdx.x >= p.sys[si + 1].cta0) ++si;
    const SweepSys s = p.sys[si];
    const int c = blockIdx.x - s.cta0;
    const int S = s.S;
    const int R = s.rows_per_cta;
    const int nb = (S + 31) / 32;
    const int row0 = c * R;
    const int nrows = max(0, min(R, S - row0));
    const int jb0 = row0 / 32, jb1 = min(nb, (row0 + R) / 32);
    const bool resident = s.resident != 0;
    const int elt = s.dtype == DAMAS_F32 ? 4 : 2;
    const int lds_bytes = s.lda * elt + 16;

    float *rh = (float *)smem;
    float *rl = rh + R;
    float *xs = rl + R;
    char *As = (char *)(xs + R);

    // ---- initial state
    if (resident) {
        const int vec_per_row = s.lda * elt / 16;
        for (int e = threadIdx.x; e < nrows * vec_per_row; e += SW_THREADS) {
            const int r = e / vec_per_row, v = e % vec_per_row;
            const uint4 *src = (const uint4 *)((const char *)s.A + ((size_t)(row0 + r) * s.lda) * elt) + v;
            *((uint4 *)(As + (size_t)r * lds_bytes) + v) = *src;
        }
    }
    for (int r = threadIdx.x; r < R; r += SW_THREADS) {
        const int i = row0 + r;
        const bool ok = r < nrows;
        if (s.init == DAMAS_INIT_STATE) {
            xs[r] = ok ? s.x[i] : 0.f;
            rh[r] = ok ? s.state[i] : 0.f;
            rl[r] = ok ? s.state[S + i] : 0.f;
        } else if (s.init == DAMAS_INIT_X) {
            xs[r] = ok ? s.x[i] : 0.f;
            rh[r] = 0.f;
            rl[r] = 0.f;
        } else {
            xs[r] = 0.f;
            rh[r] = ok ? -s.b[i] : 0.f;
            rl[r] = 0.f;
        }
    }
    if (threadIdx.x == 0) s_ctrl[0] = 0;
    __syncthreads();
    if (s.init == DAMAS_INIT_X) {
        // r_i = sum_j A_ij x_j - b_i, compensated; one warp per row
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        for (int r = warp; r < nrows; r += SW_THREADS / 32) {
            const int i = row0 + r;
            float hi = 0.f, cc = 0.f;
            for (int j0 = lane * 8; j0 < S; j0 += 256) {
                float a[8];
                load8(s, As, lds_bytes, false, i, r, j0, a);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float xj = (j0 + q < S) ? s.x[j0 + q] : 0.f;
                    float pr, pe, t;
                    two_prod(a[q], xj, pr, pe);
                    two_sum(hi, pr, hi, t);
                    cc = __fadd_rn(cc, __fadd_rn(t, pe));
                }
            }
#pragma unroll
            for (int o = 16; o >= 1; o >>= 1) {
                const float h2 = __shfl_xor_sync(FULL, hi, o), c2 = __shfl_xor_sync(FULL, cc, o);
                float t;
                two_sum(hi, h2, hi, t);
                cc = __fadd_rn(__fadd_rn(cc, c2), t);
            }
            if (lane == 0) {
                float h, t;
                two_sum(hi, -s.b[i], h, t);
                rh[r] = h;
                rl[r] = __fadd_rn(cc, t);
            }
        }
        __syncthreads();
    }

    unsigned long long active_count = 0;
    const int lane = threadIdx.x & 31;
    for (int t = 0; t < s.iters; ++t) {
        const unsigned epoch = s.epoch0 + (unsigned)t + 1u;
        for (int J = 0; J < nb; ++J) {
            const int J0 = J * 32;
            const bool own = J >= jb0 && J < jb1;
            if (own) {
                if (threadIdx.x < 32) {
                    const int k = lane, i = J0 + k, r = i - row0;
                    const bool valid = i < S;
                    const float x_old = valid ? xs[r] : 0.f;
                    const float res = valid ? __fadd_rn(rh[r], rl[r]) : 0.f;
                    float v = __fsub_rn(x_old, res);
                    const bool quiet = !valid || (x_old == 0.f && v <= 0.f);
                    const bool active = !__all_sync(FULL, quiet);
                    float dk = 0.f;
                    if (active) {
                        float arow[32];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            if (valid) {
                                load8(s, As, lds_bytes, resident, i, r, J0 + 8 * q, arow + 8 * q);
                            } else {
#pragma unroll
                                for (int u = 0; u < 8; ++u) arow[8 * q + u] = 0.f;
                            }
                        }
                        float x_new = x_old;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float vj = __shfl_sync(FULL, v, j);
                            const float xj = __shfl_sync(FULL, x_old, j);
                            const float xnj = fmaxf(vj, 0.f);
                            const float dj = __fsub_rn(xnj, xj);
                            v = __fmaf_rn(-arow[j], dj, v);
                            if (k == j) {
                                x_new = xnj;
                                dk = dj;
                            }
                        }
                        if (valid) xs[r] = x_new;
                        s.dbuf[i] = dk;
                        dsh[k] = dk;
                    }
                    __syncwarp();
                    if (k == 0) {
                        // the release store orders the warp's dx stores (made
                        // visible to lane 0 by the warp barrier) before the flag
                        if (active) ++active_count;
                        if (J != p.withhold_block) st_release_u32(s.flags + J, (epoch << 1) | (active ? 1u : 0u));
                        s_ctrl[1] = active ? 1 : 0;
                    }
                }
                __syncthreads();
            } else {
                if (threadIdx.x == 0) {
                    const unsigned long long t0 = global_ns();
                    int abort = 0, act = 0;
                    for (;;) {
                        const unsigned f = ld_acquire_u32(s.flags + J);
                        if ((f >> 1) >= epoch) {
                            act = (int)(f & 1u);
                            break;
                        }
                        if (ld_volatile_i32(p.status) != 0) {
                            abort = 1;
                            break;
                        }
                        if (global_ns() - t0 > p.timeout_ns) {
                            atomicCAS(p.status, 0, DAMAS_ETIMEDOUT);
                            abort = 1;
                            break;
                        }
                    }
                    s_ctrl[0] = abort;
                    s_ctrl[1] = act;
                }
                __syncthreads();
                if (s_ctrl[0]) return;
                if (s_ctrl[1] && threadIdx.x < 32) dsh[threadIdx.x] = ld_relaxed_f32(s.dbuf + J0 + threadIdx.x);
                __syncthreads();
            }
            if (s_ctrl[1]) apply_update(s, As, lds_bytes, resident, row0, nrows, J0, dsh, rh, rl);
            __syncthreads();
        }
    }

    for (int r = threadIdx.x; r < nrows; r += SW_THREADS) {
        s.x[row0 + r] = xs[r];
        if (s.state) {
            s.state[row0 + r] = rh[r];
            s.state[S + row0 + r] = rl[r];
        }
    }
    if (threadIdx.x == 0 && p.active_blocks && active_count) atomicAdd(p.active_blocks, active_count);
}

}  // namespace

size_t sweep_smem_bytes(int R, int lda, int dtype, bool resident) {
    size_t b = (size_t)3 * R * sizeof(float);
    if (resident) b += (size_t)R * ((size_t)lda * (dtype == DAMAS_F32 ? 4 : 2) + 16);
    return b;
}

cudaError_t sweep_occupancy(size_t smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(damas_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, damas_sweep_kernel, SW_THREADS, smem);
}

cudaError_t launch_sweep(const SweepParams &p, int grid, size_t smem, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(damas_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(SW_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, damas_sweep_kernel, p);
}
