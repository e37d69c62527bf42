// Hand-over latency probe (a measurement aid, not part of the method).  The
// Gauss-Seidel teams hand each 32-row block's dx to the next owner through
// global memory: the owner stores relaxed 64-bit words and the next owner polls
// them with relaxed loads, so every change of owner costs at least one such
// one-way hand-over.  Here CTA 0 passes a counter back and forth with CTA k,
// k = 1..npairs in turn, `rounds` times each, through one word per pair on its
// own 128-byte line, and times the rounds with the global timer.  Every wait
// is bounded; a wait that runs out sets DAMAS_ETIMEDOUT and ends that CTA, and
// the others stop at their next check of the status word.
#include "common.cuh"

namespace {

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile(const int *p) {
    int v;
    asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// false when the wait ran out (status set here) or another CTA set the status
__device__ __forceinline__ bool wait_for(const unsigned long long *f, unsigned long long want, int *status,
                                         unsigned long long timeout_ns, bool patient) {
    const unsigned long long t0 = now_ns();
    for (unsigned it = 0;; ++it) {
        if (ld_relaxed(f) == want) return true;
        if (patient) __nanosleep(500);
        if ((it & 15u) == 15u) {
            if (now_ns() - t0 > timeout_ns) {
                atomicCAS(status, 0, DAMAS_ETIMEDOUT);
                return false;
            }
            if (ld_volatile(status) != 0) return false;
        }
    }
}

__global__ void __launch_bounds__(32) handover_probe_kernel(unsigned long long *flags, int rounds, int npairs,
                                                            double *out_ns, int *status,
                                                            unsigned long long timeout_ns) {
    if (threadIdx.x != 0) return;
    const int k = blockIdx.x;
    if (k == 0) {
        for (int q = 1; q <= npairs; ++q) {
            unsigned long long *f = flags + (size_t)q * 16;
            const unsigned long long t0 = now_ns();
            for (int i = 0; i < rounds; ++i) {
                st_relaxed(f, 2ull * i + 1);
                if (!wait_for(f, 2ull * i + 2, status, timeout_ns, false)) return;
            }
            out_ns[q - 1] = (double)(now_ns() - t0) / (2.0 * rounds);
        }
    } else {
        unsigned long long *f = flags + (size_t)k * 16;
        for (int i = 0; i < rounds; ++i) {
            // the first ping comes after the earlier pairs' rounds: wait without crowding L2
            if (!wait_for(f, 2ull * i + 1, status, timeout_ns, i == 0)) return;
            st_relaxed(f, 2ull * i + 2);
        }
    }
}

// Latency of the Gauss-Seidel sweep's row chain (a measurement aid): warp 0
// runs `rounds` dependent candidate updates exactly as a block solve does them
// (the candidate's w broadcast by shuffle, the clamp as a max with -x, one FMA
// into every lane's w), then the whole CTA of SOLO_THREADS threads runs
// `rounds` barrier steps.  out[0]: ns per candidate update, out[1]: ns per
// barrier step.
constexpr int CHAIN_PROBE_THREADS = 512;
__global__ void __launch_bounds__(CHAIN_PROBE_THREADS, 1) chain_probe_kernel(int rounds, double *out, float *sink) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ unsigned long long t_start;
    float w = 1e-3f * (float)(lane + 1), xneg = -0.5f * (float)lane;
    const float a = 0.25f + 1e-3f * (float)lane;
    if (warp == 0) {
        __syncwarp();
        const unsigned long long t0 = now_ns();
        for (int i = 0; i < rounds; ++i) {
            const int j = (i * 7) & 31;
            const float wj = __shfl_sync(0xffffffffu, w, j);
            const float d = fmaxf(wj, __shfl_sync(0xffffffffu, xneg, j));
            w = __fmaf_rn(-a, d, w);
        }
        __syncwarp();
        if (lane == 0) out[0] = (double)(now_ns() - t0) / rounds;
        sink[lane] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) t_start = now_ns();
    __syncthreads();
    int acc = 0;
    for (int i = 0; i < rounds; ++i) {
        acc += (i ^ warp) & 1;
        __syncthreads();
    }
    if (threadIdx.x == 0) out[1] = (double)(now_ns() - t_start) / rounds;
    if (acc < 0) sink[32] = (float)acc;
}

}  // namespace

cudaError_t launch_chain_probe(int rounds, double *out_dev, float *sink_dev, cudaStream_t st) {
    chain_probe_kernel<<<1, CHAIN_PROBE_THREADS, 0, st>>>(rounds, out_dev, sink_dev);
    return cudaGetLastError();
}

size_t handover_probe_bytes(int npairs) { return (size_t)(npairs + 1) * 128 + (size_t)npairs * sizeof(double) + 128; }

cudaError_t launch_handover_probe(void *work, int rounds, int npairs, unsigned long long timeout_ns, cudaStream_t st,
                                  double **out_ns, int **status) {
    unsigned long long *flags = (unsigned long long *)work;
    double *ns = (double *)((char *)work + (size_t)(npairs + 1) * 128);
    int *stat = (int *)((char *)ns + (size_t)npairs * sizeof(double) + 64);
    *out_ns = ns;
    *status = stat;
    cudaError_t e = cudaMemsetAsync(work, 0, handover_probe_bytes(npairs), st);
    if (e != cudaSuccess) return e;
    void *args[] = {&flags, &rounds, &npairs, &ns, &stat, &timeout_ns};
    return cudaLaunchCooperativeKernel((const void *)handover_probe_kernel, dim3(npairs + 1), dim3(32), args, 0, st);
}
