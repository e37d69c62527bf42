// Descriptors of the persistent Gauss-Seidel launch.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

struct SweepSys {
    const void *A;            // S x lda, FP32 or BF16
    const void *At;           // A transposed (same lda), or A itself when A is symmetric
    const float *b;           // S
    float *x;                 // S, in/out
    float *state;             // 2*S + 64 or nullptr: residual (hi, lo) and the two pending dx blocks
    unsigned long long *mbox; // nb*32 mailbox words: (epoch << 32) | bits(dx)
    int lda, S, dtype, init, iters;
    int cta0, ncta, rows_per_cta, resident;
    unsigned epoch0;
};

constexpr int SWEEP_MAX_SYS = 64;  // systems per launch (the parameter block stays far below 32 KB)

struct SweepParams {
    SweepSys sys[SWEEP_MAX_SYS];
    int nsys;
    int *status;
    unsigned long long timeout_ns;
    int withhold_block;  // test hook: block index never published, or -1
    unsigned long long *stats;  // optional [3]: blocks solved, rows that entered the chain, nonzero dx (added to)
    const int *upstream; // the context's build status word, or nullptr: when it holds an error at
                         // launch (a build kernel gave up a wait, so A may hold NaN), the launch
                         // reports DAMAS_ETIMEDOUT and leaves x unchanged
};
static_assert(sizeof(SweepParams) <= 32000, "kernel parameter block");

// shared memory a CTA needs for R rows (resident: its rows of A; otherwise chain tiles only)
size_t sweep_smem_bytes(int R, int lda, int dtype, bool resident);
cudaError_t sweep_occupancy(size_t smem, int *blocks_per_sm);
cudaError_t launch_sweep(const SweepParams &p, int grid, size_t smem, cudaStream_t st);
// the single-CTA form: one CTA per system (S > 96), A streamed, no hand-overs;
// bit-identical iterates and state to the team form
// Tensor maps over each system's At (32 x 32 boxes), built by make_sweep_tile_map.
struct SoloMaps {
    CUtensorMap m[SWEEP_MAX_SYS];
};
size_t sweep_solo_smem_bytes(int R, int dtype);
cudaError_t sweep_solo_occupancy(size_t smem, int *blocks_per_sm);
bool make_sweep_tile_map(CUtensorMap *m, const void *At, int dtype, int lda, int S);
cudaError_t launch_sweep_solo(const SweepParams &p, const SoloMaps &maps, size_t smem, cudaStream_t st);
