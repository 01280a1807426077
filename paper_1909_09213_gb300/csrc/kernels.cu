// Width dispatch, set-up kernels and the shared-memory bandwidth probe.
#include <cuda_runtime.h>
#include "internal.h"

namespace cubics {

#define CUBICS_DECLARE_WIDTH(WW)                                                             \
    cudaError_t launch_search_w##WW(bool, const SearchArgs &, int, int, size_t, cudaStream_t); \
    cudaError_t occupancy_w##WW(bool, int, size_t, int *);                                   \
    cudaError_t launch_search_ext_w##WW(bool, const SearchArgs &, int, int, size_t,          \
                                        cudaStream_t);                                       \
    cudaError_t occupancy_ext_w##WW(bool, int, size_t, int *);                               \
    cudaError_t launch_prop_w##WW(bool, const PropArgs &, int, int, size_t, cudaStream_t, bool); \
    cudaError_t launch_expand_w##WW(const ExpandArgs &, int, cudaStream_t);
CUBICS_DECLARE_WIDTH(1)
CUBICS_DECLARE_WIDTH(2)
CUBICS_DECLARE_WIDTH(4)
CUBICS_DECLARE_WIDTH(8)
cudaError_t launch_search_reg(bool, const SearchArgs &, int, int, size_t, cudaStream_t);
cudaError_t occupancy_reg(bool, int, size_t, int *);

// kind: KERN_PLAIN (first-fail), KERN_EXT (learned brancher and subtree logging) or KERN_REG
// (one-word int_ne problems with register-held domains; W must be 1)
cudaError_t launch_search(int W, bool staged, int kind, const SearchArgs &A, int blocks,
                          int threads, size_t smem, cudaStream_t st) {
    if (kind == KERN_REG)
        return W == 1 ? launch_search_reg(staged, A, blocks, threads, smem, st) : cudaErrorInvalidValue;
    const bool ext = kind == KERN_EXT;
#define CUBICS_CASE(WW)                                                                      \
    case WW:                                                                                 \
        return ext ? launch_search_ext_w##WW(staged, A, blocks, threads, smem, st)           \
                   : launch_search_w##WW(staged, A, blocks, threads, smem, st);
    switch (W) {
    CUBICS_CASE(1)
    CUBICS_CASE(2)
    CUBICS_CASE(4)
    CUBICS_CASE(8)
    default: return cudaErrorInvalidValue;
    }
#undef CUBICS_CASE
}

cudaError_t occupancy_search(int W, bool staged, int kind, int threads, size_t smem, int *bps) {
    if (kind == KERN_REG)
        return W == 1 ? occupancy_reg(staged, threads, smem, bps) : cudaErrorInvalidValue;
    const bool ext = kind == KERN_EXT;
#define CUBICS_CASE(WW)                                                                      \
    case WW:                                                                                 \
        return ext ? occupancy_ext_w##WW(staged, threads, smem, bps)                         \
                   : occupancy_w##WW(staged, threads, smem, bps);
    switch (W) {
    CUBICS_CASE(1)
    CUBICS_CASE(2)
    CUBICS_CASE(4)
    CUBICS_CASE(8)
    default: return cudaErrorInvalidValue;
    }
#undef CUBICS_CASE
}

// block_per_node: one block per state, every warp of it on that state's constraints
cudaError_t launch_propagate(int W, bool staged, const PropArgs &P, int blocks, int threads,
                             size_t smem, cudaStream_t st, bool block_per_node) {
    switch (W) {
    case 1: return launch_prop_w1(staged, P, blocks, threads, smem, st, block_per_node);
    case 2: return launch_prop_w2(staged, P, blocks, threads, smem, st, block_per_node);
    case 4: return launch_prop_w4(staged, P, blocks, threads, smem, st, block_per_node);
    case 8: return launch_prop_w8(staged, P, blocks, threads, smem, st, block_per_node);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_expand(int W, const ExpandArgs &E, int blocks, cudaStream_t st) {
    switch (W) {
    case 1: return launch_expand_w1(E, blocks, st);
    case 2: return launch_expand_w2(E, blocks, st);
    case 4: return launch_expand_w4(E, blocks, st);
    case 8: return launch_expand_w8(E, blocks, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------------------ set-up kernels

// single-problem mode: team 0 holds the root record in slot 0 of its queue
__global__ void init_single_kernel(SearchArgs A) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int qcap = A.qmask + 1;
    for (int i = tid; i < qcap; i += gridDim.x * blockDim.x) A.qseq[i] = i == 0 ? 1u : (uint32_t)i;
    if (blockIdx.x == 0) {
        const uint32_t *ib = A.arena + A.inst_off[0];
        const int S = (int)ib[H_S], W = (int)ib[H_W];
        const int R = record_words(S, W);
        const uint32_t *root = ib + ib[H_OFF_ROOT];
        for (int k = threadIdx.x; k < R; k += blockDim.x)
            A.qrec[k] = k < S ? root[k] : (k == S + W ? 0xffffffffu : 0u);
        if (threadIdx.x == 0) {
            A.teams[0].work = 1;
            A.teams[0].tail = 1;
            A.teams[0].promised = 1;
        }
    }
}

// batch mode: every team's queue starts empty
__global__ void init_batch_kernel(SearchArgs A, int teams) {
    const int qcap = A.qmask + 1;
    const long long total = (long long)teams * qcap;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        A.qseq[i] = (uint32_t)(i % qcap);
}

cudaError_t launch_init_single(const SearchArgs &A, cudaStream_t st) {
    init_single_kernel<<<8, 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_init_batch(const SearchArgs &A, int teams, cudaStream_t st) {
    init_batch_kernel<<<64, 256, 0, st>>>(A, teams);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ shared-memory probe

constexpr int PROBE_WORDS4 = 4096;   // 64 KB of uint4 per block

__global__ void __launch_bounds__(1024) smem_probe_kernel(uint4 *out, int iters) {
    extern __shared__ uint4 buf[];
    for (int i = threadIdx.x; i < PROBE_WORDS4; i += blockDim.x)
        buf[i] = make_uint4(i, 3 * i, 5 * i, 7 * i);
    __syncthreads();
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
    uint32_t a = 0, b = 0, c = 0, d = 0;
    int idx = threadIdx.x;
#pragma unroll 8
    for (int it = 0; it < iters; ++it) {
        uint32_t x, y, z, w;
        // volatile: every iteration issues its load (the addresses repeat every 4 iterations)
        asm volatile("ld.volatile.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                     : "r"(base + 16u * (uint32_t)idx));
        a ^= x; b ^= y; c ^= z; d ^= w;
        idx = (idx + 1024) & (PROBE_WORDS4 - 1);
    }
    if ((a & b & c & d) == 0xffffffffu) out[0] = make_uint4(a, b, c, d);   // keeps the loads live
}

cudaError_t probe_smem(void *out, cudaStream_t st, int sms, int reps, double *gbs) {
    const int threads = 1024, blocks = 2 * sms, iters = 4096;
    const size_t smem = PROBE_WORDS4 * sizeof(uint4);
    cudaError_t e = cudaFuncSetAttribute(smem_probe_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaEvent_t e0, e1;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return e;
    float best = 1e30f;
    for (int r = 0; r < reps + 1 && e == cudaSuccess; ++r) {
        cudaEventRecord(e0, st);
        smem_probe_kernel<<<blocks, threads, smem, st>>>((uint4 *)out, iters);
        e = cudaGetLastError();
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && ms > 0.f && ms < best) best = ms;       // launch 0 is a warm-up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess)
        *gbs = (double)blocks * threads * (double)iters * 16.0 / (best * 1e-3) / 1e9;
    return e;
}

}  // namespace cubics
