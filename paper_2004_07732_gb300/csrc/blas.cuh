// BLAS-1 building blocks with FP64 reductions: warp shuffle -> block -> grid.
//
// A reduction kernel writes one partial per block; the last block to finish
// (detected with a completion counter after a memory fence) sums the partials
// in a fixed order and runs a finaliser on the totals.  The grid size and the
// per-thread element assignment depend only on n, so results are bitwise
// reproducible run to run.
#pragma once

#include "common.cuh"

namespace dwf {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 152 * 8;   // upper bound on reduction grid size
constexpr int RED_MAX = 4;            // reduced quantities per kernel

inline int red_grid(long long n) {
    long long b = (n + RED_THREADS - 1) / RED_THREADS;
    if (b < 1) b = 1;
    return (int)(b < RED_BLOCKS ? b : RED_BLOCKS);
}

// Grid for reductions over FP32 vectors read as float4: about 8 complex values
// per thread (fewer, fuller blocks keep the block-sum and completion tail short).
inline int red_grid4(long long n) {
    long long b = (n + 8LL * RED_THREADS - 1) / (8LL * RED_THREADS);
    if (b < 1) b = 1;
    return (int)(b < RED_BLOCKS ? b : RED_BLOCKS);
}

// Device scratch of one reduction stream: RED_MAX*RED_BLOCKS partials, a
// counter, and 64 doubles of solver scalars.
struct RedScratch {
    double* partials;
    unsigned* counter;
};

// Library-owned scratch for a call or a solver handle (stream-ordered allocation).
struct Workspace {
    void* base = nullptr;
    double* partials = nullptr;
    unsigned* counter = nullptr;
    double* scal = nullptr;    // 64 doubles
    cudaStream_t st = nullptr;
    dwf_status reserve(cudaStream_t s);
    RedScratch red() const { return RedScratch{partials, counter}; }
    ~Workspace();
};

template <int N>
__device__ __forceinline__ void warp_sum(double (&v)[N]) {
#pragma unroll
    for (int k = 0; k < N; ++k)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], off);
}

// Block-wide sum; thread 0 ends with the totals.  blockDim.x == RED_THREADS.
template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N]) {
    __shared__ double sh[N][RED_THREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    warp_sum<N>(v);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = lane < RED_THREADS / 32 ? sh[k][lane] : 0.0;
        warp_sum<N>(v);
    }
}

// Block-wide sum of FP32 per-thread partials: the tree over each warp in FP32
// (five shuffle-adds in a fixed order), the per-warp sums in FP64 (thread q < N
// adds quantity q over the warps in order); every thread ends with the totals.
// GB300 runs FP64 at a small fraction of its FP32 rate, and a tree of FP64
// shuffle-adds per thread and quantity made the many-quantity solver
// reductions FP64-bound.
template <int N>
__device__ __forceinline__ void block_sum_f(const float (&vin)[N], double (&v)[N]) {
    __shared__ double sh[N][RED_THREADS / 32];
    __shared__ double tot[N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float f[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        f[k] = vin[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) f[k] += __shfl_down_sync(0xffffffffu, f[k], off);
    }
    __syncthreads();                                  // the shared arrays may be in use from a previous call
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[k][warp] = (double)f[k];
    __syncthreads();
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        double s = 0.0;
        for (int u = 0; u < RED_THREADS / 32; ++u) s += sh[k][u];
        tot[k] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = tot[k];
}

// Completion counters: RED_GROUPS group counters and one top counter, each
// on its own 128-byte line, so that the blocks of a grid do not all contend
// for one address (a single counter serialised ~1000 atomics per reduction).
constexpr int RED_GROUPS = 32;
constexpr int RED_CSTRIDE = 32;   // unsigneds between counters (128 bytes)

// True in exactly one block: the last to finish.  Group g = blockIdx % 32
// counts its blocks; the last block of each group bumps the top counter.
__device__ __forceinline__ bool grid_last_block(unsigned* counters) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g = blockIdx.x % RED_GROUPS;
        const unsigned gsize = (gridDim.x - g + RED_GROUPS - 1) / RED_GROUPS;
        const unsigned ngroups = gridDim.x < RED_GROUPS ? gridDim.x : RED_GROUPS;
        bool l = false;
        if (atomicAdd(counters + g * RED_CSTRIDE, 1u) == gsize - 1) {
            counters[g * RED_CSTRIDE] = 0u;
            __threadfence();
            l = atomicAdd(counters + RED_GROUPS * RED_CSTRIDE, 1u) == ngroups - 1;
            if (l) counters[RED_GROUPS * RED_CSTRIDE] = 0u;
        }
        last = l;
    }
    __syncthreads();
    return last;
}

// Sum over the blocks of a grid, in the grid's last block: quantity k of block
// b at part[k * stride + b].  Warp w sums quantities w, w + 8, ...: lane l adds
// blocks l, l + 32, ... in FP64, then a fixed FP64 shuffle tree.  Every thread
// of the block ends with the totals.
template <int N>
__device__ __forceinline__ void grid_final_sum(const double* part, size_t stride, double (&v)[N]) {
    __shared__ double tot[N];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = warp; k < N; k += RED_THREADS / 32) {
        double s = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) s += __ldcg(part + (size_t)k * stride + b);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) tot[k] = s;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = tot[k];
}

// grid_reduce for FP32 per-thread partials: block_sum_f, then grid_final_sum.
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce_f(const float (&vf)[N], RedScratch rs, Fin fin) {
    double v[N];
    block_sum_f<N>(vf, v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) rs.partials[k * RED_BLOCKS + blockIdx.x] = v[k];
    }
    if (!grid_last_block(rs.counter)) return;
    __threadfence();
    double w[N];
    grid_final_sum<N>(rs.partials, RED_BLOCKS, w);
    if (threadIdx.x == 0) fin(w);
}

// Grid-wide reduction with a finaliser fin(double* totals) run by one thread.
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[N], RedScratch rs, Fin fin) {
    block_sum<N>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) rs.partials[k * RED_BLOCKS + blockIdx.x] = v[k];
    }
    if (!grid_last_block(rs.counter)) return;
    __threadfence();
    double w[N];
    grid_final_sum<N>(rs.partials, RED_BLOCKS, w);
    if (threadIdx.x == 0) fin(w);
}

// Either reduction by the type of the per-thread partials: FP32 partials take
// grid_reduce_f, FP64 partials (FP64 data) keep every sum in FP64.
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce_any(const float (&v)[N], RedScratch rs, Fin fin) {
    grid_reduce_f<N>(v, rs, fin);
}
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce_any(const double (&v)[N], RedScratch rs, Fin fin) {
    double w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = v[k];
    grid_reduce<N>(w, rs, fin);
}

// <x, y> over n complex values into out[0..1] (device).  FP64 data, or exact =
// true: every product accumulated in FP64.  FP32 data with exact = false:
// per-thread FP32 partials over a few elements, FP64 across threads (GB300's
// FP64 units make per-element FP64 accumulation the bottleneck otherwise).
dwf_status dot_device(const void* x, const void* y, long long n, bool f64, RedScratch rs, double* out,
                      cudaStream_t st, bool exact = false);

}  // namespace dwf
