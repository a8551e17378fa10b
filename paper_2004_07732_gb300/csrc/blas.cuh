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
constexpr int RED_BLOCKS = 152 * 4;   // upper bound on reduction grid size
constexpr int RED_MAX = 4;            // reduced quantities per kernel

inline int red_grid(long long n) {
    long long b = (n + RED_THREADS - 1) / RED_THREADS;
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

// Grid-wide reduction with a finaliser fin(double* totals) run by one thread.
template <int N, class Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[N], RedScratch rs, Fin fin) {
    __shared__ bool last;
    block_sum<N>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) rs.partials[k * RED_BLOCKS + blockIdx.x] = v[k];
        __threadfence();
        unsigned t = atomicAdd(rs.counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        w[k] = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) w[k] += __ldcg(rs.partials + k * RED_BLOCKS + b);
    }
    block_sum<N>(w);
    if (threadIdx.x == 0) {
        fin(w);
        *rs.counter = 0u;
    }
}

// <x, y> over n complex values into out[0..1] (device), FP64 accumulation.
dwf_status dot_device(const void* x, const void* y, long long n, bool f64, RedScratch rs, double* out,
                      cudaStream_t st);

}  // namespace dwf
