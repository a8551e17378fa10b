// Reductions and the stream-ordered workspace of libdwfmg.
#include "blas.cuh"

namespace dwf {

dwf_status Workspace::reserve(cudaStream_t s) {
    st = s;
    const size_t cbytes = sizeof(unsigned) * (RED_GROUPS + 1) * RED_CSTRIDE;
    size_t bytes = sizeof(double) * ((size_t)RED_MAX * RED_BLOCKS + 64) + cbytes;
    cudaError_t e = cudaMallocAsync(&base, bytes, s);
    if (e != cudaSuccess) {
        set_error("workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        base = nullptr;
        return DWF_ERR_OOM;
    }
    partials = reinterpret_cast<double*>(base);
    scal = partials + (size_t)RED_MAX * RED_BLOCKS;
    counter = reinterpret_cast<unsigned*>(scal + 64);
    DWF_CHECK_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 64 + cbytes, s));
    return DWF_OK;
}

Workspace::~Workspace() {
    if (base) cudaFreeAsync(base, st);
}

template <class C>
__global__ void __launch_bounds__(RED_THREADS) k_dot(const C* __restrict__ x, const C* __restrict__ y, long long n,
                                                     RedScratch rs, double* out) {
    double v[2] = {0.0, 0.0};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        C a = x[i], b = y[i];
        double ax = a.x, ay = a.y, bx = b.x, by = b.y;
        v[0] += ax * bx + ay * by;
        v[1] += ax * by - ay * bx;
    }
    grid_reduce<2>(v, rs, [=] __device__(double* t) { out[0] = t[0]; out[1] = t[1]; });
}

// FP32 vectors: per-thread FP32 partials over a few elements, FP64 across threads
__global__ void __launch_bounds__(RED_THREADS) k_dot32(const float2* __restrict__ x, const float2* __restrict__ y,
                                                       long long n, RedScratch rs, double* out) {
    float re = 0.f, im = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 a = x[i], b = y[i];
        re += a.x * b.x + a.y * b.y;
        im += a.x * b.y - a.y * b.x;
    }
    double v[2] = {re, im};
    grid_reduce<2>(v, rs, [=] __device__(double* t) { out[0] = t[0]; out[1] = t[1]; });
}

dwf_status dot_device(const void* x, const void* y, long long n, bool f64, RedScratch rs, double* out,
                      cudaStream_t st, bool exact) {
    if (f64) k_dot<double2><<<red_grid(n), RED_THREADS, 0, st>>>((const double2*)x, (const double2*)y, n, rs, out);
    else if (exact) k_dot<float2><<<red_grid(n), RED_THREADS, 0, st>>>((const float2*)x, (const float2*)y, n, rs, out);
    else     k_dot32<<<red_grid4(n), RED_THREADS, 0, st>>>((const float2*)x, (const float2*)y, n, rs, out);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf
