// Reductions and the stream-ordered workspace of libdwfmg.
#include "blas.cuh"

namespace dwf {

dwf_status Workspace::reserve(cudaStream_t s) {
    st = s;
    size_t bytes = sizeof(double) * ((size_t)RED_MAX * RED_BLOCKS + 64) + 256;
    cudaError_t e = cudaMallocAsync(&base, bytes, s);
    if (e != cudaSuccess) {
        set_error("workspace allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        base = nullptr;
        return DWF_ERR_OOM;
    }
    partials = reinterpret_cast<double*>(base);
    scal = partials + (size_t)RED_MAX * RED_BLOCKS;
    counter = reinterpret_cast<unsigned*>(scal + 64);
    DWF_CHECK_CUDA(cudaMemsetAsync(scal, 0, sizeof(double) * 64 + 256, s));
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

dwf_status dot_device(const void* x, const void* y, long long n, bool f64, RedScratch rs, double* out,
                      cudaStream_t st) {
    int g = red_grid(n);
    if (f64) k_dot<double2><<<g, RED_THREADS, 0, st>>>((const double2*)x, (const double2*)y, n, rs, out);
    else     k_dot<float2><<<g, RED_THREADS, 0, st>>>((const float2*)x, (const float2*)y, n, rs, out);
    DWF_CHECK_LAUNCH();
    return DWF_OK;
}

}  // namespace dwf
