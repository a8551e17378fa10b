// Diagnostic: exercise the bounded-wait error path of the library's device
// waits without faulting or hanging the GPU.  Each kernel waits for an event
// that nothing will deliver, gives up after the requested time (measured with
// %globaltimer), records the timeout in a status word and returns; the host
// reports DWF_ERR_TIMEOUT.  The context stays usable afterwards.
#include "common.cuh"

namespace dwf {
namespace {

__device__ __forceinline__ unsigned long long ns_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// An mbarrier expecting two arrivals receives one: the phase never completes.
__global__ void k_wait_mbarrier(unsigned long long budget_ns, int* status) {
    __shared__ unsigned long long bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 2;" ::"r"(a) : "memory");
    __syncthreads();
    if (threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
    __syncthreads();
    const unsigned long long t0 = ns_now();
    uint32_t ok = 0;
    while (!ok) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(a) : "memory");
        if (ns_now() - t0 > budget_ns) break;
    }
    if (!ok && threadIdx.x == 0) atomicExch(status, (int)DWF_ERR_TIMEOUT);
}

// A software grid barrier that expects one block more than the grid has.
__global__ void k_wait_grid(unsigned* counter, unsigned long long budget_ns, int* status) {
    __shared__ int timed_out;
    if (threadIdx.x == 0) {
        timed_out = 0;
        atomicAdd(counter, 1u);
        const unsigned expected = gridDim.x + 1;
        const unsigned long long t0 = ns_now();
        volatile unsigned* c = counter;
        while (*c < expected) {
            if (ns_now() - t0 > budget_ns) { timed_out = 1; break; }
            __nanosleep(256);
        }
    }
    __syncthreads();
    if (timed_out && threadIdx.x == 0) atomicExch(status, (int)DWF_ERR_TIMEOUT);
}

}  // namespace
}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_check_wait_timeout(int which, double seconds, void* stream) {
    clear_error();
    if (which != 0 && which != 1) { set_error("which must be 0 (mbarrier) or 1 (grid barrier)"); return DWF_ERR_ARG; }
    if (!(seconds > 0.0) || seconds > 10.0) { set_error("seconds must be in (0, 10]"); return DWF_ERR_ARG; }
    cudaStream_t st = as_stream(stream);
    const unsigned long long budget = (unsigned long long)(seconds * 1e9);
    void* buf = nullptr;
    DWF_CHECK_CUDA(cudaMallocAsync(&buf, 256, st));
    DWF_CHECK_CUDA(cudaMemsetAsync(buf, 0, 256, st));
    int* status = (int*)buf;
    unsigned* counter = (unsigned*)buf + 16;
    if (which == 0) {
        k_wait_mbarrier<<<1, 32, 0, st>>>(budget, status);
    } else {
        int nsm = 1, dev = 0;
        DWF_CHECK_CUDA(cudaGetDevice(&dev));
        DWF_CHECK_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        void* args[] = {&counter, (void*)&budget, &status};
        DWF_CHECK_CUDA(cudaLaunchCooperativeKernel((const void*)k_wait_grid, dim3(nsm), dim3(32), args, 0, st));
    }
    DWF_CHECK_LAUNCH();
    int h = 0;
    DWF_CHECK_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWF_CHECK_CUDA(cudaStreamSynchronize(st));
    cudaFreeAsync(buf, st);
    if (h == DWF_ERR_TIMEOUT) {
        set_error("bounded device wait gave up after %.3f s (as intended by this check)", seconds);
        return DWF_ERR_TIMEOUT;
    }
    return DWF_OK;
}
