// Shared device/host helpers of libdwfmg: complex arithmetic, link loads,
// status reporting and geometry checks.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>
#include <stdarg.h>

#include "../../include/dwf.h"

namespace dwf {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define DWF_CHECK_CUDA(call)                                                     \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) {                                                 \
            ::dwf::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,          \
                             cudaGetErrorString(e_));                            \
            return DWF_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

#define DWF_CHECK_LAUNCH()                                                       \
    do {                                                                         \
        cudaError_t e_ = cudaGetLastError();                                     \
        if (e_ != cudaSuccess) {                                                 \
            ::dwf::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,      \
                             cudaGetErrorString(e_));                            \
            return DWF_ERR_CUDA;                                                 \
        }                                                                        \
    } while (0)

#define DWF_TRY(expr)                                                            \
    do {                                                                         \
        dwf_status s_ = (expr);                                                  \
        if (s_ != DWF_OK) return s_;                                             \
    } while (0)

// ---------------------------------------------------------------------------
// geometry
// ---------------------------------------------------------------------------
struct Geom {
    int nd;
    int L[4];
    int Ls;
    int group;
    int anti[4];
    long long V;       // d-dim sites
    int nspin, ncol;   // per-site spinor shape
};

dwf_status check_geom(const dwf_geom* g, Geom* out);
bool valid_prec(int prec);

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }
// spinor buffers are read as float4 / double2: 16-byte alignment is part of the ABI
inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// ---------------------------------------------------------------------------
// complex arithmetic on float2 / double2
// ---------------------------------------------------------------------------
template <class R> struct cplx;
template <> struct cplx<float> { using T = float2; };
template <> struct cplx<double> { using T = double2; };

template <class C> __host__ __device__ __forceinline__ C mk(decltype(C().x) a, decltype(C().x) b) {
    C c; c.x = a; c.y = b; return c;
}
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <class C, class R> __host__ __device__ __forceinline__ C scale(C a, R s) { C c; c.x = a.x * s; c.y = a.y * s; return c; }
// a * b
template <class C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
// conj(a) * b
template <class C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C c; c.x = a.x * b.x + a.y * b.y; c.y = a.x * b.y - a.y * b.x; return c;
}
// i * a
template <class C> __host__ __device__ __forceinline__ C times_i(C a) { C c; c.x = -a.y; c.y = a.x; return c; }

// ---------------------------------------------------------------------------
// link storage: complex value in the storage type of a precision
// ---------------------------------------------------------------------------
struct LinkF64 { using store = double2; using real = double; };
struct LinkF32 { using store = float2; using real = float; };
struct LinkH16 { using store = __half2; using real = float; };
struct LinkBF16 { using store = __nv_bfloat162; using real = float; };

__device__ __forceinline__ double2 load_link(const double2* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float2 load_link(const float2* p, long long i) { return __ldg(p + i); }
__device__ __forceinline__ float2 load_link(const __half2* p, long long i) {
    __half2 h = __ldg(p + i);
    return __half22float2(h);
}
__device__ __forceinline__ float2 load_link(const __nv_bfloat162* p, long long i) {
    __nv_bfloat162 h = __ldg(p + i);
    return __bfloat1622float2(h);
}

}  // namespace dwf
