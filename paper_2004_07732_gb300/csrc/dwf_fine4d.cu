// 4-d SU(3) Shamir operator (the 4-d extension of Eq. DWoperator).
#include "common.cuh"
#include "fine_kernels.cuh"

namespace dwf {

dwf_status fine_apply_4d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st) {
    (void)g; (void)U; (void)psi; (void)out; (void)M5; (void)mf; (void)dagger; (void)prec; (void)s_chunk; (void)st;
    set_error("4-d SU(3) operator not built yet");
    return DWF_ERR_UNSUPPORTED;
}

}  // namespace dwf
