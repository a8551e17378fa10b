// Internal interfaces between the translation units of libdwfmg.
#pragma once

#include "common.cuh"

namespace dwf {

struct Fine2dParams {
    long long V;
    int L0, L1, Ls;
    int anti0, anti1;
    double diag;   // d - M5 + 1
    double mf;
    int s_chunk;
    int s_base, s_end;   // slices [s_base, s_end) written by k_dwf2d (0, Ls for the whole operator)
};

struct Fine4dParams {
    long long V;
    int L[4];
    int Ls;
    int anti[4];
    double diag;
    double mf;
    float diag_f, mf_f;   // the same in FP32 for the FP32 kernels
    int s_chunk;
};

int choose_s_chunk(long long V, int Ls);

// One right-hand side of a batched 2-d apply: its lattice, links and vectors,
// and the first virtual block of its range (blocks of 256 sites).
constexpr int BATCH_MAX = 256;
struct BatchDesc2d {
    Fine2dParams p;
    const void* U;
    const void* psi;
    void* out;
    long long block0;
};
// Descriptors of one batched launch, passed by value as a __grid_constant__
// kernel parameter (no device allocation or host copy per call).
constexpr int BATCH_LAUNCH_MAX = 128;
struct BatchArgs2d {
    int nrhs;
    long long total_blocks;
    BatchDesc2d d[BATCH_LAUNCH_MAX];
};
dwf_status fine_apply_2d_batched(const BatchArgs2d& args, bool dagger, int prec, cudaStream_t st);

// out = D_DW(mf) psi or its adjoint, on the canonical layout; `prec` selects
// spinor / link storage.  s_chunk <= 0 picks the default.
dwf_status fine_apply_2d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st);
// nrhs right-hand sides of one 2-d lattice stored back to back; skip: per
// right-hand-side device flags (may be null), nonzero leaves that output untouched.
dwf_status fine_apply_2d_multi(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int nrhs, const int* skip, cudaStream_t st);
// out slices [s_lo, s_hi) of D_DW(mf) psi (psi must hold slices s_lo - 1 .. s_hi and, for the
// walls, 0 and Ls - 1); 2-d only
dwf_status fine_apply_2d_range(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                               bool dagger, int prec, int s_lo, int s_hi, cudaStream_t st);
// skip: optional device flag; nonzero leaves out untouched (one right-hand side)
dwf_status fine_apply_4d(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                         bool dagger, int prec, int s_chunk, cudaStream_t st, const int* skip = nullptr);

// the 4-d operator on the slice-paired packed layout (FP32 spinors, even Ls; dwf_fine4d_pair.cu)
// (skip: optional device flag; nonzero leaves out untouched)
dwf_status fine_apply_4d_paired(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                                bool dagger, int prec, cudaStream_t st, const int* skip = nullptr);
dwf_status pack_spinor_paired(const Geom& g, const void* psi, void* packed, cudaStream_t st);
dwf_status unpack_spinor_paired(const Geom& g, const void* packed, void* psi, cudaStream_t st);

// nrhs right-hand sides stored back to back with per-right-hand-side skip flags:
// any nrhs on 2-d lattices, one right-hand side on 4-d lattices
inline dwf_status fine_apply_rhs(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                                 bool dagger, int prec, int nrhs, const int* skip, cudaStream_t st) {
    if (g.nd == 2) return fine_apply_2d_multi(g, U, psi, out, M5, mf, dagger, prec, nrhs, skip, st);
    if (nrhs != 1) { set_error("4-d lattices take one right-hand side per call"); return DWF_ERR_UNSUPPORTED; }
    return fine_apply_4d(g, U, psi, out, M5, mf, dagger, prec, 0, st, skip);
}

inline dwf_status fine_apply(const Geom& g, const void* U, const void* psi, void* out, double M5, double mf,
                             bool dagger, int prec, cudaStream_t st, int s_chunk = 0) {
    if (g.nd == 2) return fine_apply_2d(g, U, psi, out, M5, mf, dagger, prec, s_chunk, st);
    return fine_apply_4d(g, U, psi, out, M5, mf, dagger, prec, s_chunk, st);
}

// number of complex values per 5-d / d-dim site
inline long long site_dof(const Geom& g) { return (long long)g.nspin * g.ncol; }
inline long long spinor_len(const Geom& g) { return g.V * g.Ls * site_dof(g); }
inline long long link_len(const Geom& g) { return g.V * g.nd * (long long)(g.ncol * g.ncol); }

}  // namespace dwf
