// Internal structures of the two-level domain-wall multigrid (Sec. 2.3).
#pragma once

#include <map>
#include <vector>

#include "common.cuh"
#include "fine_kernels.cuh"
#include "blas.cuh"

namespace dwf {

constexpr int MG_MAX_NVEC = 32;
constexpr int MG_MAX_DIRS = 9;   // self + 2 * 4

// Geometry of the coarse level and of the aggregation map.
struct MgGeom {
    int nd;
    int L[4];        // fine lattice
    int b[4];        // aggregate extent
    int Lc[4];       // coarse lattice
    long long V, Vc;
    int nb;          // fine sites per aggregate
    int nchd;        // fine dof per chirality per site (1 for 2-d U(1), 6 for 4-d SU(3))
    int nvec;
    int ncd;         // coarse dof per site = 2 * nvec
    int ndir;        // 2 * nd + 1
    int Ls, Ls_c;
};

// Device-owned buffers are released by a single cudaFree of `arena`.
struct dwf_mg_impl;

}  // namespace dwf

struct dwf_mg {
    dwf::Geom G;          // fine geometry
    dwf::MgGeom mg;
    double M5, mf;
    dwf_mg_params prm;
    cudaStream_t st;
    // device buffers (owned)
    void* U64;            // complex128 links
    void* Ulo;            // fine links in prm.fine_prec storage
    double2* nullv;       // relaxed near-null vectors [vec][site][spin][color]
    double2* P64;         // prolongator [site][chir][l][k]
    float2* P32;
    double2* Y64;         // Galerkin blocks [xc][dir][row][col]
    float2* Y32;          // FP32 copy, column-major per block: [xc][dir][col][row]
    float2* Yd32;         // FP32 adjoint blocks Y[x+dir][-dir]^dag, column-major (generic stencil)
    void* Ytile;          // blocks read by the 2-d tile stencil: Y32, or an FP16 column-major copy
    int ytile_half;       // 1 when Ytile holds FP16 (half2) blocks
    void* Ymma;           // FP16 blocks in tensor-core fragment order (48 dof, FP16 blocks), else nullptr
    int* status;          // device status word of the setup kernels
    std::vector<void*> allocs;
    // solver workspace (allocated on first solve)
    bool ws_ready;
    dwf::Workspace ws;
    double* hsc;          // pinned host mirror of solver scalars
    std::vector<void*> fine_vecs;   // FP32 fine vectors
    std::vector<void*> coarse_vecs; // FP32 coarse vectors
    void* x64;            // FP64 solution accumulator
    void* r64;            // FP64 residual
    void* solver_meta;    // device pointer arrays and CGS scratch of the solver
    bool solver_meta_ready;
    cudaGraphExec_t coarse_graph_first;   // captured coarse GCR: prologue + one restart cycle
    cudaGraphExec_t coarse_graph_cycle;   // captured coarse GCR: one restart cycle
    cudaStream_t cap_stream;              // private stream used only to record graphs
    void* batched;                        // workspace and graphs of the batched solver (mg_batched.cu)
    mutable std::map<int, int> tc_choice; // autotuned form of the many-right-hand-side coarse contraction, by nrhs
};

namespace dwf {

dwf_status mg_alloc(dwf_mg* h, void** p, size_t bytes);

// Coarse operator application (Eq. coarsenDW) on FP32 coarse vectors;
// `skip` (device, may be null): the launch does nothing when *skip != 0.
dwf_status coarse_dwf_apply(const dwf_mg* h, const float2* in, float2* out, double mf, bool dagger,
                            const int* skip, cudaStream_t st);
dwf_status build_adjoint_blocks(dwf_mg* h, cudaStream_t st);
// tensor-core coarse stencil on nrhs right-hand sides ([rhs][s][site][dof]);
// skip_rhs: per right-hand-side device flags (may be null)
dwf_status coarse_apply_multi_tc(const dwf_mg* h, int nrhs, const float2* in, float2* out, double mf, bool dagger,
                                 const int* skip_rhs, cudaStream_t st);
// Autotuner of that contraction: times every eligible form (mma.sync with 1, 2 or 4
// column tiles of 8 per warp; tcgen05 with FP16 blocks from 128 columns) on in -> out
// (scratch: contents are overwritten) and keeps the fastest for nrhs.  Synchronises
// `st`; must not run during stream capture.  No-op once nrhs is tuned.
dwf_status coarse_tc_tune(const dwf_mg* h, int nrhs, const float2* in, float2* out, cudaStream_t st);
// one-time kernel attributes of the coarse stencil (outside any stream capture)
dwf_status coarse_init_attributes();
// Wall transfers (Eq. TruncProjectInterpolate) on nrhs vectors stored back to
// back; skip: per right-hand-side device flags (may be null).
dwf_status restrict_wall(const dwf_mg* h, const float2* r_fine, float2* r_coarse, const int* skip, cudaStream_t st,
                         int nrhs = 1);
dwf_status prolong_wall(const dwf_mg* h, const float2* e_coarse, float2* e_fine, const int* skip, cudaStream_t st,
                        int nrhs = 1);

// One cooperative launch running the whole coarsest CGNR; vec6 = six coarse
// work vectors, partials = 3 * grid doubles, bar = 16 bytes of barrier state.
// out_iters accumulates the iteration count over calls.
dwf_status coarse_cgnr_persistent(const dwf_mg* h, const float2* rc, float2* ec, float2* const* vec6, double* partials,
                                  void* bar, int* out_iters, double* out_rr2, cudaStream_t st);

// the batched K-cycle on nrhs right-hand sides stored back to back (mg_batched.cu)
dwf_status mg_solve_batched_impl(dwf_mg* h, int nrhs, const double2* B, double2* X, double tol, int maxiter,
                                 dwf_solve_stats* stats);
// releases the batched solver's workspace of a handle
void batched_state_free(dwf_mg* h);

// One cooperative launch running a whole coarse GCR solve (restart
// coarse_restart): S = coarse_restart + 1 residual slots, W = coarse_restart
// vectors, t = one vector, partials = (2 + 2 * 16 + 3) * grid doubles, bar = 16
// bytes of barrier state.  out_iters accumulates the steps over calls.
bool coarse_gcr_persistent_ok(const dwf_mg* h);
dwf_status coarse_gcr_persistent(const dwf_mg* h, const float2* rc, float2* ec, float2* const* S, float2* const* W,
                                 float2* t, double* partials, void* bar, int* out_iters, double* out_rr2,
                                 cudaStream_t st);

inline long long fine_len(const dwf_mg* h) { return h->G.V * h->G.Ls * site_dof(h->G); }
inline long long coarse_len(const dwf_mg* h) { return h->mg.Vc * h->mg.Ls_c * h->mg.ncd; }

}  // namespace dwf
