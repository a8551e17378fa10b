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

// Parameters of one coarse stencil launch (Eq. coarsenDW on a coarse lattice).
struct CoarseParams {
    long long Vc;
    int nd;
    int Lc[4];
    int Ls_c;
    int ncd, nvec, ndir;
    float mf;
};

// Aggregation of a lattice L into blocks b (coarse lattice Lc).
struct AggIndex {
    int nd, L[4], b[4], Lc[4];
    // fine site of local index l in aggregate xc
    __host__ __device__ long long fine_site(long long xc, int l) const {
        long long site = 0, stride = 1;
        long long rem = xc;
        int lr = l;
        for (int mu = 0; mu < nd; ++mu) {
            int c = (int)(rem % Lc[mu]);
            rem /= Lc[mu];
            int lc = lr % b[mu];
            lr /= b[mu];
            site += (long long)(c * b[mu] + lc) * stride;
            stride *= L[mu];
        }
        return site;
    }
};

// State of one near-null relaxation (CG on the homogeneous normal system).
struct NvState {
    double rr, rr0, alpha, beta;
    int done, iters;
};

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
    void* Upk;            // the same links in the slice-paired layout (when pk), else nullptr
    int pk;               // 1: the K-cycle keeps its FP32 fine vectors in the slice-paired layout
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
    void* lvl3;                           // third level and coarsest deflation (mg_level3.cu), or nullptr
    mutable std::map<int, int> tc_choice; // autotuned form of the many-right-hand-side coarse contraction, by
                                          // nrhs (slice-major vectors) or -nrhs (site-major vectors)
};

namespace dwf {

dwf_status mg_alloc(dwf_mg* h, void** p, size_t bytes);

// Coarse operator application (Eq. coarsenDW) on FP32 coarse vectors;
// `skip` (device, may be null): the launch does nothing when *skip != 0.
dwf_status coarse_dwf_apply(const dwf_mg* h, const float2* in, float2* out, double mf, bool dagger,
                            const int* skip, cudaStream_t st);
dwf_status build_adjoint_blocks(dwf_mg* h, cudaStream_t st);
// tensor-core coarse stencil on nrhs right-hand sides, vectors in `layout`
// (DWF_COARSE_SLICE_MAJOR: [rhs][s][site][dof]; DWF_COARSE_SITE_MAJOR:
// [site][rhs][s][dof]); skip_rhs: per right-hand-side device flags (may be null)
dwf_status coarse_apply_multi_tc(const dwf_mg* h, int nrhs, const float2* in, float2* out, double mf, bool dagger,
                                 const int* skip_rhs, cudaStream_t st, int layout = DWF_COARSE_SLICE_MAJOR);
// Autotuner of that contraction: times every eligible form (mma.sync with 1, 2 or 4
// column tiles of 8 per warp; tcgen05 with FP16 blocks from 128 columns) on in -> out
// (scratch: contents are overwritten) and keeps the fastest for nrhs.  Synchronises
// `st`; must not run during stream capture.  No-op once (nrhs, layout) is tuned.
dwf_status coarse_tc_tune(const dwf_mg* h, int nrhs, const float2* in, float2* out, cudaStream_t st,
                          int layout = DWF_COARSE_SLICE_MAJOR);
// one-time kernel attributes of the coarse stencil (outside any stream capture)
dwf_status coarse_init_attributes();
// Wall transfers (Eq. TruncProjectInterpolate) on nrhs vectors stored back to
// back; skip: per right-hand-side device flags (may be null).  packed: the fine
// vectors are in the slice-paired 4-d layout (dwf_pack_spinor, V a multiple of 32).
dwf_status restrict_wall(const dwf_mg* h, const float2* r_fine, float2* r_coarse, const int* skip, cudaStream_t st,
                         int nrhs = 1, bool packed = false);
dwf_status prolong_wall(const dwf_mg* h, const float2* e_coarse, float2* e_fine, const int* skip, cudaStream_t st,
                        int nrhs = 1, bool packed = false);

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

// per-site kernel of the coarse stencil on FP32 column-major blocks (any
// coarse lattice with 24 <= ncd, ncd * Ls_c <= 512); the adjoint uses sigma_3
dwf_status coarse_site_apply(const CoarseParams& p, const __half2* B, const float2* in, float2* out, bool dagger,
                             const int* skip, int* status, cudaStream_t st);
dwf_status coarse_site_apply(const CoarseParams& p, const float2* B, const float2* in, float2* out, bool dagger,
                             const int* skip, int* status, cudaStream_t st);

// grid of an element-wise kernel over n values (at most 8 blocks of 256 per SM)
inline int level_ew_grid(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 152LL * 8 ? b : 152LL * 8);
}

// setup kernels shared with the third level (mg_setup.cu)
__global__ void __launch_bounds__(RED_THREADS) k_nv_init(double2* __restrict__ r, const double2* __restrict__ Av, long long n, RedScratch rs,
                          NvState* S, int maxiter);
__global__ void __launch_bounds__(RED_THREADS) k_nv_alpha(const double2* __restrict__ t, long long n, RedScratch rs, NvState* S);
__global__ void __launch_bounds__(RED_THREADS) k_nv_update(double2* __restrict__ x, double2* __restrict__ r, const double2* __restrict__ p,
                            const double2* __restrict__ Ap, long long n, RedScratch rs, NvState* S, double tol2,
                            int maxiter);
__global__ void k_nv_p(double2* __restrict__ p, const double2* __restrict__ r, long long n, const NvState* S);
__global__ void k_block_ortho(const double2* __restrict__ vecs, double2* __restrict__ P, AggIndex ai, int nchd,
                              int ncol, int dof, int nvec, long long V, int nb, int* status, int cblock);
__global__ void k_blocks_to_f32(const double2* __restrict__ Y, float2* __restrict__ Y32, long long nblocks, int ncd);
__global__ void k_blocks_to_f16(const double2* __restrict__ Y, __half2* __restrict__ Y16, long long nblocks, int ncd);
__global__ void k_d2f(const double2* __restrict__ a, float2* __restrict__ b, long long n);

// the third level: the level-2 solve of the K-cycle (FGCR preconditioned by the
// level-3 solve) from r_c to e_c on one right-hand side; iteration counts out
dwf_status level2_solve(dwf_mg* h, const float2* rc, float2* ec, int* l2_iters, int* l3_iters, cudaStream_t st);
void level3_free(dwf_mg* h);

inline long long fine_len(const dwf_mg* h) { return h->G.V * h->G.Ls * site_dof(h->G); }
inline long long coarse_len(const dwf_mg* h) { return h->mg.Vc * h->mg.Ls_c * h->mg.ncd; }

}  // namespace dwf
