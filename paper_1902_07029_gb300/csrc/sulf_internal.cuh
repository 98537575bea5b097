// Internal declarations of the sulfmg CUDA library (GB300, sm_103a).
//
// Data layout (per multigrid level, all resident in device memory):
//   * dense box arrays of n^dim nodes, x fastest: level set phi (FP64), node
//     type (int8: 0 inactive, 1 inside, 2 ghost, 3 band), and the vectors of the
//     level as interleaved (s, c) pairs -- double2 (FP64) or float2 (FP32) --
//     so one 16- or 8-byte load fetches both unknowns of a node;
//   * compacted int32 index lists built once per level: inside nodes split by
//     red-black colour, ghosts, band nodes; kernels run one thread per listed
//     node, so inactive regions of the box cost nothing but the list;
//   * per-ghost boundary-row data (upwind signs, 1-D weights at offsets 0,1,2),
//     per-band-node upwind references, and node->ghost / node->band maps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/sulfmg.h"

#define SULF_MAXLEV 20

namespace sulf {

enum { T_OUT = 0, T_IN = 1, T_GHOST = 2, T_BAND = 3 };

template <typename T>
struct V2;
template <>
struct V2<double> {
    typedef double2 t;
};
template <>
struct V2<float> {
    typedef float2 t;
};

// Geometry of one level (precision independent).
struct LevelGeo {
    int dim = 2, N = 0, n = 0;
    long long nn = 0;
    long long st[3] = {1, 0, 0};
    double lo = 0, h = 0;
    double* phi = nullptr;
    int8_t* type = nullptr;
    int nin[2] = {0, 0};
    int* inl[2] = {nullptr, nullptr};  // inside nodes by colour (parity of the index sum)
    int ng = 0;
    int* gidx = nullptr;    // ghost nodes, box order
    int* gpos = nullptr;    // node -> ghost index or -1
    int8_t* gkind = nullptr;  // 0 quadratic, 1 linear, 2 identity row
    int8_t* gm = nullptr;     // ng*dim upwind signs
    double* gw = nullptr;     // ng*dim*3 1-D weights at offsets 0,1,2
    float* gw32 = nullptr;
    double* gB = nullptr;     // ng*dim boundary points
    int8_t* gord = nullptr;   // ng*dim per-axis interpolation orders of the row
    double* gth = nullptr;    // ng*dim theta per axis at B
    double* gnt = nullptr;    // ng*dim unit normal of the interpolated level set at B
    // each ghost's boundary row as a member table, member-major (kk * ng + gi)
    // over the K = 3^dim members of its upwind stencil: tensor weight (0 when
    // absent), box node, ghost index of the member or -1
    double* gwk = nullptr;
    float* gwk32 = nullptr;
    int* gnode = nullptr;
    int* gsrc = nullptr;
    int nb = 0;
    int* bidx = nullptr;     // band nodes, box order
    int* bref = nullptr;     // nb*dim: >=0 band index, -1 none, <=-2 ghost node -(idx+2)
    double* ban = nullptr;   // nb*dim |n_a|
    float* ban32 = nullptr;
    // the band extension as one linear operator (CSR over band nodes): the
    // extended defect at band node b is sum_j eval[j] * res(eidx[j]) over
    // j in [eptr[b], eptr[b+1]), eidx a ghost node
    int* eptr = nullptr;
    int* eidx = nullptr;
    double* eval = nullptr;
    float* eval32 = nullptr;
    long long ne = 0;
    // the P passes of the ghost relaxation composed into one affine map per
    // ghost (CSR over ghosts): s_g after the passes is sum_j gop_val[j] *
    // u(gop_code[j]) over j in [gop_ptr[gi], gop_ptr[gi+1]), u(code) the s of
    // box node code (code >= 0), else with u = ~code: the s of ghost u >> 1
    // before the passes (u even) or the right-hand side of box node u >> 1 (u
    // odd).  Built for (gop_tau, gop_passes, gop_bc); gop_on false where the
    // map would be too large (the passes then run one by one).
    int* gop_ptr = nullptr;
    int* gop_code = nullptr;
    double* gop_val = nullptr;
    float* gop_val32 = nullptr;
    long long gop_nnz = 0, gop_cap = 0;
    bool gop_on = false;
    double gop_tau = 0;
    int gop_passes = 0, gop_bc = -1;
    // lexicographic smoother (built on first use): the inside nodes ordered by
    // the index sum i+j(+k) (a wavefront), then box order; lexptr[d] is the
    // first position of wavefront d, nlexd wavefronts
    int* lex = nullptr;
    int* lexptr = nullptr;
    int nlexd = 0;
    // tiles of the temporally blocked FP32 sweep (3-D): ids ((tz * tile_ny) +
    // ty) * tile_nx + tx of the 32 x 8 x 16 tiles that hold an inside node
    int* tiles = nullptr;
    int ntiles = 0, tile_nx = 0, tile_ny = 0;
    int nact = 0;            // coarsest level: active list and map
    int* act = nullptr;
    int* apos = nullptr;
    int kinds[3] = {0, 0, 0};
};

// Vectors of one level for one precision.
template <typename T>
struct LevelVec {
    typedef typename V2<T>::t T2;
    T2* Wc = nullptr;   // (s, c) the Jacobian coefficients are evaluated at
    T2* rhs = nullptr;  // right-hand side of J x = rhs on this level
    // FP64 levels: rhs again per list position (inside colour 0, colour 1,
    // ghosts), written beside rhs by each of its writers (the Newton residual
    // F, the restriction, the debug inputs); the colour sweeps and the
    // residual read it in whole sectors.  Null for FP32 levels.
    T2* rhsc = nullptr;
    T2* x = nullptr;    // unknown: Newton update (finest) or coarse-grid error
    T2* res = nullptr;  // defect rhs - J x (band entries: extended defect)
    T* gbuf[2] = {nullptr, nullptr};   // ghost s values between relaxation passes
    T2* x2 = nullptr;   // the other unknown buffer of the tiled sweep (which writes one while reading the other)
    T* Ainv = nullptr;  // coarsest level: inverse of the assembled Jacobian
    T* A = nullptr;     // coarsest level: work matrix
    // Jacobian stencil coefficients, refreshed once per Newton iteration from
    // Wc (the matrix is constant during a linear solve):
    T2* edge[3] = {nullptr, nullptr, nullptr};  // per node (g, e) toward the +axis neighbour:
                                                // g = kappa (phi_q + phi_p), e = kappa alpha (s_p - s_q)
    T2* Pa = nullptr;  // inside nodes: (J^ss_pp, J^sc_pp)
    T2* Pb = nullptr;  //               (J^cs_pp, J^cc_pp)
    T2* Ia = nullptr;  //               rows of the inverse of that 2x2 block
    T2* Ib = nullptr;
    // the same blocks per position t of the inside lists (colour 0, then
    // colour 1): (Pa, Pb) at 2t, 2t+1 of Pc and (Ia, Ib) of Ic.  A colour's
    // sweep visits every other node of a box row, so box-ordered arrays give
    // it half-used 32-byte sectors; these give it whole ones
    T2* Pc = nullptr;
    T2* Ic = nullptr;
    T2* gc = nullptr;  // per ghost: (J^cs_gg, J^cc_gg)
    T* gci = nullptr;  // per ghost: 1 / J^cc_gg (an FP64 division costs ~10 instructions
                       // of a pipe with two lanes per SM per clock: divided once per
                       // Newton iteration instead of at every use)
};

// Jacobian coefficients of a level (Sec. 3.4, exact derivative of F).
template <typename T>
struct Coef {
    T alpha, beta;
    T a2mc;  // a / (2 m_c)
    T a2ms;  // a / (2 m_s)
    T idt;   // 1 / dt
    T kap;   // d / (4 h^2)
    T tau;   // ghost relaxation parameter
};

// Constants of the Newton residual on the finest level (Eqs. FDs, FDc, BCs).
struct FConst {
    double alpha, beta, amc, ams;  // a/m_c, a/m_s
    double idt, dh2;               // 1/dt, d/(2h^2)
    double sb;                     // Dirichlet value
    const double2* src;            // optional CN-averaged sources (f1, f2) per box node
    const double* sbg;             // optional Dirichlet value per ghost
};

// Device memory owned by one handle, from the device's stream-ordered pool
// (cudaMallocAsync / cudaFreeAsync on the handle's stream), so creating and
// destroying domains does not synchronise the work of other streams.
struct DevMem {
    std::vector<void*> ptrs;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;
    void* get(size_t n);
    void release();
};

// ---- geometry (geometry.cu) ----
int build_level_geometry(LevelGeo& L, const LevelGeo* finer, bool finest, bool coarsest, DevMem& mem,
                         cudaStream_t s, std::string& err, long long& launches);
// (re)build the boundary rows of a level's ghosts for boundary condition bc
// (0 Dirichlet, Eq. BCs; 1 Neumann, Eq. BCsN): normals, orders, weights,
// member tables; the finest level refuses identity rows (SULF_EGEOM)
int build_ghost_rows(LevelGeo& L, int bc, bool finest, cudaStream_t s, std::string& err, long long& launches);
// (re)build the composed ghost relaxation map of a level for relaxation
// parameter tau, `passes` passes and the current rows (boundary condition bc);
// leaves gop_on false where a row or the whole map exceeds its size bound
int build_ghost_op(LevelGeo& L, double tau, int passes, int bc, DevMem& mem, cudaStream_t s, std::string& err,
                   long long& launches);
// entries per ghost the composed map may hold on average (device-memory bound)
constexpr int kGopAvg2 = 24, kGopAvg3 = 27;
// whether the level's composed map applies to relaxation parameter tau (in
// the precision of the cycle) and `passes` passes
template <typename T>
inline bool ghost_op_ready(const LevelGeo& L, T tau, int passes) {
    return L.gop_on && L.gop_passes == passes && (T)L.gop_tau == tau;
}

// ---- multigrid and Newton kernels (kernels.cu); each returns kernels launched ----
template <int D, typename T>
int launch_coefs(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, cudaStream_t s);
// snap: when not null, the same launch also copies the s of every ghost of the
// level into snap (ghost order); the inside update never writes a ghost
template <int D, typename T>
int launch_relax_inside(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int colour, bool pointwise,
                        T* snap, cudaStream_t s);
// one lexicographic collective Gauss-Seidel sweep over the inside nodes,
// wavefront by wavefront in one CTA (nodes of a wavefront do not couple; its
// lower neighbours are already updated, its upper ones not: exactly the box
// order of a lexicographic sweep); snap as in launch_relax_inside
template <int D, typename T>
int launch_relax_lex(const LevelGeo& L, const LevelVec<T>& V, T* snap, cudaStream_t s);
// one red-black sweep of the FP32 collective smoother (both colours,
// stencil coefficients from (s, c)) over the level's tiles, temporally
// blocked in shared memory (3-D): reads xin, writes xout at the inside nodes
// and ghosts; snap as in launch_relax_inside
int launch_sweep_tiled(const LevelGeo& L, const float2* Wc, const float2* rhs, const float2* xin, float2* xout,
                       const Coef<float>& c, float* snap, cudaStream_t s);
// the ghost relaxation of one sweep: the composed map when `composed` (the
// caller checked ghost_op_ready and had the preceding inside launch copy the
// ghosts' s into V.gbuf[0]), else pass by pass
template <int D, typename T>
int launch_relax_ghosts(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int passes, bool composed,
                        cudaStream_t s);
template <int D, typename T>
int launch_residual(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, unsigned long long* norm,
                    cudaStream_t s);
// the finest-level FP64 defect of the mixed form stored, rounded to FP32, as
// the next FP32 right-hand side (the FP64 defect itself is not stored)
template <int D>
int launch_residual_to32(const LevelGeo& L, const LevelVec<double>& V, float2* out, unsigned long long* norm,
                         cudaStream_t s);
template <int D, typename T>
int launch_extend(const LevelGeo& L, const LevelVec<T>& V, cudaStream_t s);
// first_red: also the red half of the coarse level's first relaxation from
// the zero error, for the red inside nodes (the caller then skips that launch)
template <int D, typename T>
int launch_restrict(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                    bool first_red, bool pointwise, cudaStream_t s);
template <int D, typename T>
int launch_prolong(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                   cudaStream_t s);
template <int D, typename T>
int launch_inject(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                  cudaStream_t s);
template <int D, typename T>
int launch_coarsest_factor(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int* singular,
                           cudaStream_t s);
template <int D, typename T>
int launch_coarsest_solve(const LevelGeo& L, const LevelVec<T>& V, cudaStream_t s);

template <int D>
int launch_old_time(const LevelGeo& L, const double2* Wn, double2* G, const FConst& fc, cudaStream_t s);
// the list-ordered copy (rhsc) of a level's box-ordered rhs, for inputs
// written into rhs directly
int launch_gather_list(const LevelGeo& L, const double2* box, double2* list, cudaStream_t s);
// (Fc: the list-ordered copy of F, the finest level's rhsc, or null)
template <int D>
int launch_newton_F(const LevelGeo& L, const double2* W, const double2* G, double2* F, double2* Fc,
                    const FConst& fc, unsigned long long* norm, cudaStream_t s);
int launch_newton_update(const LevelGeo& L, double2* W, const double2* x, unsigned long long* norms,
                         cudaStream_t s);
int launch_norm_active(const LevelGeo& L, const double2* v, unsigned long long* norm, cudaStream_t s);

// linear extrapolation of u (device box of level L) from its inside nodes to
// the rest of the box (levelset.cu); q, q2, u2 are work arrays of nn doubles
int launch_extrapolate(const LevelGeo& L, double* u, double* q, double* q2, double* u2, int iters, cudaStream_t s);

// CN average of manufactured source terms: src = ((f1o+f1n)/2, (f2o+f2n)/2)
int launch_average_sources(long long nn, const double* f4, double2* src, cudaStream_t s);

// the convergence test at the end of a cycle of the device-side loop
// (conditional graph node h): cycles counts, rnorms[cycle-1] records the
// defect norm
int launch_cycle_check(cudaGraphConditionalHandle h, const unsigned long long* norm, const int* singular,
                       const double* thr, int max_cycles, int* cycles, double* rnorms, cudaStream_t s);

// mixed precision transfers on the finest level (active nodes)
int launch_to_float(const LevelGeo& L, const double2* src, float2* dst, cudaStream_t s);
int launch_accumulate(const LevelGeo& L, double2* x, const float2* e, cudaStream_t s);

// state import / export
int launch_reset_state(const LevelGeo& L, double2* W, double s0, double c0, cudaStream_t s);
int launch_import_state(const LevelGeo& L, double2* W, const double* sv, const double* cv, cudaStream_t s);
int launch_export_state(const LevelGeo& L, const double2* W, double* sv, double* cv, int8_t* tv, cudaStream_t s);

// fused coarsest levels of the V-cycle, one CTA (tail.cu)
size_t tail_desc_bytes(int L);
template <typename T>
int upload_tail_desc(const LevelGeo* G, const LevelVec<T>* V, int L, void* dev, cudaStream_t s);
// compose: every level from l0 down relaxes its ghosts by the composed map
// (the descriptor's pointers are those of the maps built for the current
// solver controls and boundary condition)
template <int D, typename T>
int launch_tail(const void* dev_desc, const LevelGeo* G, int l0, int L, const sulf_solver& sv, int bc, bool compose,
                cudaStream_t s);
// the fused levels l0 .. L-1 of K instances' cycles in one launch (one CTA
// per instance; dev_descs: device array of the instances' descriptors; G[i]:
// instance i's level geometry; masked instances skipped)
template <int D, typename T>
int launch_tail_batched(const void* const* dev_descs, int K, const int* active, const LevelGeo* const* G, int l0,
                        int L, const sulf_solver& sv, int bc, bool compose, cudaStream_t s);

// factor of tau_s for Neumann ghost rows on a level of spacing h (Eq.
// CFLcondN): 4 h / (3 sqrt(dim)), i.e. 2 sqrt(2) h / 3 in 2-D
__host__ __device__ inline double tail_tau_scale(int dim, double h) {
    return 4.0 * h / (3.0 * (dim == 3 ? 1.7320508075688772 : 1.4142135623730951));
}

// Programmatic dependent launch.  Every kernel of the Newton and multigrid
// path starts with pdl_enter(): griddepcontrol.wait blocks until the previous
// kernel on the stream has completed and its writes are visible (a no-op when
// the kernel was launched without the attribute), then launch_dependents lets
// the next kernel's CTAs be scheduled while this one runs.  The next grid
// therefore waits, resident, for this one instead of paying its launch latency
// after it; at most two grids of a stream are in flight.  All threads pass the
// wait before any global access.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// launches made by the calling thread use the attribute while on (solver.cu
// switches it per call from sulf_solver::pdl)
void set_launch_pdl(bool on);
bool launch_pdl();
// the FP64 inside relaxation's register budget (sulf_solver::relax_occupancy)
// for launches made by the calling thread
void set_launch_occupancy(int occ);
int launch_occupancy();
// FP32 inside relaxation with the coefficients recomputed from (s, c)
// (sulf_solver::relax_matrix_free) for launches made by the calling thread
void set_launch_matrix_free(int mf);
int launch_matrix_free();

// the first failed launch of the calling thread is remembered (a failed launch
// inside stream capture only surfaces later, as an invalidated capture) and
// reported with the next CUDA error
void note_launch_error(cudaError_t e, unsigned grid, unsigned block, size_t smem);
std::string take_launch_error();

template <typename... P, typename... A>
inline void launch_k(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = launch_pdl() ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
    if (e != cudaSuccess) note_launch_error(e, grid, block, smem);
}

// read-only views of a handle (solver.cu)
const LevelGeo* handle_fine_geo(sulf_handle h);
const sulf_model* handle_model(sulf_handle h);
int handle_bc(sulf_handle h);
cudaStream_t handle_stream(sulf_handle h);
void handle_count_launches(sulf_handle h, int n);
int handle_device(sulf_handle h);       // the device the handle was created on
void** handle_noalloc_slot(sulf_handle h);  // per-handle cache of a device address (noalloc.cu)
// lock-step batching (solver.cu): whether a domain can join a class (and the
// class key: domains with equal keys and equal (dt, nsteps) step together),
// and nsteps CN steps of K such domains, all on stream s, in lock step
bool lockstep_key(sulf_handle h, std::vector<double>& key);
int lockstep_advance(const sulf_handle* hs, int K, double dt, int nsteps, int* status, std::vector<std::string>& err,
                     cudaStream_t s);

}  // namespace sulf

#define SULF_CUDA_TRY(expr)                                       \
    do {                                                          \
        cudaError_t e__ = (expr);                                 \
        if (e__ != cudaSuccess) return sulf_fail_cuda(e__, #expr); \
    } while (0)

int sulf_fail_cuda(cudaError_t e, const char* what);
int sulf_fail(int code, const std::string& msg);
