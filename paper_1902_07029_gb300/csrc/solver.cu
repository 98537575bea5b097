// Host orchestration and C ABI of the sulfmg library: one handle per domain,
// the multigrid hierarchy resident on the device, Crank-Nicolson steps solved
// by Newton-Raphson (arXiv:1902.07029, Sec. 3.1 and 3.4) with level-set
// multigrid cycles (Sec. 3.5) issued as kernels on the handle's stream.
#include <array>
#include <chrono>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/sulfmg_debug.h"
#include "lockstep.cuh"
#include "sulf_internal.cuh"

using namespace sulf;

static thread_local std::string g_err;

int sulf_fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

int sulf_fail_cuda(cudaError_t e, const char* what) {
    g_err = std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e);
    std::string first = sulf::take_launch_error();
    if (!first.empty()) g_err += "; first failed launch: " + first;
    return e == cudaErrorMemoryAllocation ? SULF_ENOMEM : SULF_EDEVICE;
}

namespace sulf {

namespace {
// keep freed blocks in the device pool instead of returning them at each
// synchronisation (set once per device)
void retain_pool_memory() {
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ULL;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}
}  // namespace

void* DevMem::get(size_t n) {
    void* p = nullptr;
    size_t sz = (n + 255) & ~size_t(255);
    if (sz == 0) sz = 256;
    retain_pool_memory();
    if (cudaMallocAsync(&p, sz, stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    // set-up only: make the block usable from any stream right away
    if (cudaStreamSynchronize(stream) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    bytes += sz;
    return p;
}

void DevMem::release() {
    for (void* p : ptrs) cudaFreeAsync(p, stream);
    if (stream) cudaStreamSynchronize(stream);
    ptrs.clear();
    bytes = 0;
}

}  // namespace sulf

struct sulf_domain {
    int dim = 2, N = 0, L = 0;
    double lo = 0, hi = 0;
    LevelGeo geo[SULF_MAXLEV];
    LevelVec<double> v64[SULF_MAXLEV];
    LevelVec<float> v32[SULF_MAXLEV];
    bool have32 = false;
    int bc = 0;  // boundary condition for s: 0 Dirichlet (Eq. BCs), 1 Neumann (Eq. BCsN)
    double2* W = nullptr;   // state, = v64[0].Wc
    double2* Wn = nullptr;  // state at t_n
    double2* G = nullptr;   // old-time part of the CN step
    unsigned long long* dnorm = nullptr;
    unsigned long long* hnorm = nullptr;  // pinned
    int* dsing = nullptr;
    double* stage = nullptr;  // 2*nn doubles + nn bytes, device staging for state I/O
    // manufactured-solution inputs (optional): CN-averaged sources per box
    // node, their upload staging, and Dirichlet values per ghost
    double2* src = nullptr;
    double* src_stage = nullptr;
    double* sbg = nullptr;
    bool src_on = false, sbg_on = false;
    double* xbuf = nullptr;  // 5 * nn doubles: extrapolation of initial data
    sulf_model model{};
    sulf_solver solver{};
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    bool fmg_now = false;              // the next cycle_body is the full-multigrid cycle
    int device = 0;                    // the CUDA device current at creation
    void* noalloc_scratch = nullptr;   // device address of noalloc.cu's static scratch, looked up on
                                       // this handle's first sulf_newton_residual_noalloc call
    DevMem mem;
    double t = 0, dt = 0;
    // statistics
    int newton_last = 0, cycles_last = 0;
    long long newton_total = 0, cycles_total = 0, steps_total = 0, launches = 0;
    double last_rho = 0, last_fnorm = 0;
    // profiling of the finest-level inside relaxation: 0 off, 1 the first
    // finest-level sweep of every cycle, 2 every finest-level sweep
    int prof = 0;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    double prof_ms = 0;
    long long prof_n = 0;
    // one multigrid cycle captured as a CUDA graph, per precision; recaptured
    // when anything baked into it changes
    struct CycleGraph {
        cudaGraphExec_t exec = nullptr;
        double dt = 0;
        sulf_solver sv{};
        int prof = 0;
        long long kernels = 0;
        size_t ev0 = 0, ev1 = 0;
    } graph[2];
    bool capturing = false;
    // The linear solve as one graph launch, per precision: a conditional
    // while node whose body is one cycle and its convergence test on the
    // device (no host round trip per cycle).  Rebuilt when anything baked
    // into it changes; off for good on this handle if the runtime refuses it.
    struct LoopGraph {
        cudaGraphExec_t exec = nullptr;
        double dt = 0;
        sulf_solver sv{};
        int max_cycles = 0;
        long long kernels = 0;  // per cycle
    } loop[2];
    bool loop_off = false;
    bool loop_used = false;  // the last linear solve ran as one loop-graph launch
    int* dcyc = nullptr;      // cycles run by the device loop
    double* drn = nullptr;    // their defect norms (kLoopMaxCycles)
    double* dthr = nullptr;   // threshold rtol * |F|
    double* hloop = nullptr;  // pinned: threshold, cycle count, norms
    // fused coarsest levels: device descriptors per precision
    void* tail_desc[2] = {nullptr, nullptr};
    bool tail_ready[2] = {false, false};
};

namespace {

// Jacobi steps of each stage of the initial-data extrapolation (d tau = h/2:
// the ghosts lie within about 2 h of the inside nodes whose normal derivative
// is known, and the steps contract toward the steady state)
constexpr int kExtrapolationIters = 64;

sulf_solver default_solver() {
    sulf_solver s;
    s.nu1 = 2;
    s.nu2 = 2;
    s.cycle = 1;
    s.max_newton = 20;
    s.max_cycles = 30;
    s.ghost_sweeps = 4;
    s.newton_tol = 1e-10;
    s.lin_rtol = 1e-10;
    s.tau_s = 0.9;
    s.precision = 0;
    s.smoother = 0;
    s.graphs = 1;
    s.fuse_below = -1;
    s.pdl = 1;
    s.ghost_compose = 1;
    s.relax_occupancy = 0;
    s.relax_matrix_free = 1;
    return s;
}

sulf_model default_model() {
    sulf_model m;
    m.a = 1e4;
    m.d = 0.1;
    m.m_s = 64.06;
    m.m_c = 100.09;
    m.alpha = 0.01;
    m.beta = 0.1;
    m.s_ext = 1.0;
    m.s0 = 0.0;
    m.c0 = 10.0;
    return m;
}

double host_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

double bits_to_double(unsigned long long b) {
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
}

// the ghost relaxation parameter of level l; Neumann rows have a diagonal of
// order 1/h: tau_s scales the bound of Eq. CFLcondN, 2 sqrt(2) h / 3 in 2-D,
// i.e. 4 h / (3 sqrt(d))
double level_tau(const sulf_domain* d, int l) {
    return d->bc ? d->solver.tau_s * tail_tau_scale(d->dim, d->geo[l].h) : d->solver.tau_s;
}

template <typename T>
Coef<T> make_coef(const sulf_domain* d, int l) {
    Coef<T> c;
    const sulf_model& m = d->model;
    double h = d->geo[l].h;
    c.alpha = (T)m.alpha;
    c.beta = (T)m.beta;
    c.a2mc = (T)(m.a / (2.0 * m.m_c));
    c.a2ms = (T)(m.a / (2.0 * m.m_s));
    c.idt = (T)(1.0 / d->dt);
    c.kap = (T)(m.d / (4.0 * h * h));
    c.tau = (T)level_tau(d, l);
    return c;
}

FConst make_fconst(const sulf_domain* d) {
    FConst f;
    const sulf_model& m = d->model;
    double h = d->geo[0].h;
    f.alpha = m.alpha;
    f.beta = m.beta;
    f.amc = m.a / m.m_c;
    f.ams = m.a / m.m_s;
    f.idt = 1.0 / d->dt;
    f.dh2 = m.d / (2.0 * h * h);
    f.sb = m.s_ext;
    f.src = d->src_on ? d->src : nullptr;
    f.sbg = d->sbg_on ? d->sbg : nullptr;
    return f;
}

template <typename T>
int alloc_vectors(sulf_domain* d, LevelVec<T>* V, bool share_state) {
    typedef typename V2<T>::t T2;
    for (int l = 0; l < d->L; l++) {
        const LevelGeo& G = d->geo[l];
        LevelVec<T>& v = V[l];
        size_t nb2 = sizeof(T2) * G.nn;
        if (!(share_state && l == 0)) v.Wc = (T2*)d->mem.get(nb2);
        v.rhs = (T2*)d->mem.get(nb2);
        v.x = (T2*)d->mem.get(nb2);
        v.res = (T2*)d->mem.get(nb2);
        for (int k = 0; k < 2; k++) v.gbuf[k] = (T*)d->mem.get(sizeof(T) * (G.ng + 1));
        for (int a = 0; a < G.dim; a++) v.edge[a] = (T2*)d->mem.get(nb2);
        v.Pa = (T2*)d->mem.get(nb2);
        v.Pb = (T2*)d->mem.get(nb2);
        v.Ia = (T2*)d->mem.get(nb2);
        v.Ib = (T2*)d->mem.get(nb2);
        const size_t nc2 = sizeof(T2) * 2 * ((size_t)G.nin[0] + G.nin[1] + 1);
        v.Pc = (T2*)d->mem.get(nc2);
        v.Ic = (T2*)d->mem.get(nc2);
        v.gc = (T2*)d->mem.get(sizeof(T2) * (G.ng + 1));
        v.gci = (T*)d->mem.get(sizeof(T) * (G.ng + 1));
        if (std::is_same<T, double>::value) {
            const size_t nl = sizeof(T2) * ((size_t)G.nin[0] + G.nin[1] + G.ng + 1);
            v.rhsc = (T2*)d->mem.get(nl);
            if (!v.rhsc) return sulf_fail(SULF_ENOMEM, "out of device memory");
            SULF_CUDA_TRY(cudaMemsetAsync(v.rhsc, 0, nl, d->stream));
        }
        if (!v.Pa || !v.Pb || !v.Ia || !v.Ib || !v.Pc || !v.Ic || !v.gc || !v.gci || !v.edge[0] || !v.edge[1] ||
            (G.dim == 3 && !v.edge[2]))
            return sulf_fail(SULF_ENOMEM, "out of device memory");
        if ((!share_state || l > 0) && !v.Wc) return sulf_fail(SULF_ENOMEM, "out of device memory");
        if (!v.rhs || !v.x || !v.res || !v.gbuf[0] || !v.gbuf[1])
            return sulf_fail(SULF_ENOMEM, "out of device memory");
        if (v.Wc) SULF_CUDA_TRY(cudaMemsetAsync(v.Wc, 0, nb2, d->stream));
        SULF_CUDA_TRY(cudaMemsetAsync(v.rhs, 0, nb2, d->stream));
        SULF_CUDA_TRY(cudaMemsetAsync(v.x, 0, nb2, d->stream));
        SULF_CUDA_TRY(cudaMemsetAsync(v.res, 0, nb2, d->stream));
        if (l == d->L - 1) {
            size_t m = 2 * (size_t)G.nact;
            v.A = (T*)d->mem.get(sizeof(T) * (m * m + 1));
            v.Ainv = (T*)d->mem.get(sizeof(T) * (m * m + 1));
            if (!v.A || !v.Ainv) return sulf_fail(SULF_ENOMEM, "out of device memory");
        }
    }
    return SULF_OK;
}

int ensure32(sulf_domain* d) {
    if (d->have32) return SULF_OK;
    int rc = alloc_vectors<float>(d, d->v32, false);
    if (rc) return rc;
    d->have32 = true;
    return SULF_OK;
}

// ---- profiling events around the finest-level inside relaxation ----
cudaEvent_t next_event(sulf_domain* d) {
    if (d->evused == d->evpool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        d->evpool.push_back(e);
    }
    return d->evpool[d->evused++];
}

int read_norms(sulf_domain* d, int n) {
    SULF_CUDA_TRY(cudaMemcpyAsync(d->hnorm, d->dnorm, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                                  d->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
    return SULF_OK;
}

// first level handled by the fused coarse-level cycle (-1: none)
int tail_level(const sulf_domain* d) {
    // automatic threshold: the fused kernel runs on one SM, whose FP64 rate is
    // two lanes per clock, so FP64 cycles fuse only the smallest levels
    const int fb = d->solver.fuse_below >= 0 ? d->solver.fuse_below : (d->solver.precision == 0 ? 150 : 1000);
    if (fb <= 0 || d->solver.cycle != 1 || d->solver.smoother == 2) return -1;
    for (int l = 0; l < d->L - 1; l++)
        if ((long long)d->geo[l].nin[0] + d->geo[l].nin[1] + d->geo[l].ng <= fb) return l;
    return -1;
}

// device descriptors of the levels for the fused cycle (pointers are fixed once
// the vectors exist); must run outside stream capture
template <int D, typename T>
int ensure_tail(sulf_domain* d, const LevelVec<T>* V) {
    int p = std::is_same<T, float>::value ? 1 : 0;
    if (d->tail_ready[p]) return SULF_OK;
    if (!d->tail_desc[p]) {
        d->tail_desc[p] = d->mem.get(tail_desc_bytes(d->L));
        if (!d->tail_desc[p]) return sulf_fail(SULF_ENOMEM, "out of device memory");
    }
    int rc = upload_tail_desc<T>(d->geo, V, d->L, d->tail_desc[p], d->stream);
    if (rc) return rc;
    d->tail_ready[p] = true;
    return SULF_OK;
}

// forget the captured cycles (they hold pointers and parameters that changed)
void drop_graphs(sulf_domain* d) {
    for (auto& g : d->graph)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
    for (auto& g : d->loop)
        if (g.exec) {
            cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
        }
}

// (re)build the composed ghost relaxation of every level whose map was built
// for another relaxation parameter, pass count or boundary condition
int refresh_ghost_ops(sulf_domain* d) {
    if (!d->solver.ghost_compose) return SULF_OK;
    bool changed = false;
    for (int l = 0; l < d->L; l++) {
        LevelGeo& G = d->geo[l];
        const double tau = level_tau(d, l);
        if (G.gop_bc == d->bc && G.gop_passes == d->solver.ghost_sweeps && G.gop_tau == tau) continue;
        std::string err;
        int rc = build_ghost_op(G, tau, d->solver.ghost_sweeps, d->bc, d->mem, d->stream, err, d->launches);
        if (rc) return sulf_fail(rc, err);
        changed = true;
    }
    if (changed) {
        // the fused kernel's descriptors hold the maps' pointers
        drop_graphs(d);
        d->tail_ready[0] = d->tail_ready[1] = false;
    }
    return SULF_OK;
}

// levels (3-D, FP32 cycles) whose red-black sweeps run as one temporally
// blocked kernel (sulf_solver::relax_matrix_free = 2): those with at least
// kTileMinInside inside nodes; the sweep writes the other unknown buffer, so
// it needs an even number of sweeps per relaxation (nu1, nu2 even)
constexpr long long kTileMinInside = 100000;
bool tiled_level(const sulf_domain* d, int l) {
    const LevelGeo& G = d->geo[l];
    return d->solver.relax_matrix_free == 2 && d->solver.precision == 1 && d->solver.smoother == 0 && G.dim == 3 &&
           d->solver.nu1 % 2 == 0 && d->solver.nu2 % 2 == 0 && G.tiles != nullptr && d->v32[l].x2 != nullptr;
}

// ---- multigrid on precision T ----
template <int D, typename T>
struct MG {
    sulf_domain* d;
    LevelVec<T>* V;
    int fine_sweeps = 0;  // finest-level sweeps issued so far in this cycle

    // skip_red: the red half-sweep was done by the restriction (from zero)
    int relax(int l, bool skip_red = false) {
        const LevelGeo& G = d->geo[l];
        Coef<T> c = make_coef<T>(d, l);
        bool pw = d->solver.smoother == 1;
        const bool timed_sweep = l == 0 && (d->prof == 2 || (d->prof == 1 && fine_sweeps == 0));
        if (l == 0) fine_sweeps++;
        // the composed ghost relaxation starts from a copy of the ghosts' s
        // taken by the second colour's launch
        const bool gop =
            d->solver.ghost_compose && G.gop_bc == d->bc && ghost_op_ready<T>(G, c.tau, d->solver.ghost_sweeps);
        // one event bracket around the two colour launches of a timed sweep
        // (inside stream capture a plain record only adds a dependency; the
        // external flag makes it an event-record node of the graph)
        const unsigned fl = d->capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
        if (timed_sweep) cudaEventRecordWithFlags(next_event(d), d->stream, fl);
        if (std::is_same<T, float>::value && !skip_red && tiled_level(d, l)) {
            // both colours in one temporally blocked launch into the other
            // buffer, which then becomes the level's unknown
            LevelVec<float>& U = reinterpret_cast<LevelVec<float>&>(V[l]);
            Coef<float> cf;
            cf.alpha = (float)c.alpha;
            cf.beta = (float)c.beta;
            cf.a2mc = (float)c.a2mc;
            cf.a2ms = (float)c.a2ms;
            cf.idt = (float)c.idt;
            cf.kap = (float)c.kap;
            cf.tau = (float)c.tau;
            d->launches += launch_sweep_tiled(G, U.Wc, U.rhs, U.x, U.x2, cf, gop ? U.gbuf[0] : nullptr, d->stream);
            std::swap(U.x, U.x2);
        } else if (d->solver.smoother == 2)
            d->launches += launch_relax_lex<D, T>(G, V[l], gop ? V[l].gbuf[0] : nullptr, d->stream);
        else
            for (int colour = skip_red ? 1 : 0; colour < 2; colour++)
                d->launches += launch_relax_inside<D, T>(G, V[l], c, colour, pw,
                                                         gop && colour == 1 ? V[l].gbuf[0] : nullptr, d->stream);
        if (timed_sweep) cudaEventRecordWithFlags(next_event(d), d->stream, fl);
        d->launches += launch_relax_ghosts<D, T>(G, V[l], c, d->solver.ghost_sweeps, gop, d->stream);
        return SULF_OK;
    }

    // red_done: level l's error was just restricted to zero and its first
    // red half-sweep done with it
    int cycle(int l, bool red_done = false) {
        if (l == d->L - 1) {
            d->launches += launch_coarsest_solve<D, T>(d->geo[l], V[l], d->stream);
            return SULF_OK;
        }
        int p = std::is_same<T, float>::value ? 1 : 0;
        int rc;
        if (l == tail_level(d) && d->tail_ready[p] && d->solver.cycle == 1) {
            // this level and all coarser ones in one single-CTA launch
            bool compose = d->solver.ghost_compose != 0;
            for (int k = l; k < d->L && compose; k++) {
                const LevelGeo& G = d->geo[k];
                compose = G.ng == 0 || (G.gop_bc == d->bc &&
                                        ghost_op_ready<T>(G, make_coef<T>(d, k).tau, d->solver.ghost_sweeps));
            }
            rc = launch_tail<D, T>(d->tail_desc[p], d->geo, l, d->L, d->solver, d->bc, compose, d->stream);
            if (rc) return rc;
            d->launches += 1;
            return SULF_OK;
        }
        for (int k = 0; k < d->solver.nu1; k++)
            if ((rc = relax(l, red_done && k == 0))) return rc;
        d->launches += launch_residual<D, T>(d->geo[l], V[l], make_coef<T>(d, l), nullptr, d->stream);
        d->launches += launch_extend<D, T>(d->geo[l], V[l], d->stream);
        // the next level starts from a zero error: where it runs as separate
        // kernels and pre-relaxes, the restriction also does its first red
        // half-sweep (which would read only zeros)
        const int lc = l + 1;
        const bool fused_tail = lc == tail_level(d) && d->tail_ready[p] && d->solver.cycle == 1;
        const bool fr = d->solver.nu1 >= 1 && lc < d->L - 1 && !fused_tail && d->solver.smoother != 2 &&
                        !(std::is_same<T, float>::value && tiled_level(d, lc));
        d->launches += launch_restrict<D, T>(d->geo[l], V[l], d->geo[lc], V[lc], fr, d->solver.smoother == 1,
                                             d->stream);
        int gam = d->solver.cycle == 2 ? 2 : 1;
        for (int g = 0; g < gam; g++)
            if ((rc = cycle(lc, fr && g == 0))) return rc;
        d->launches += launch_prolong<D, T>(d->geo[l], V[l], d->geo[l + 1], V[l + 1], d->stream);
        for (int k = 0; k < d->solver.nu2; k++)
            if ((rc = relax(l))) return rc;
        return SULF_OK;
    }

    // Full multigrid, the first cycle of a linear solve with cycle = 3: the
    // right-hand side goes down the hierarchy by the cycles' own residual (of
    // the zero start), band extension and restriction; the coarsest level is
    // solved directly; each finer level starts from the interpolated coarse
    // solution and takes one V-cycle.  Every level's x is zero on entry (the
    // finest by the caller, the coarse ones by the restriction).
    int fmg() {
        const bool pw = d->solver.smoother == 1;
        for (int l = 0; l + 1 < d->L; l++) {
            d->launches += launch_residual<D, T>(d->geo[l], V[l], make_coef<T>(d, l), nullptr, d->stream);
            d->launches += launch_extend<D, T>(d->geo[l], V[l], d->stream);
            d->launches += launch_restrict<D, T>(d->geo[l], V[l], d->geo[l + 1], V[l + 1], false, pw, d->stream);
        }
        d->launches += launch_coarsest_solve<D, T>(d->geo[d->L - 1], V[d->L - 1], d->stream);
        for (int l = d->L - 2; l >= 0; l--) {
            d->launches += launch_prolong<D, T>(d->geo[l], V[l], d->geo[l + 1], V[l + 1], d->stream);
            if (int rc = cycle(l)) return rc;
        }
        return SULF_OK;
    }

    // coarse coefficients from V[0].Wc, the stencil coefficients of every
    // level and the coarsest factorisation (once per Newton iteration)
    int prepare() {
        for (int l = 1; l < d->L; l++)
            d->launches += launch_inject<D, T>(d->geo[l - 1], V[l - 1], d->geo[l], V[l], d->stream);
        for (int l = 0; l < d->L; l++)
            d->launches += launch_coefs<D, T>(d->geo[l], V[l], make_coef<T>(d, l), d->stream);
        SULF_CUDA_TRY(cudaMemsetAsync(d->dsing, 0, sizeof(int), d->stream));
        int lc = d->L - 1;
        d->launches += launch_coarsest_factor<D, T>(d->geo[lc], V[lc], make_coef<T>(d, lc), d->dsing, d->stream);
        return SULF_OK;
    }
};

// sum the device time of the event pairs [from, to) of the pool
int accumulate_prof(sulf_domain* d, size_t from, size_t to) {
    for (size_t k = from; k + 1 < to; k += 2) {
        float e = 0;
        SULF_CUDA_TRY(cudaEventElapsedTime(&e, d->evpool[k], d->evpool[k + 1]));
        d->prof_ms += e;
        d->prof_n += 2;  // a bracket holds the two colour launches of a sweep
    }
    return SULF_OK;
}

bool same_solver(const sulf_solver& a, const sulf_solver& b) {
    return a.nu1 == b.nu1 && a.nu2 == b.nu2 && a.cycle == b.cycle && a.max_newton == b.max_newton &&
           a.max_cycles == b.max_cycles && a.ghost_sweeps == b.ghost_sweeps && a.newton_tol == b.newton_tol &&
           a.lin_rtol == b.lin_rtol && a.tau_s == b.tau_s && a.precision == b.precision && a.smoother == b.smoother &&
           a.graphs == b.graphs && a.fuse_below == b.fuse_below && a.pdl == b.pdl &&
           a.ghost_compose == b.ghost_compose && a.relax_occupancy == b.relax_occupancy &&
           a.relax_matrix_free == b.relax_matrix_free;
}

// One cycle of the linear solve on the finest level, then the FP64 defect
// r = F - J dW, its max-norm and the coarsest-level singularity flag copied to
// pinned host memory.  FP64: a multigrid cycle on J dW = F.  Mixed: an FP32
// cycle on J e = r from e = 0, dW += e, then the next FP32 right-hand side.
template <int D>
int cycle_body(sulf_domain* d, const cudaGraphConditionalHandle* loop = nullptr, int max_cycles = 0) {
    const LevelGeo& G0 = d->geo[0];
    LevelVec<double>& V0 = d->v64[0];
    const bool fmg = d->fmg_now && d->L > 1;
    if (d->solver.precision == 0) {
        if (d->L == 1)
            d->launches += launch_coarsest_solve<D, double>(G0, V0, d->stream);
        else if (int rc = fmg ? MG<D, double>{d, d->v64}.fmg() : MG<D, double>{d, d->v64}.cycle(0))
            return rc;
    } else {
        LevelVec<float>& U0 = d->v32[0];
        SULF_CUDA_TRY(cudaMemsetAsync(U0.x, 0, sizeof(float2) * G0.nn, d->stream));
        if (d->L == 1)
            d->launches += launch_coarsest_solve<D, float>(G0, U0, d->stream);
        else if (int rc = fmg ? MG<D, float>{d, d->v32}.fmg() : MG<D, float>{d, d->v32}.cycle(0))
            return rc;
        d->launches += launch_accumulate(G0, V0.x, U0.x, d->stream);
    }
    SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 2, d->stream));
    if (d->solver.precision == 1)  // straight into the next FP32 right-hand side
        d->launches += launch_residual_to32<D>(G0, V0, d->v32[0].rhs, d->dnorm, d->stream);
    else
        d->launches += launch_residual<D, double>(G0, V0, make_coef<double>(d, 0), d->dnorm, d->stream);
    if (!loop) {
        SULF_CUDA_TRY(
            cudaMemcpyAsync(d->hnorm, d->dnorm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, d->stream));
        SULF_CUDA_TRY(cudaMemcpyAsync(d->hnorm + 6, d->dsing, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    }
    if (loop) d->launches += launch_cycle_check(*loop, d->dnorm, d->dsing, d->dthr, max_cycles, d->dcyc, d->drn, d->stream);
    return SULF_OK;
}

constexpr int kLoopMaxCycles = 256;

// build the device-side loop graph of precision p: [cycle counter := 0] ->
// while (condition) { cycle; test }.  Returns false (and turns the loop off
// for this handle) where the runtime does not take it.
template <int D>
bool build_loop(sulf_domain* d, int max_cycles) {
    const int p = d->solver.precision;
    sulf_domain::LoopGraph& g = d->loop[p];
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    if (!d->dcyc) {
        d->dcyc = (int*)d->mem.get(sizeof(int) * 4);
        d->drn = (double*)d->mem.get(sizeof(double) * kLoopMaxCycles);
        d->dthr = (double*)d->mem.get(sizeof(double) * 2);
        if (!d->dcyc || !d->drn || !d->dthr) return false;
    }
    if (!d->hloop && cudaMallocHost(&d->hloop, sizeof(double) * (4 + kLoopMaxCycles)) != cudaSuccess) {
        d->hloop = nullptr;
        cudaGetLastError();
        return false;
    }
    cudaGraph_t outer = nullptr;
    if (cudaGraphCreate(&outer, 0) != cudaSuccess) return false;
    bool ok = false;
    do {
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, outer, 1, cudaGraphCondAssignDefault) != cudaSuccess) break;
        cudaMemsetParams mp = {};
        mp.dst = d->dcyc;
        mp.value = 0;
        mp.elementSize = sizeof(int);
        mp.width = 1;
        mp.height = 1;
        cudaGraphNode_t zero;
        if (cudaGraphAddMemsetNode(&zero, outer, nullptr, 0, &mp) != cudaSuccess) break;
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cn;
        if (cudaGraphAddNode(&cn, outer, &zero, nullptr, 1, &cp) != cudaSuccess) break;
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(d->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
            cudaSuccess)
            break;
        d->capturing = true;
        const long long l0 = d->launches;
        int rc = cycle_body<D>(d, &h, max_cycles);
        cudaGraph_t got = nullptr;
        cudaError_t e = cudaStreamEndCapture(d->stream, &got);
        d->capturing = false;
        g.kernels = d->launches - l0;
        d->launches = l0;
        if (rc || e != cudaSuccess) break;
        if (cudaGraphInstantiate(&g.exec, outer, 0) != cudaSuccess) {
            g.exec = nullptr;
            break;
        }
        ok = true;
    } while (false);
    cudaGraphDestroy(outer);
    if (!ok) {
        cudaGetLastError();
        take_launch_error();
        g_err.clear();
        d->loop_off = true;
        return false;
    }
    g.dt = d->dt;
    g.sv = d->solver;
    g.max_cycles = max_cycles;
    return true;
}

// The cycles of one linear solve as one launch of the loop graph; same
// results and statistics as the host loop.  Returns the number of cycles, 0
// where the loop is unavailable (the caller runs the host loop), or a
// negative error.
template <int D>
int device_loop(sulf_domain* d, double fnorm, int max_cycles, double rtol, double* rnorms) {
    if (d->loop_off || !d->solver.graphs || d->prof || max_cycles > kLoopMaxCycles || d->solver.cycle == 3) return 0;
    const int p = d->solver.precision;
    sulf_domain::LoopGraph& g = d->loop[p];
    if (!g.exec || g.dt != d->dt || !same_solver(g.sv, d->solver) || g.max_cycles != max_cycles)
        if (!build_loop<D>(d, max_cycles)) return 0;
    d->hloop[0] = rtol * fnorm;
    SULF_CUDA_TRY(cudaMemcpyAsync(d->dthr, d->hloop, sizeof(double), cudaMemcpyHostToDevice, d->stream));
    SULF_CUDA_TRY(cudaGraphLaunch(g.exec, d->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(d->hloop + 1, d->dcyc, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(d->hloop + 4, d->drn, sizeof(double) * max_cycles, cudaMemcpyDeviceToHost,
                                  d->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(d->hnorm + 6, d->dsing, sizeof(int), cudaMemcpyDeviceToHost, d->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
    const int c = *(int*)(d->hloop + 1);
    d->launches += g.kernels * c;
    if (*(int*)(d->hnorm + 6)) return sulf_fail(SULF_ENOTCONV, "singular coarsest-level Jacobian");
    const double* rn = d->hloop + 4;
    for (int k = 0; k < c && rnorms; k++) rnorms[k] = rn[k];
    const double prev = c >= 2 ? rn[c - 2] : fnorm;
    d->last_rho = prev > 0 ? rn[c - 1] / prev : 0.0;
    return c;
}


// launches of the calling thread use programmatic dependent launch while the
// scope lives
struct PdlScope {
    bool old;
    int old_occ, old_mf;
    explicit PdlScope(bool on, int occ = 0, int mf = 0)
        : old(launch_pdl()), old_occ(launch_occupancy()), old_mf(launch_matrix_free()) {
        set_launch_pdl(on);
        set_launch_occupancy(occ);
        set_launch_matrix_free(mf);
    }
    ~PdlScope() {
        set_launch_pdl(old);
        set_launch_occupancy(old_occ);
        set_launch_matrix_free(old_mf);
    }
};

// run one cycle: replay the captured graph (capturing it first if needed), or
// launch the kernels directly
template <int D>
int run_cycle(sulf_domain* d) {
    int p = d->solver.precision;
    if (!d->solver.graphs) {
        size_t e0 = d->evused;
        int rc = cycle_body<D>(d);
        if (rc) return rc;
        SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
        rc = accumulate_prof(d, e0, d->evused);
        d->evused = e0;
        return rc;
    }
    sulf_domain::CycleGraph& g = d->graph[p];
    // an instantiated graph may be launched on any stream: a new stream alone
    // needs no recapture
    if (!g.exec || g.dt != d->dt || !same_solver(g.sv, d->solver) || g.prof != d->prof) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
        d->evused = 0;
        g.ev0 = 0;
        long long l0 = d->launches;
        SULF_CUDA_TRY(cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal));
        d->capturing = true;
        int rc = cycle_body<D>(d);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamEndCapture(d->stream, &graph);
        d->capturing = false;
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return sulf_fail_cuda(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return sulf_fail_cuda(e, "cudaGraphInstantiate");
        g.kernels = d->launches - l0;
        d->launches = l0;
        g.ev1 = d->evused;
        g.dt = d->dt;
        g.sv = d->solver;
        g.prof = d->prof;
    }
    SULF_CUDA_TRY(cudaGraphLaunch(g.exec, d->stream));
    d->launches += g.kernels;
    SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
    if (d->prof) return accumulate_prof(d, g.ev0, g.ev1);
    return SULF_OK;
}

// Solve J(W) dW = F on the finest level: FP64 cycles, or FP32 cycles on the
// FP64 defect (defect correction).  v64[0].rhs holds F, the result is left in
// v64[0].x.  Returns the number of cycles, or a negative error.
template <int D>
int linear_solve(sulf_domain* d, double fnorm, int max_cycles, double rtol, double* rnorms) {
    const LevelGeo& G0 = d->geo[0];
    SULF_CUDA_TRY(cudaMemsetAsync(d->v64[0].x, 0, sizeof(double2) * G0.nn, d->stream));
    int rc;
    if (d->solver.precision == 0) {
        rc = ensure_tail<D, double>(d, d->v64);
        if (rc) return rc;
        rc = MG<D, double>{d, d->v64}.prepare();
    } else {
        rc = ensure32(d);
        if (rc) return rc;
        rc = ensure_tail<D, float>(d, d->v32);
        if (rc) return rc;
        d->launches += launch_to_float(G0, d->W, d->v32[0].Wc, d->stream);
        // the FP64 defect of the outer iteration needs the FP64 finest-level coefficients
        d->launches += launch_coefs<D, double>(G0, d->v64[0], make_coef<double>(d, 0), d->stream);
        rc = MG<D, float>{d, d->v32}.prepare();
        if (rc) return rc;
        d->launches += launch_to_float(G0, d->v64[0].rhs, d->v32[0].rhs, d->stream);
    }
    if (rc) return rc;
    int c = device_loop<D>(d, fnorm, max_cycles, rtol, rnorms);
    d->loop_used = c > 0;
    if (c) return c;
    double rprev = fnorm;
    int cyc;
    for (cyc = 1; cyc <= max_cycles; cyc++) {
        if (d->solver.cycle == 3 && cyc == 1) {
            // the full-multigrid cycle, launched directly (the cycles after it
            // are V-cycles, replayed from their graph)
            size_t e0 = d->evused;
            d->fmg_now = true;
            rc = cycle_body<D>(d);
            d->fmg_now = false;
            if (rc) return rc;
            SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
            rc = accumulate_prof(d, e0, d->evused);
            d->evused = e0;
        } else {
            rc = run_cycle<D>(d);
        }
        if (rc) return rc;
        if (*(int*)(d->hnorm + 6)) return sulf_fail(SULF_ENOTCONV, "singular coarsest-level Jacobian");
        double rn = bits_to_double(d->hnorm[0]);
        if (rnorms) rnorms[cyc - 1] = rn;
        d->last_rho = rprev > 0 ? rn / rprev : 0.0;
        rprev = rn;
        if (rn <= rtol * fnorm || rn != rn) break;
    }
    return cyc > max_cycles ? max_cycles : cyc;
}

// one Crank-Nicolson step by Newton-Raphson (Sec. 3.4)
template <int D>
int cn_step(sulf_domain* d) {
    const LevelGeo& G0 = d->geo[0];
    LevelVec<double>& V0 = d->v64[0];
    FConst fc = make_fconst(d);
    SULF_CUDA_TRY(cudaMemcpyAsync(d->Wn, d->W, sizeof(double2) * G0.nn, cudaMemcpyDeviceToDevice, d->stream));
    d->launches += launch_old_time<D>(G0, d->Wn, d->G, fc, d->stream);
    SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 4, d->stream));
    d->launches += launch_newton_F<D>(G0, d->W, d->G, V0.rhs, V0.rhsc, fc, d->dnorm, d->stream);
    int rc = read_norms(d, 1);
    if (rc) return rc;
    double fn = bits_to_double(d->hnorm[0]);
    d->newton_last = 0;
    d->cycles_last = 0;
    if (fn < d->solver.newton_tol) {
        d->t += d->dt;
        d->steps_total++;
        d->last_fnorm = fn;
        return SULF_OK;
    }
    for (int k = 1; k <= d->solver.max_newton; k++) {
        int nc = linear_solve<D>(d, fn, d->solver.max_cycles, d->solver.lin_rtol, nullptr);
        if (nc < 0) return nc;
        d->cycles_last += nc;
        d->cycles_total += nc;
        SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 4, d->stream));
        d->launches += launch_newton_update(G0, d->W, V0.x, d->dnorm, d->stream);
        d->launches += launch_newton_F<D>(G0, d->W, d->G, V0.rhs, V0.rhsc, fc, d->dnorm + 2, d->stream);
        rc = read_norms(d, 3);
        if (rc) return rc;
        double dn = bits_to_double(d->hnorm[0]), wn = bits_to_double(d->hnorm[1]);
        fn = bits_to_double(d->hnorm[2]);
        d->newton_last = k;
        d->newton_total++;
        d->last_fnorm = fn;
        if (fn != fn || dn != dn) break;
        double rel = wn > 0 ? dn / wn : dn;
        if ((fn < rel ? fn : rel) < d->solver.newton_tol) {
            d->t += d->dt;
            d->steps_total++;
            return SULF_OK;
        }
    }
    char buf[128];
    snprintf(buf, sizeof buf, "Newton did not converge (|F|_inf = %g)", fn);
    return sulf_fail(SULF_ENOTCONV, buf);
}

bool valid(sulf_handle h) { return h != nullptr; }

// tile lists of the temporally blocked sweep (tiles holding an inside node)
// and the second unknown buffer, for the 3-D levels with enough inside nodes
int ensure_tiles(sulf_domain* d) {
    if (d->dim != 3 || !d->have32) return SULF_OK;
    for (int l = 0; l < d->L; l++) {
        LevelGeo& G = d->geo[l];
        if (G.tiles || (long long)G.nin[0] + G.nin[1] < kTileMinInside) continue;
        std::vector<int8_t> t(G.nn);
        SULF_CUDA_TRY(cudaMemcpyAsync(t.data(), G.type, G.nn, cudaMemcpyDeviceToHost, d->stream));
        SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
        const int tx = 32, ty = 8, tz = 16;  // the kernel's tile (kTileX, kTileY, kTileZ)
        const int nx = (G.n + tx - 1) / tx, ny = (G.n + ty - 1) / ty, nz = (G.n + tz - 1) / tz;
        std::vector<char> has((size_t)nx * ny * nz, 0);
        for (long long p = 0; p < G.nn; p++)
            if (t[p] == T_IN) {
                const int i = (int)(p % G.n), j = (int)((p / G.n) % G.n), k = (int)(p / ((long long)G.n * G.n));
                has[((size_t)(k / tz) * ny + j / ty) * nx + i / tx] = 1;
            }
        std::vector<int> list;
        for (size_t q = 0; q < has.size(); q++)
            if (has[q]) list.push_back((int)q);
        int* dl = (int*)d->mem.get(sizeof(int) * (list.size() + 1));
        float2* x2 = (float2*)d->mem.get(sizeof(float2) * G.nn);
        if (!dl || !x2) return sulf_fail(SULF_ENOMEM, "out of device memory");
        SULF_CUDA_TRY(cudaMemcpyAsync(dl, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, d->stream));
        SULF_CUDA_TRY(cudaMemsetAsync(x2, 0, sizeof(float2) * G.nn, d->stream));
        SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
        G.tiles = dl;
        G.ntiles = (int)list.size();
        G.tile_nx = nx;
        G.tile_ny = ny;
        d->v32[l].x2 = x2;
    }
    return SULF_OK;
}

// wavefront lists of the lexicographic smoother, built once per level on the
// host from the node types: inside nodes ordered by i+j(+k), then box order
int ensure_lex(sulf_domain* d) {
    for (int l = 0; l < d->L; l++) {
        LevelGeo& G = d->geo[l];
        if (G.lex) continue;
        std::vector<int8_t> t(G.nn);
        SULF_CUDA_TRY(cudaMemcpyAsync(t.data(), G.type, G.nn, cudaMemcpyDeviceToHost, d->stream));
        SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
        const int nd = G.dim * (G.n - 1) + 1;
        std::vector<int> ptr(nd + 1, 0), list;
        for (long long p = 0; p < G.nn; p++)
            if (t[p] == T_IN) ptr[p % G.n + (p / G.n) % G.n + p / ((long long)G.n * G.n) + 1]++;
        for (int k = 0; k < nd; k++) ptr[k + 1] += ptr[k];
        list.resize(ptr[nd] > 0 ? ptr[nd] : 1);
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (long long p = 0; p < G.nn; p++)
            if (t[p] == T_IN) list[fill[p % G.n + (p / G.n) % G.n + p / ((long long)G.n * G.n)]++] = (int)p;
        int* dl = (int*)d->mem.get(sizeof(int) * list.size());
        int* dp = (int*)d->mem.get(sizeof(int) * (nd + 1));
        if (!dl || !dp) return sulf_fail(SULF_ENOMEM, "out of device memory");
        SULF_CUDA_TRY(cudaMemcpyAsync(dl, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice, d->stream));
        SULF_CUDA_TRY(cudaMemcpyAsync(dp, ptr.data(), sizeof(int) * (nd + 1), cudaMemcpyHostToDevice, d->stream));
        SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
        G.lex = dl;
        G.lexptr = dp;
        G.nlexd = nd;
    }
    return SULF_OK;
}

int copy_in(sulf_domain* d, void* dst, const void* src, size_t n) {
    SULF_CUDA_TRY(cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, d->stream));
    return SULF_OK;
}

}  // namespace

// read-only views of a handle for entry points defined in other files
namespace sulf {
const LevelGeo* handle_fine_geo(sulf_handle h) { return h ? &h->geo[0] : nullptr; }
const sulf_model* handle_model(sulf_handle h) { return h ? &h->model : nullptr; }
int handle_bc(sulf_handle h) { return h ? h->bc : 0; }
cudaStream_t handle_stream(sulf_handle h) { return h ? h->stream : nullptr; }
void handle_count_launches(sulf_handle h, int n) {
    if (h) h->launches += n;
}
int handle_device(sulf_handle h) { return h ? h->device : -1; }
void** handle_noalloc_slot(sulf_handle h) { return h ? &h->noalloc_scratch : nullptr; }
}  // namespace sulf

// ===========================================================================
// C ABI

extern "C" {

const char* sulf_last_error(void) { return g_err.c_str(); }

void sulf_destroy(sulf_handle h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto& g : h->graph)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : h->evpool) cudaEventDestroy(e);
    h->mem.release();
    if (h->hnorm) cudaFreeHost(h->hnorm);
    if (h->hloop) cudaFreeHost(h->hloop);
    for (auto& g : h->loop)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int sulf_create_domain(const double* levelset, int dim, const double* box, int N, int coarsest_N, sulf_handle* out) {
    if (!out) return sulf_fail(SULF_EINVAL, "out is NULL");
    *out = nullptr;
    if (!levelset || !box || (dim != 2 && dim != 3) || N < 2 || coarsest_N < 2 || !(box[1] > box[0]))
        return sulf_fail(SULF_EINVAL, "invalid arguments");
    int nl = 1, Nl = N;
    while (Nl > coarsest_N && Nl % 2 == 0) {
        Nl /= 2;
        nl++;
    }
    if (Nl != coarsest_N || nl > SULF_MAXLEV) return sulf_fail(SULF_EINVAL, "N must be coarsest_N times a power of two");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return sulf_fail(SULF_EDEVICE, "no CUDA device");
    int cur_dev = 0;
    if (cudaGetDevice(&cur_dev) != cudaSuccess) return sulf_fail(SULF_EDEVICE, "cudaGetDevice failed");
    sulf_domain* d = new sulf_domain();
    d->device = cur_dev;
    d->dim = dim;
    d->N = N;
    d->L = nl;
    d->lo = box[0];
    d->hi = box[1];
    d->model = default_model();
    d->solver = default_solver();
    d->dt = 1.0;
    if (cudaStreamCreateWithFlags(&d->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete d;
        return sulf_fail(SULF_EDEVICE, "cannot create a CUDA stream");
    }
    d->stream = d->own_stream;
    d->mem.stream = d->own_stream;
    std::string err;
    int rc = SULF_OK;
    for (int l = 0; l < nl && rc == SULF_OK; l++) {
        LevelGeo& G = d->geo[l];
        G.dim = dim;
        G.N = N >> l;
        G.n = G.N + 1;
        G.nn = 1;
        for (int a = 0; a < dim; a++) G.nn *= G.n;
        G.st[0] = 1;
        G.st[1] = G.n;
        G.st[2] = dim == 3 ? (long long)G.n * G.n : 0;
        G.lo = box[0];
        G.h = (box[1] - box[0]) / G.N;
        if (l == 0) {
            G.phi = (double*)d->mem.get(sizeof(double) * G.nn);
            if (!G.phi) {
                rc = sulf_fail(SULF_ENOMEM, "out of device memory");
                break;
            }
            if (cudaMemcpyAsync(G.phi, levelset, sizeof(double) * G.nn, cudaMemcpyHostToDevice, d->stream) !=
                cudaSuccess) {
                rc = sulf_fail(SULF_EDEVICE, "level-set upload failed");
                break;
            }
        }
        rc = build_level_geometry(G, l ? &d->geo[l - 1] : nullptr, l == 0, l == nl - 1, d->mem, d->stream, err,
                                  d->launches);
        if (rc) sulf_fail(rc, err);
    }
    if (rc == SULF_OK) rc = alloc_vectors<double>(d, d->v64, false);
    if (rc == SULF_OK) {
        long long nn = d->geo[0].nn;
        d->W = d->v64[0].Wc;
        d->Wn = (double2*)d->mem.get(sizeof(double2) * nn);
        d->G = (double2*)d->mem.get(sizeof(double2) * nn);
        d->dnorm = (unsigned long long*)d->mem.get(sizeof(unsigned long long) * 8);
        d->dsing = (int*)d->mem.get(sizeof(int) * 2);
        d->stage = (double*)d->mem.get(sizeof(double) * 2 * nn + nn + 16);
        if (!d->Wn || !d->G || !d->dnorm || !d->dsing || !d->stage)
            rc = sulf_fail(SULF_ENOMEM, "out of device memory");
        else if (cudaMallocHost(&d->hnorm, sizeof(unsigned long long) * 8) != cudaSuccess)
            rc = sulf_fail(SULF_ENOMEM, "out of pinned host memory");
        else {
            cudaMemsetAsync(d->Wn, 0, sizeof(double2) * nn, d->stream);
            cudaMemsetAsync(d->G, 0, sizeof(double2) * nn, d->stream);
            d->launches += launch_reset_state(d->geo[0], d->W, d->model.s0, d->model.c0, d->stream);
            if (cudaStreamSynchronize(d->stream) != cudaSuccess) rc = sulf_fail(SULF_EDEVICE, "initialisation failed");
        }
    }
    if (rc == SULF_OK) rc = refresh_ghost_ops(d);
    if (rc != SULF_OK) {
        std::string keep = g_err;
        sulf_destroy(d);
        g_err = keep;
        return rc;
    }
    *out = d;
    return SULF_OK;
}

int sulf_set_model(sulf_handle h, const sulf_model* m) {
    if (!valid(h) || !m) return sulf_fail(SULF_EINVAL, "invalid arguments");
    if (!(m->d >= 0) || !(m->m_s > 0) || !(m->m_c > 0)) return sulf_fail(SULF_EINVAL, "invalid model parameters");
    h->model = *m;
    h->t = 0;
    h->launches += launch_reset_state(h->geo[0], h->W, m->s0, m->c0, h->stream);
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SULF_OK;
}

int sulf_set_solver(sulf_handle h, const sulf_solver* s) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    sulf_solver v = s ? *s : default_solver();
    if (v.nu1 < 0 || v.nu2 < 0 || v.nu1 + v.nu2 < 1 || v.cycle < 1 || v.cycle > 3 || v.max_newton < 1 ||
        v.max_cycles < 1 || v.ghost_sweeps < 1 || !(v.tau_s > 0 && v.tau_s < 1) || !(v.newton_tol > 0) ||
        !(v.lin_rtol > 0) || (v.precision != 0 && v.precision != 1) || v.smoother < 0 || v.smoother > 2 ||
        (v.graphs != 0 && v.graphs != 1) || v.fuse_below < -1 ||
        (v.pdl != 0 && v.pdl != 1) || (v.ghost_compose != 0 && v.ghost_compose != 1) ||
        (v.relax_occupancy != 0 && v.relax_occupancy != 1) || v.relax_matrix_free < 0 || v.relax_matrix_free > 2)
        return sulf_fail(SULF_EINVAL, "solver controls out of range");
    h->solver = v;
    if (int rc = refresh_ghost_ops(h)) return rc;
    if (v.smoother == 2)
        if (int rc = ensure_lex(h)) return rc;
    if (v.precision == 1) {
        if (int rc = ensure32(h)) return rc;
        if (v.relax_matrix_free == 2) return ensure_tiles(h);
    }
    return SULF_OK;
}

int sulf_set_stream(sulf_handle h, void* stream) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    // every call returns with the handle's device work complete, so the old
    // stream needs no synchronisation (it may belong to another thread that is
    // capturing a graph on it right now)
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return SULF_OK;
}

int sulf_step(sulf_handle h, double dt, int nsteps) {
    if (!valid(h) || !(dt > 0) || nsteps < 0) return sulf_fail(SULF_EINVAL, "invalid arguments");
    h->dt = dt;
    PdlScope pdl(h->solver.pdl != 0, h->solver.relax_occupancy, h->solver.relax_matrix_free);
    for (int k = 0; k < nsteps; k++) {
        int rc = h->dim == 2 ? cn_step<2>(h) : cn_step<3>(h);
        if (rc) {
            cudaStreamSynchronize(h->stream);  // leave no work in flight
            return rc;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sulf_fail_cuda(e, "kernel launch");
    return SULF_OK;
}

int sulf_get_state_device(sulf_handle h, double* s_dev, double* c_dev) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    h->launches += launch_export_state(h->geo[0], h->W, s_dev, c_dev, nullptr, h->stream);
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SULF_OK;
}

int sulf_get_state(sulf_handle h, double* s, double* c, int8_t* type) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    long long nn = h->geo[0].nn;
    double* ds = h->stage;
    double* dc = h->stage + nn;
    int8_t* dt = (int8_t*)(h->stage + 2 * nn);
    h->launches += launch_export_state(h->geo[0], h->W, ds, dc, dt, h->stream);
    if (s) SULF_CUDA_TRY(cudaMemcpyAsync(s, ds, sizeof(double) * nn, cudaMemcpyDeviceToHost, h->stream));
    if (c) SULF_CUDA_TRY(cudaMemcpyAsync(c, dc, sizeof(double) * nn, cudaMemcpyDeviceToHost, h->stream));
    if (type) SULF_CUDA_TRY(cudaMemcpyAsync(type, dt, nn, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SULF_OK;
}

int sulf_set_state_device(sulf_handle h, const double* s_dev, const double* c_dev, double t) {
    if (!valid(h) || !s_dev || !c_dev) return sulf_fail(SULF_EINVAL, "invalid arguments");
    h->launches += launch_import_state(h->geo[0], h->W, s_dev, c_dev, h->stream);
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->t = t;
    return SULF_OK;
}

int sulf_set_state_extrapolated(sulf_handle h, const double* s, const double* c, double t) {
    if (!valid(h) || !s || !c) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G0 = h->geo[0];
    const long long nn = G0.nn;
    if (!h->xbuf) h->xbuf = (double*)h->mem.get(sizeof(double) * 5 * nn);
    if (!h->xbuf) return sulf_fail(SULF_ENOMEM, "out of device memory");
    double *us = h->xbuf, *uc = h->xbuf + nn, *q = h->xbuf + 2 * nn, *q2 = h->xbuf + 3 * nn, *u2 = h->xbuf + 4 * nn;
    SULF_CUDA_TRY(cudaMemcpyAsync(us, s, sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(uc, c, sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
    h->launches += launch_extrapolate(G0, us, q, q2, u2, kExtrapolationIters, h->stream);
    h->launches += launch_extrapolate(G0, uc, q, q2, u2, kExtrapolationIters, h->stream);
    h->launches += launch_import_state(G0, h->W, us, uc, h->stream);
    SULF_CUDA_TRY(cudaGetLastError());
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->t = t;
    return SULF_OK;
}

int sulf_set_state(sulf_handle h, const double* s, const double* c, double t) {
    if (!valid(h) || !s || !c) return sulf_fail(SULF_EINVAL, "invalid arguments");
    long long nn = h->geo[0].nn;
    SULF_CUDA_TRY(cudaMemcpyAsync(h->stage, s, sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(h->stage + nn, c, sizeof(double) * nn, cudaMemcpyHostToDevice, h->stream));
    return sulf_set_state_device(h, h->stage, h->stage + nn, t);
}

int sulf_set_bc(sulf_handle h, int type) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    if (type != 0 && type != 1) return sulf_fail(SULF_EINVAL, "boundary condition must be 0 (Dirichlet) or 1 (Neumann)");
    if (type == h->bc) return SULF_OK;
    std::string err;
    for (int l = 0; l < h->L; l++) {
        int rc = build_ghost_rows(h->geo[l], type, l == 0, h->stream, err, h->launches);
        if (rc) {
            // put the previous rows back
            std::string ignore;
            for (int k = 0; k <= l; k++) build_ghost_rows(h->geo[k], h->bc, k == 0, h->stream, ignore, h->launches);
            return sulf_fail(rc, err);
        }
    }
    h->bc = type;
    // the captured cycles bake the relaxation parameter and the fused kernel's
    // boundary condition: capture them again
    drop_graphs(h);
    return refresh_ghost_ops(h);
}

int sulf_set_sources(sulf_handle h, const double* f1_old, const double* f1_new, const double* f2_old,
                     const double* f2_new) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    const int given = (f1_old != nullptr) + (f1_new != nullptr) + (f2_old != nullptr) + (f2_new != nullptr);
    if (given == 0) {
        h->src_on = false;
        return SULF_OK;
    }
    if (given != 4) return sulf_fail(SULF_EINVAL, "give all four source arrays or none");
    const long long nn = h->geo[0].nn;
    if (!h->src) h->src = (double2*)h->mem.get(sizeof(double2) * nn);
    if (!h->src_stage) h->src_stage = (double*)h->mem.get(sizeof(double) * 4 * nn);
    if (!h->src || !h->src_stage) return sulf_fail(SULF_ENOMEM, "out of device memory");
    const double* in[4] = {f1_old, f1_new, f2_old, f2_new};
    for (int k = 0; k < 4; k++)
        SULF_CUDA_TRY(cudaMemcpyAsync(h->src_stage + k * nn, in[k], sizeof(double) * nn, cudaMemcpyHostToDevice,
                                      h->stream));
    h->launches += launch_average_sources(nn, h->src_stage, h->src, h->stream);
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->src_on = true;
    return SULF_OK;
}

int sulf_set_ghost_values(sulf_handle h, const double* sb) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    if (!sb) {
        h->sbg_on = false;
        return SULF_OK;
    }
    const int ng = h->geo[0].ng;
    if (!h->sbg) h->sbg = (double*)h->mem.get(sizeof(double) * (ng + 1));
    if (!h->sbg) return sulf_fail(SULF_ENOMEM, "out of device memory");
    SULF_CUDA_TRY(cudaMemcpyAsync(h->sbg, sb, sizeof(double) * ng, cudaMemcpyHostToDevice, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->sbg_on = true;
    return SULF_OK;
}

int sulf_get_stats(sulf_handle h, sulf_stats* o) {
    if (!valid(h) || !o) return sulf_fail(SULF_EINVAL, "invalid arguments");
    o->t = h->t;
    o->newton_last = h->newton_last;
    o->cycles_last = h->cycles_last;
    o->newton_total = h->newton_total;
    o->cycles_total = h->cycles_total;
    o->steps_total = h->steps_total;
    o->last_rho = h->last_rho;
    o->last_fnorm = h->last_fnorm;
    o->kernel_launches = h->launches;
    o->levels = h->L;
    o->n_inside = h->geo[0].nin[0] + (long long)h->geo[0].nin[1];
    o->n_ghost = h->geo[0].ng;
    for (int k = 0; k < 3; k++) o->ghost_rows[k] = h->geo[0].kinds[k];
    o->device_bytes = h->mem.bytes;
    o->loop_graph = h->loop_used ? 1 : 0;
    return SULF_OK;
}

int sulf_set_profiling(sulf_handle h, int on) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (on < 0 || on > 2) return sulf_fail(SULF_EINVAL, "profiling mode must be 0, 1 or 2");
    h->prof = on;
    h->prof_ms = 0;
    h->prof_n = 0;
    return SULF_OK;
}

int sulf_kernel_time(sulf_handle h, double* ms, long long* launches) {
    if (!valid(h)) return sulf_fail(SULF_EINVAL, "invalid handle");
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (ms) *ms = h->prof_ms;
    if (launches) *launches = h->prof_n;
    h->prof_ms = 0;
    h->prof_n = 0;
    return SULF_OK;
}

// ---------------------------------------------------------------------------
// stage-level entry points (sulfmg_debug.h)

static int dbg_level_ok(sulf_handle h, int l) { return valid(h) && l >= 0 && l < h->L; }

int sulf_dbg_level_info(sulf_handle h, int l, int64_t* info) {
    if (!dbg_level_ok(h, l) || !info) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    info[0] = G.N;
    info[1] = G.n;
    info[2] = G.ng;
    info[3] = G.nb;
    info[4] = l == h->L - 1 ? G.nact : 0;
    info[5] = G.nin[0] + (int64_t)G.nin[1];
    for (int k = 0; k < 3; k++) info[6 + k] = G.kinds[k];
    info[9] = G.gop_on ? G.gop_nnz : -1;
    info[10] = G.gop_on ? G.gop_passes : 0;
    return SULF_OK;
}

int sulf_dbg_level_type(sulf_handle h, int l, int8_t* type) {
    if (!dbg_level_ok(h, l) || !type) return sulf_fail(SULF_EINVAL, "invalid arguments");
    SULF_CUDA_TRY(cudaMemcpyAsync(type, h->geo[l].type, h->geo[l].nn, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SULF_OK;
}

int sulf_dbg_level_ghosts(sulf_handle h, int l, int64_t* idx, int8_t* kind, int8_t* m, double* w, double* B) {
    if (!dbg_level_ok(h, l)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    int D = G.dim;
    std::vector<int> tmp(G.ng + 1);
    SULF_CUDA_TRY(cudaMemcpyAsync(tmp.data(), G.gidx, sizeof(int) * G.ng, cudaMemcpyDeviceToHost, h->stream));
    if (kind) SULF_CUDA_TRY(cudaMemcpyAsync(kind, G.gkind, G.ng, cudaMemcpyDeviceToHost, h->stream));
    if (m) SULF_CUDA_TRY(cudaMemcpyAsync(m, G.gm, (size_t)G.ng * D, cudaMemcpyDeviceToHost, h->stream));
    if (w) SULF_CUDA_TRY(cudaMemcpyAsync(w, G.gw, sizeof(double) * G.ng * D * 3, cudaMemcpyDeviceToHost, h->stream));
    if (B) SULF_CUDA_TRY(cudaMemcpyAsync(B, G.gB, sizeof(double) * G.ng * D, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (idx)
        for (int k = 0; k < G.ng; k++) idx[k] = tmp[k];
    return SULF_OK;
}

int sulf_dbg_level_rows(sulf_handle h, int l, double* wk, double* nt) {
    if (!dbg_level_ok(h, l)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    const int D = G.dim, K = D == 2 ? 9 : 27;
    if (wk) {
        std::vector<double> t((size_t)K * G.ng + 1);
        SULF_CUDA_TRY(cudaMemcpyAsync(t.data(), G.gwk, sizeof(double) * K * G.ng, cudaMemcpyDeviceToHost, h->stream));
        SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
        for (int gi = 0; gi < G.ng; gi++)
            for (int kk = 0; kk < K; kk++) wk[(size_t)gi * K + kk] = t[(size_t)kk * G.ng + gi];
    }
    if (nt) SULF_CUDA_TRY(cudaMemcpyAsync(nt, G.gnt, sizeof(double) * G.ng * D, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    return SULF_OK;
}

// copy a level vector to the host, zero outside the nodes whose type is in mask
static int dbg_copy_out(sulf_handle h, int l, const double2* src, double* dst, bool with_band) {
    const LevelGeo& G = h->geo[l];
    std::vector<int8_t> ty(G.nn);
    SULF_CUDA_TRY(cudaMemcpyAsync(dst, src, sizeof(double2) * G.nn, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaMemcpyAsync(ty.data(), G.type, G.nn, cudaMemcpyDeviceToHost, h->stream));
    SULF_CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (long long i = 0; i < G.nn; i++) {
        bool keep = ty[i] == T_IN || ty[i] == T_GHOST || (with_band && ty[i] == T_BAND);
        if (!keep) dst[2 * i] = dst[2 * i + 1] = 0.0;
    }
    return SULF_OK;
}

int sulf_dbg_eval_F(sulf_handle h, double dt, const double* W, const double* Wn, double* F) {
    if (!valid(h) || !W || !Wn || !F || !(dt > 0)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G0 = h->geo[0];
    h->dt = dt;
    int rc = copy_in(h, h->W, W, sizeof(double2) * G0.nn);
    if (!rc) rc = copy_in(h, h->Wn, Wn, sizeof(double2) * G0.nn);
    if (rc) return rc;
    FConst fc = make_fconst(h);
    SULF_CUDA_TRY(cudaMemsetAsync(h->dnorm, 0, 8, h->stream));
    if (h->dim == 2) {
        h->launches += launch_old_time<2>(G0, h->Wn, h->G, fc, h->stream);
        h->launches += launch_newton_F<2>(G0, h->W, h->G, h->v64[0].rhs, h->v64[0].rhsc, fc, h->dnorm, h->stream);
    } else {
        h->launches += launch_old_time<3>(G0, h->Wn, h->G, fc, h->stream);
        h->launches += launch_newton_F<3>(G0, h->W, h->G, h->v64[0].rhs, h->v64[0].rhsc, fc, h->dnorm, h->stream);
    }
    return dbg_copy_out(h, 0, h->v64[0].rhs, F, false);
}

int sulf_dbg_apply_J(sulf_handle h, int l, double dt, const double* Wc, const double* x, double* out) {
    if (!dbg_level_ok(h, l) || !Wc || !x || !out || !(dt > 0)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    LevelVec<double>& V = h->v64[l];
    h->dt = dt;
    int rc = copy_in(h, V.Wc, Wc, sizeof(double2) * G.nn);
    if (!rc) rc = copy_in(h, V.x, x, sizeof(double2) * G.nn);
    if (rc) return rc;
    SULF_CUDA_TRY(cudaMemsetAsync(V.rhs, 0, sizeof(double2) * G.nn, h->stream));
    h->launches += launch_gather_list(G, V.rhs, V.rhsc, h->stream);
    if (h->dim == 2) {
        h->launches += launch_coefs<2, double>(G, V, make_coef<double>(h, l), h->stream);
        h->launches += launch_residual<2, double>(G, V, make_coef<double>(h, l), nullptr, h->stream);
    } else {
        h->launches += launch_coefs<3, double>(G, V, make_coef<double>(h, l), h->stream);
        h->launches += launch_residual<3, double>(G, V, make_coef<double>(h, l), nullptr, h->stream);
    }
    rc = dbg_copy_out(h, l, V.res, out, false);
    if (rc) return rc;
    for (long long i = 0; i < 2 * G.nn; i++) out[i] = -out[i] + 0.0;
    return SULF_OK;
}

int sulf_dbg_smooth(sulf_handle h, int l, double dt, const double* Wc, const double* rhs, double* x, int sweeps) {
    if (!dbg_level_ok(h, l) || !Wc || !rhs || !x || !(dt > 0) || sweeps < 0)
        return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    LevelVec<double>& V = h->v64[l];
    h->dt = dt;
    int rc = copy_in(h, V.Wc, Wc, sizeof(double2) * G.nn);
    if (!rc) rc = copy_in(h, V.rhs, rhs, sizeof(double2) * G.nn);
    if (!rc) h->launches += launch_gather_list(G, V.rhs, V.rhsc, h->stream);
    if (!rc) rc = copy_in(h, V.x, x, sizeof(double2) * G.nn);
    if (rc) return rc;
    if (h->dim == 2)
        h->launches += launch_coefs<2, double>(G, V, make_coef<double>(h, l), h->stream);
    else
        h->launches += launch_coefs<3, double>(G, V, make_coef<double>(h, l), h->stream);
    for (int k = 0; k < sweeps; k++) {
        if (h->dim == 2)
            MG<2, double>{h, h->v64}.relax(l);
        else
            MG<3, double>{h, h->v64}.relax(l);
    }
    return dbg_copy_out(h, l, V.x, x, false);
}

int sulf_dbg_restrict(sulf_handle h, int l, double* res, double* rhs_coarse) {
    if (!valid(h) || l < 0 || l + 1 >= h->L || !res || !rhs_coarse) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G = h->geo[l];
    int rc = copy_in(h, h->v64[l].res, res, sizeof(double2) * G.nn);
    if (rc) return rc;
    if (h->dim == 2) {
        h->launches += launch_extend<2, double>(G, h->v64[l], h->stream);
        h->launches += launch_restrict<2, double>(G, h->v64[l], h->geo[l + 1], h->v64[l + 1], false, false, h->stream);
    } else {
        h->launches += launch_extend<3, double>(G, h->v64[l], h->stream);
        h->launches += launch_restrict<3, double>(G, h->v64[l], h->geo[l + 1], h->v64[l + 1], false, false, h->stream);
    }
    rc = dbg_copy_out(h, l, h->v64[l].res, res, true);
    if (rc) return rc;
    return dbg_copy_out(h, l + 1, h->v64[l + 1].rhs, rhs_coarse, false);
}

int sulf_dbg_prolong(sulf_handle h, int l, const double* xc, double* xf) {
    if (!valid(h) || l < 0 || l + 1 >= h->L || !xc || !xf) return sulf_fail(SULF_EINVAL, "invalid arguments");
    int rc = copy_in(h, h->v64[l + 1].x, xc, sizeof(double2) * h->geo[l + 1].nn);
    if (!rc) rc = copy_in(h, h->v64[l].x, xf, sizeof(double2) * h->geo[l].nn);
    if (rc) return rc;
    if (h->dim == 2)
        h->launches += launch_prolong<2, double>(h->geo[l], h->v64[l], h->geo[l + 1], h->v64[l + 1], h->stream);
    else
        h->launches += launch_prolong<3, double>(h->geo[l], h->v64[l], h->geo[l + 1], h->v64[l + 1], h->stream);
    return dbg_copy_out(h, l, h->v64[l].x, xf, false);
}

int sulf_dbg_inject(sulf_handle h, const double* Wc0, int l, double* Wc_out) {
    if (!dbg_level_ok(h, l) || !Wc0 || !Wc_out) return sulf_fail(SULF_EINVAL, "invalid arguments");
    int rc = copy_in(h, h->v64[0].Wc, Wc0, sizeof(double2) * h->geo[0].nn);
    if (rc) return rc;
    for (int k = 1; k <= l; k++) {
        if (h->dim == 2)
            h->launches += launch_inject<2, double>(h->geo[k - 1], h->v64[k - 1], h->geo[k], h->v64[k], h->stream);
        else
            h->launches += launch_inject<3, double>(h->geo[k - 1], h->v64[k - 1], h->geo[k], h->v64[k], h->stream);
    }
    return dbg_copy_out(h, l, h->v64[l].Wc, Wc_out, false);
}

int sulf_dbg_coarsest_solve(sulf_handle h, double dt, const double* Wc0, const double* rhs_c, double* x_c) {
    if (!valid(h) || !Wc0 || !rhs_c || !x_c || !(dt > 0)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    h->dt = dt;
    int lc = h->L - 1;
    int rc = copy_in(h, h->W, Wc0, sizeof(double2) * h->geo[0].nn);
    if (rc) return rc;
    rc = h->dim == 2 ? MG<2, double>{h, h->v64}.prepare() : MG<3, double>{h, h->v64}.prepare();
    if (rc) return rc;
    rc = copy_in(h, h->v64[lc].rhs, rhs_c, sizeof(double2) * h->geo[lc].nn);
    if (!rc) h->launches += launch_gather_list(h->geo[lc], h->v64[lc].rhs, h->v64[lc].rhsc, h->stream);
    if (rc) return rc;
    if (h->dim == 2)
        h->launches += launch_coarsest_solve<2, double>(h->geo[lc], h->v64[lc], h->stream);
    else
        h->launches += launch_coarsest_solve<3, double>(h->geo[lc], h->v64[lc], h->stream);
    return dbg_copy_out(h, lc, h->v64[lc].x, x_c, false);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lock-step batching: K domains of one size class advance their Newton
// iterations and multigrid cycles in lock step, each phase of a cycle one
// launch over all instances' work lists (lockstep.cu); an instance leaves a
// linear solve (or the Newton loop) when its own test says so and is masked
// from then on, so every instance runs the iterations and cycles it runs
// alone.  The Newton-level steps (old-time part, residual F, update, the
// coefficients and the coarsest inverse of each Newton iteration) run per
// instance, on up to eight forked branches of the class's stream.  Each
// phase of a step (its start, a Newton iteration's set-up, a cycle, a Newton
// update) is captured once as a CUDA graph and replayed.
namespace {

constexpr int kBatchT = 256;
constexpr int kLockMaxCoarsest = 2048;  // coarsest active nodes (32 KB of FP64 right-hand side)

template <int D, typename T>
BLev<D, T> blev_of(sulf_domain* d, LevelVec<T>* V, int l) {
    const LevelGeo& G = d->geo[l];
    LevelVec<T>& v = V[l];
    BLev<D, T> b;
    b.ls = stages::make_lists(G);
    b.tb = stages::ghost_tab<T>(G);
    b.cf = stages::coef_ptr<D, T>(v);
    b.c = make_coef<T>(d, l);
    b.Wc = v.Wc;
    b.rhs = v.rhs;
    b.rhsc = v.rhsc;
    b.x = v.x;
    b.res = v.res;
    b.type = G.type;
    b.n = G.n;
    b.st1 = G.st[1];
    b.st2 = G.st[2];
    b.gop_ptr = G.gop_ptr;
    b.gop_code = G.gop_code;
    b.gop_val = std::is_same<T, float>::value ? (const T*)G.gop_val32 : (const T*)G.gop_val;
    b.gc = v.gc;
    b.gci = v.gci;
    b.snap = v.gbuf[0];
    b.nb = G.nb;
    b.eptr = G.eptr;
    b.eidx = G.eidx;
    b.bidx = G.bidx;
    b.eval = std::is_same<T, float>::value ? (const T*)G.eval32 : (const T*)G.eval;
    b.nact = G.nact;
    b.act = G.act;
    b.Ainv = v.Ainv;
    return b;
}

// device and pinned host memory of one lock-step call, released at its end
struct Scratch {
    std::vector<void*> p, ph;
    cudaStream_t s;
    void* get(size_t n) {
        void* q = nullptr;
        if (cudaMallocAsync(&q, n < 256 ? 256 : n, s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        p.push_back(q);
        return q;
    }
    void* get_host(size_t n) {
        void* q = nullptr;
        if (cudaMallocHost(&q, n < 256 ? 256 : n) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ph.push_back(q);
        return q;
    }
    ~Scratch() {
        cudaStreamSynchronize(s);
        for (void* q : p) cudaFreeAsync(q, s);
        cudaStreamSynchronize(s);
        for (void* q : ph) cudaFreeHost(q);
    }
};

// One phase of a lock-step step (its work enqueued by a function on the
// class's stream), replayed from a CUDA graph captured at its first run: the
// kernel parameters of every phase are fixed for the whole call (pointers,
// dt, the models), only device data changes between runs.  The launch
// counts of the captured run are added again at every replay.
struct PhaseGraph {
    cudaGraphExec_t exec = nullptr;
    bool failed = false;
    long long dclass = 0;
    std::vector<long long> dinst;
    ~PhaseGraph() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

// CTA prefix over instances (pre[i] = CTAs of instances < i), uploaded
struct Blocks {
    const int* d = nullptr;
    int total = 0;
};

template <int D>
struct LockClass {
    std::vector<sulf_domain*> h;
    int K = 0, L = 0;
    cudaStream_t s = nullptr;
    Scratch* mem = nullptr;
    const BLev<D, double>* l64[SULF_MAXLEV] = {};
    const BLev<D, float>* l32[SULF_MAXLEV] = {};
    Blocks red[SULF_MAXLEV], black[SULF_MAXLEV], gop[SULF_MAXLEV], act[SULF_MAXLEV], ext[SULF_MAXLEV], coarse;
    int max_nact = 0;
    int* dactive = nullptr;
    std::vector<int> active;
    unsigned long long* dnorm = nullptr;
    unsigned long long* hnorm = nullptr;  // pinned
    long long launches = 0;
    bool graphs = true;
    // the fused coarse levels ltail .. L-1 (-1: none), one CTA per instance:
    // the instances' descriptors (device array) and level geometry
    int ltail = -1;
    const void* const* dtail = nullptr;
    std::vector<const LevelGeo*> geos;
    // branches of the per-instance phases (instance i on aux[i % naux])
    static constexpr int kMaxAux = 8;
    cudaStream_t aux[kMaxAux] = {};
    cudaEvent_t ev_fork = nullptr, ev_join[kMaxAux] = {};
    int naux = 0;

    ~LockClass() {
        for (int j = 0; j < naux; j++) {
            if (aux[j]) cudaStreamDestroy(aux[j]);
            if (ev_join[j]) cudaEventDestroy(ev_join[j]);
        }
        if (ev_fork) cudaEventDestroy(ev_fork);
    }

    // fn(i, stream) for every instance, on parallel branches joined back
    // into the class's stream (each handle's stream is the branch's meanwhile)
    template <class F>
    int per_instance(F&& fn) {
        SULF_CUDA_TRY(cudaEventRecord(ev_fork, s));
        for (int j = 0; j < naux; j++) SULF_CUDA_TRY(cudaStreamWaitEvent(aux[j], ev_fork, 0));
        int rc = SULF_OK;
        for (int i = 0; i < K && rc == SULF_OK; i++) {
            cudaStream_t b = aux[i % naux];
            h[i]->stream = b;
            rc = fn(i, b);
            h[i]->stream = s;
        }
        for (int j = 0; j < naux; j++) {
            SULF_CUDA_TRY(cudaEventRecord(ev_join[j], aux[j]));
            SULF_CUDA_TRY(cudaStreamWaitEvent(s, ev_join[j], 0));
        }
        return rc;
    }

    // run phase fn: replay its graph, or capture it (falling back to direct
    // launches where capture fails), then wait for it
    template <class F>
    int run_phase(PhaseGraph& g, F&& fn) {
        if (g.exec) {
            SULF_CUDA_TRY(cudaGraphLaunch(g.exec, s));
            launches += g.dclass;
            for (int i = 0; i < K; i++) h[i]->launches += g.dinst[i];
        } else {
            const long long c0 = launches;
            std::vector<long long> i0(K);
            for (int i = 0; i < K; i++) i0[i] = h[i]->launches;
            bool done = false;
            if (graphs && !g.failed && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                int rc = fn();
                cudaGraph_t gr = nullptr;
                cudaError_t e = cudaStreamEndCapture(s, &gr);
                if (rc == SULF_OK && e == cudaSuccess && gr && take_launch_error().empty() &&
                    cudaGraphInstantiate(&g.exec, gr, 0) == cudaSuccess) {
                    g.dclass = launches - c0;
                    g.dinst.resize(K);
                    for (int i = 0; i < K; i++) g.dinst[i] = h[i]->launches - i0[i];
                    done = cudaGraphLaunch(g.exec, s) == cudaSuccess;
                }
                if (gr) cudaGraphDestroy(gr);
                if (!done) {
                    if (g.exec) cudaGraphExecDestroy(g.exec);
                    g.exec = nullptr;
                    g.failed = true;
                    cudaGetLastError();
                    take_launch_error();
                    launches = c0;
                    for (int i = 0; i < K; i++) h[i]->launches = i0[i];
                }
            }
            if (!done)
                if (int rc = fn()) return rc;
        }
        SULF_CUDA_TRY(cudaStreamSynchronize(s));
        std::string e = take_launch_error();
        if (!e.empty()) return sulf_fail(SULF_EDEVICE, "lock-step launch failed: " + e);
        return SULF_OK;
    }

    int upload_blocks(Blocks& b, const std::vector<long long>& units, int per_cta) {
        std::vector<int> pre(K + 1, 0);
        for (int i = 0; i < K; i++) pre[i + 1] = pre[i] + (int)((units[i] + per_cta - 1) / per_cta);
        int* dp = (int*)mem->get(sizeof(int) * (K + 1));
        if (!dp) return sulf_fail(SULF_ENOMEM, "out of device memory");
        SULF_CUDA_TRY(cudaMemcpyAsync(dp, pre.data(), sizeof(int) * (K + 1), cudaMemcpyHostToDevice, s));
        b.d = dp;
        b.total = pre[K];
        return SULF_OK;
    }

    template <typename T>
    int upload_levels(LevelVec<T>* (*vec)(sulf_domain*), const BLev<D, T>** out) {
        for (int l = 0; l < L; l++) {
            std::vector<BLev<D, T>> v(K);
            for (int i = 0; i < K; i++) v[i] = blev_of<D, T>(h[i], vec(h[i]), l);
            BLev<D, T>* dv = (BLev<D, T>*)mem->get(sizeof(BLev<D, T>) * K);
            if (!dv) return sulf_fail(SULF_ENOMEM, "out of device memory");
            SULF_CUDA_TRY(cudaMemcpyAsync(dv, v.data(), sizeof(BLev<D, T>) * K, cudaMemcpyHostToDevice, s));
            SULF_CUDA_TRY(cudaStreamSynchronize(s));  // the host vector goes out of scope
            out[l] = dv;
        }
        return SULF_OK;
    }

    int setup() {
        const bool mixed = h[0]->solver.precision == 1;
        if (int rc = upload_levels<double>([](sulf_domain* d) { return d->v64; }, l64)) return rc;
        if (mixed)
            if (int rc = upload_levels<float>([](sulf_domain* d) { return d->v32; }, l32)) return rc;
        for (int l = 0; l < L; l++) {
            std::vector<long long> r(K), b(K), g(K), a(K), e(K);
            for (int i = 0; i < K; i++) {
                const LevelGeo& G = h[i]->geo[l];
                r[i] = G.nin[0];
                b[i] = G.nin[1] > G.ng ? G.nin[1] : G.ng;
                g[i] = (long long)G.ng * stages::kGopLanes;
                a[i] = (long long)G.nin[0] + G.nin[1] + G.ng;
                e[i] = G.nb;
            }
            if (int rc = upload_blocks(red[l], r, kBatchT)) return rc;
            if (int rc = upload_blocks(black[l], b, kBatchT)) return rc;
            if (int rc = upload_blocks(gop[l], g, kBatchT)) return rc;
            if (int rc = upload_blocks(act[l], a, kBatchT)) return rc;
            if (int rc = upload_blocks(ext[l], e, kBatchT)) return rc;
        }
        std::vector<long long> rows(K);
        for (int i = 0; i < K; i++) {
            rows[i] = 2LL * h[i]->geo[L - 1].nact;
            max_nact = std::max(max_nact, h[i]->geo[L - 1].nact);
        }
        if (int rc = upload_blocks(coarse, rows, kBatchT / 32)) return rc;
        dactive = (int*)mem->get(sizeof(int) * K);
        dnorm = (unsigned long long*)mem->get(sizeof(unsigned long long) * K);
        hnorm = (unsigned long long*)mem->get_host(sizeof(unsigned long long) * K);
        if (!dactive || !dnorm || !hnorm) return sulf_fail(SULF_ENOMEM, "out of memory");
        active.assign(K, 0);
        SULF_CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        naux = std::min(K, kMaxAux);
        for (int j = 0; j < naux; j++) {
            SULF_CUDA_TRY(cudaStreamCreateWithFlags(&aux[j], cudaStreamNonBlocking));
            SULF_CUDA_TRY(cudaEventCreateWithFlags(&ev_join[j], cudaEventDisableTiming));
        }
        graphs = h[0]->solver.graphs != 0;
        // the fused coarse levels: from the first level that every
        // instance's threshold fuses
        for (int i = 0; i < K; i++) {
            const int t = tail_level(h[i]);
            if (t < 0) {
                ltail = -1;
                break;
            }
            ltail = std::max(ltail, t);
        }
        if (ltail >= 0) {
            std::vector<const void*> dd(K);
            for (int i = 0; i < K; i++) {
                sulf_domain* d = h[i];
                int rc = mixed ? ensure_tail<D, float>(d, d->v32) : ensure_tail<D, double>(d, d->v64);
                if (rc) return rc;
                dd[i] = d->tail_desc[mixed ? 1 : 0];
                geos.push_back(d->geo);
            }
            void* p = mem->get(sizeof(void*) * K);
            if (!p) return sulf_fail(SULF_ENOMEM, "out of device memory");
            SULF_CUDA_TRY(cudaMemcpyAsync(p, dd.data(), sizeof(void*) * K, cudaMemcpyHostToDevice, s));
            SULF_CUDA_TRY(cudaStreamSynchronize(s));
            dtail = (const void* const*)p;
        }
        SULF_CUDA_TRY(cudaStreamSynchronize(s));
        return SULF_OK;
    }

    int set_active() {
        SULF_CUDA_TRY(cudaMemcpyAsync(dactive, active.data(), sizeof(int) * K, cudaMemcpyHostToDevice, s));
        SULF_CUDA_TRY(cudaStreamSynchronize(s));
        return SULF_OK;
    }

    template <typename T>
    void relax(const BLev<D, T>* const* lv, int l) {
        // FP32: coefficients formed from Wc where the solver asks for it
        const BPhase ph = std::is_same<T, float>::value && h[0]->solver.relax_matrix_free ? BPhase::relax_mf
                                                                                          : BPhase::relax;
        launches += launch_batched<D, T>(ph, lv[l], nullptr, red[l].d, red[l].total, K, dactive, 0, nullptr, 0, s);
        launches += launch_batched<D, T>(ph, lv[l], nullptr, black[l].d, black[l].total, K, dactive, 1, nullptr, 0,
                                         s);
        launches += launch_batched<D, T>(BPhase::ghost_op, lv[l], nullptr, gop[l].d, gop[l].total, K, dactive, 0,
                                         nullptr, 0, s);
    }

    template <typename T>
    void cycle(const BLev<D, T>* const* lv, int l) {
        if (l == ltail) {
            launches += launch_tail_batched<D, T>(dtail, K, dactive, geos.data(), l, L, h[0]->solver, h[0]->bc,
                                                  true, s);
            return;
        }
        if (l == L - 1) {
            launches += launch_batched<D, T>(BPhase::coarsest, lv[l], nullptr, coarse.d, coarse.total, K, dactive, 0,
                                             nullptr, sizeof(T) * 2 * (size_t)max_nact, s);
            return;
        }
        const sulf_solver& sv = h[0]->solver;
        for (int k = 0; k < sv.nu1; k++) relax<T>(lv, l);
        launches += launch_batched<D, T>(BPhase::residual, lv[l], nullptr, act[l].d, act[l].total, K, dactive, 0,
                                         nullptr, 0, s);
        launches += launch_batched<D, T>(BPhase::extend, lv[l], nullptr, ext[l].d, ext[l].total, K, dactive, 0,
                                         nullptr, 0, s);
        launches += launch_batched<D, T>(BPhase::restrict_to, lv[l], lv[l + 1], act[l + 1].d, act[l + 1].total, K,
                                         dactive, 0, nullptr, 0, s);
        cycle<T>(lv, l + 1);
        launches += launch_batched<D, T>(BPhase::prolong_from, lv[l], lv[l + 1], act[l].d, act[l].total, K, dactive,
                                         0, nullptr, 0, s);
        for (int k = 0; k < sv.nu2; k++) relax<T>(lv, l);
    }

    // one cycle of every active instance's linear solve, then the FP64
    // defect with each instance's max-norm (copied to hnorm)
    int cycle_body() {
        const bool mixed = h[0]->solver.precision == 1;
        if (mixed) {
            launches += launch_batched_mixed<D>(BPhase::zero32, l64[0], l32[0], act[0].d, act[0].total, K, dactive,
                                                s);
            cycle<float>(l32, 0);
            launches += launch_batched_mixed<D>(BPhase::accumulate, l64[0], l32[0], act[0].d, act[0].total, K,
                                                dactive, s);
        } else {
            cycle<double>(l64, 0);
        }
        SULF_CUDA_TRY(cudaMemsetAsync(dnorm, 0, sizeof(unsigned long long) * K, s));
        if (mixed)  // the FP64 defect goes straight into the next FP32 right-hand side
            launches += launch_batched_mixed<D>(BPhase::residual_to32, l64[0], l32[0], act[0].d, act[0].total, K,
                                                dactive, s, dnorm);
        else
            launches += launch_batched<D, double>(BPhase::residual, l64[0], nullptr, act[0].d, act[0].total, K,
                                                  dactive, 0, dnorm, 0, s);
        SULF_CUDA_TRY(cudaMemcpyAsync(hnorm, dnorm, sizeof(unsigned long long) * K, cudaMemcpyDeviceToHost, s));
        return SULF_OK;
    }
};

// one CN step of every instance whose status is SULF_OK, Newton iterations
// and cycles in lock step; an instance that fails gets its code in status[i]
// and its message in err[i] (and keeps the state it failed in)
template <int D>
struct LockGraphs {
    PhaseGraph begin, prepare, cycle, update;
};

// The per-instance phases run for every instance of the class, whatever its
// state: an instance that left its Newton loop (converged, or failed) gets a
// zero update (its x is zeroed by the set-up and its cycles are masked), so
// its state does not change, and its norms are not read.
template <int D>
int lockstep_step(LockClass<D>& C, LockGraphs<D>& P, int* status, std::vector<std::string>& err) {
    const int K = C.K;
    const sulf_solver& sv = C.h[0]->solver;
    auto fail = [&](int i, int code, const std::string& msg) {
        status[i] = sulf_fail(code, msg);
        err[i] = msg;
    };
    std::vector<double> fn(K, 0.0);
    // the old-time part of each CN system and its first residual
    int rc = C.run_phase(P.begin, [&] {
        return C.per_instance([&](int i, cudaStream_t b) {
            sulf_domain* d = C.h[i];
            const LevelGeo& G0 = d->geo[0];
            FConst fc = make_fconst(d);
            SULF_CUDA_TRY(cudaMemcpyAsync(d->Wn, d->W, sizeof(double2) * G0.nn, cudaMemcpyDeviceToDevice, b));
            d->launches += launch_old_time<D>(G0, d->Wn, d->G, fc, b);
            SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 4, b));
            d->launches += launch_newton_F<D>(G0, d->W, d->G, d->v64[0].rhs, d->v64[0].rhsc, fc, d->dnorm, b);
            SULF_CUDA_TRY(cudaMemcpyAsync(d->hnorm, d->dnorm, sizeof(unsigned long long), cudaMemcpyDeviceToHost, b));
            return SULF_OK;
        });
    });
    if (rc) return rc;
    std::vector<int> inewton(K, 0);  // instance still in its Newton loop
    for (int i = 0; i < K; i++) {
        if (status[i] != SULF_OK) continue;
        sulf_domain* d = C.h[i];
        d->newton_last = 0;
        d->cycles_last = 0;
        fn[i] = bits_to_double(d->hnorm[0]);
        if (fn[i] < d->solver.newton_tol) {
            d->t += d->dt;
            d->steps_total++;
            d->last_fnorm = fn[i];
        } else {
            inewton[i] = 1;
        }
    }
    for (int k = 1; k <= sv.max_newton; k++) {
        bool any = false;
        for (int i = 0; i < K; i++) any = any || inewton[i];
        if (!any) break;
        // per instance: the Jacobian of this Newton iteration on every level
        rc = C.run_phase(P.prepare, [&] {
            return C.per_instance([&](int i, cudaStream_t b) {
                sulf_domain* d = C.h[i];
                const LevelGeo& G0 = d->geo[0];
                SULF_CUDA_TRY(cudaMemsetAsync(d->v64[0].x, 0, sizeof(double2) * G0.nn, b));
                int r;
                if (sv.precision == 0) {
                    r = MG<D, double>{d, d->v64}.prepare();
                } else {
                    d->launches += launch_to_float(G0, d->W, d->v32[0].Wc, b);
                    d->launches += launch_coefs<D, double>(G0, d->v64[0], make_coef<double>(d, 0), b);
                    r = MG<D, float>{d, d->v32}.prepare();
                    if (!r) d->launches += launch_to_float(G0, d->v64[0].rhs, d->v32[0].rhs, b);
                    // the batched cycles zero the FP32 error at the active
                    // nodes only; the others stay zero from here
                    SULF_CUDA_TRY(cudaMemsetAsync(d->v32[0].x, 0, sizeof(float2) * G0.nn, b));
                }
                if (r) return r;
                SULF_CUDA_TRY(cudaMemcpyAsync(d->hnorm + 6, d->dsing, sizeof(int), cudaMemcpyDeviceToHost, b));
                return SULF_OK;
            });
        });
        if (rc) return rc;
        for (int i = 0; i < K; i++) {
            C.active[i] = inewton[i];
            if (inewton[i] && *(int*)(C.h[i]->hnorm + 6)) {
                fail(i, SULF_ENOTCONV, "singular coarsest-level Jacobian");
                inewton[i] = 0;
                C.active[i] = 0;
            }
        }
        // the cycles of the linear solves, in lock step
        std::vector<double> rprev(fn);
        std::vector<int> cyc(K, 0);
        if (int rc = C.set_active()) return rc;
        for (int c = 1; c <= sv.max_cycles; c++) {
            bool on = false;
            for (int i = 0; i < K; i++) on = on || C.active[i];
            if (!on) break;
            if ((rc = C.run_phase(P.cycle, [&] { return C.cycle_body(); }))) return rc;
            bool changed = false;
            for (int i = 0; i < K; i++) {
                if (!C.active[i]) continue;
                sulf_domain* d = C.h[i];
                const double rn = bits_to_double(C.hnorm[i]);
                d->last_rho = rprev[i] > 0 ? rn / rprev[i] : 0.0;
                rprev[i] = rn;
                cyc[i] = c;
                if (rn <= sv.lin_rtol * fn[i] || rn != rn || c == sv.max_cycles) {
                    C.active[i] = 0;
                    changed = true;
                }
            }
            if (changed)
                if (int rc = C.set_active()) return rc;
        }
        // per instance: the Newton update, the new residual and the test
        rc = C.run_phase(P.update, [&] {
            return C.per_instance([&](int i, cudaStream_t b) {
                sulf_domain* d = C.h[i];
                const LevelGeo& G0 = d->geo[0];
                FConst fc = make_fconst(d);
                SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 4, b));
                d->launches += launch_newton_update(G0, d->W, d->v64[0].x, d->dnorm, b);
                d->launches += launch_newton_F<D>(G0, d->W, d->G, d->v64[0].rhs, d->v64[0].rhsc, fc, d->dnorm + 2, b);
                SULF_CUDA_TRY(
                    cudaMemcpyAsync(d->hnorm, d->dnorm, sizeof(unsigned long long) * 3, cudaMemcpyDeviceToHost, b));
                return SULF_OK;
            });
        });
        if (rc) return rc;
        for (int i = 0; i < K; i++) {
            if (!inewton[i]) continue;
            sulf_domain* d = C.h[i];
            d->cycles_last += cyc[i];
            d->cycles_total += cyc[i];
            const double dn = bits_to_double(d->hnorm[0]), wn = bits_to_double(d->hnorm[1]);
            fn[i] = bits_to_double(d->hnorm[2]);
            d->newton_last = k;
            d->newton_total++;
            d->last_fnorm = fn[i];
            const double rel = wn > 0 ? dn / wn : dn;
            if (fn[i] != fn[i] || dn != dn) {
                inewton[i] = 0;
                char buf[128];
                snprintf(buf, sizeof buf, "Newton did not converge (|F|_inf = %g)", fn[i]);
                fail(i, SULF_ENOTCONV, buf);
            } else if ((fn[i] < rel ? fn[i] : rel) < d->solver.newton_tol) {
                inewton[i] = 0;
                d->t += d->dt;
                d->steps_total++;
            }
        }
    }
    for (int i = 0; i < K; i++)
        if (inewton[i]) {
            char buf[128];
            snprintf(buf, sizeof buf, "Newton did not converge (|F|_inf = %g)", fn[i]);
            fail(i, SULF_ENOTCONV, buf);
        }
    return SULF_OK;
}

// nsteps CN steps of the class hs (each handle's stream is s); status and
// err per instance; the return code is that of a failure of the class as a
// whole (device memory, a launch)
template <int D>
int lockstep_run(const std::vector<sulf_domain*>& hs, double dt, int nsteps, int* status,
                 std::vector<std::string>& err, cudaStream_t s) {
    LockClass<D> C;
    Scratch mem;
    mem.s = s;
    C.h = hs;
    C.K = (int)hs.size();
    C.L = hs[0]->L;
    C.s = s;
    C.mem = &mem;
    for (sulf_domain* d : hs) {
        d->dt = dt;
        if (d->solver.precision == 1)
            if (int rc = ensure32(d)) return rc;
        if (int rc = refresh_ghost_ops(d)) return rc;
    }
    if (int rc = C.setup()) return rc;
    PdlScope pdl(hs[0]->solver.pdl != 0, 0, 0);
    LockGraphs<D> P;
    for (int k = 0; k < nsteps; k++) {
        if (int rc = lockstep_step<D>(C, P, status, err)) return rc;
        bool any = false;
        for (int i = 0; i < C.K; i++) any = any || status[i] == SULF_OK;
        if (!any) break;
    }
    // the batched launches, shared out over the instances
    const long long per = C.launches / C.K;
    for (sulf_domain* d : hs) d->launches += per;
    return SULF_OK;
}

}  // namespace

namespace sulf {

// whether a domain can join a lock-step class, and the class key
bool lockstep_key(sulf_handle h, std::vector<double>& key) {
    const sulf_domain* d = h;
    const sulf_solver& v = d->solver;
    if (v.cycle != 1 || v.smoother != 0 || !v.ghost_compose || d->src_on || d->sbg_on || d->prof || d->L < 2)
        return false;
    // the batched coarsest solve stages the right-hand side in shared memory
    if (d->geo[d->L - 1].nact > kLockMaxCoarsest) return false;
    for (int l = 0; l < d->L; l++) {
        const LevelGeo& G = d->geo[l];
        if (G.ng == 0) continue;
        const double tau = level_tau(d, l);
        if (!(G.gop_on && G.gop_bc == d->bc && G.gop_passes == v.ghost_sweeps && G.gop_tau == tau)) return false;
    }
    key = {(double)d->dim, (double)d->N, (double)d->L, (double)d->bc, (double)v.precision, (double)v.nu1,
           (double)v.nu2, (double)v.ghost_sweeps, v.tau_s, v.newton_tol, v.lin_rtol, (double)v.max_newton,
           (double)v.max_cycles, (double)v.pdl, (double)(v.precision == 1 && v.relax_matrix_free != 0)};
    return true;
}

int lockstep_advance(const sulf_handle* hs, int K, double dt, int nsteps, int* status, std::vector<std::string>& err,
                     cudaStream_t s) {
    std::vector<sulf_domain*> v(hs, hs + K);
    err.assign(K, std::string());
    for (int i = 0; i < K; i++) status[i] = SULF_OK;
    for (sulf_domain* d : v)
        if (d->stream != s) return sulf_fail(SULF_EINVAL, "lock-step class on mixed streams");
    int rc = v[0]->dim == 2 ? lockstep_run<2>(v, dt, nsteps, status, err, s)
                            : lockstep_run<3>(v, dt, nsteps, status, err, s);
    cudaStreamSynchronize(s);
    return rc;
}

}  // namespace sulf

// ---------------------------------------------------------------------------
// Autotuning of the controls that change only speed: the fused-level
// threshold, the composed ghost relaxation and dependent launch.  A candidate
// is timed on the handle's own problem -- the Newton system of a CN step of
// size dt from the current state -- as a linear solve of a fixed number of
// cycles (the defect test is off), once to build its graphs and once timed.
// The state is not changed.  Results are kept per problem class for the
// process, so same-size instances of a batch tune once.
namespace {

typedef std::array<int, 9> TuneKey;  // dim, N, coarsest N, precision, cycle, smoother, nu1, nu2, bc
std::mutex g_tune_mu;
std::map<TuneKey, sulf_tune_result> g_tune_cache;

TuneKey tune_key(const sulf_domain* d) {
    return {d->dim, d->N, d->N >> (d->L - 1), d->solver.precision, d->solver.cycle, d->solver.smoother,
            d->solver.nu1, d->solver.nu2, d->bc};
}

// ms per cycle of the current controls (the fixed set-up of the solve --
// injection, coefficients, coarsest inverse -- is included, as in a step)
template <int D>
int time_solve(sulf_domain* d, double fnorm, int ncycles, double* ms) {
    PdlScope pdl(d->solver.pdl != 0, d->solver.relax_occupancy, d->solver.relax_matrix_free);
    int c = linear_solve<D>(d, fnorm, ncycles, 0.0, nullptr);  // builds the graphs of this candidate
    if (c < 0) return c;
    SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
    const double t0 = host_ms();
    c = linear_solve<D>(d, fnorm, ncycles, 0.0, nullptr);
    if (c < 0) return c;
    SULF_CUDA_TRY(cudaStreamSynchronize(d->stream));
    *ms = (host_ms() - t0) / ncycles;
    return SULF_OK;
}

template <int D>
int autotune(sulf_domain* d, double dt, sulf_tune_result* out) {
    const LevelGeo& G0 = d->geo[0];
    d->dt = dt;
    FConst fc = make_fconst(d);
    SULF_CUDA_TRY(cudaMemcpyAsync(d->Wn, d->W, sizeof(double2) * G0.nn, cudaMemcpyDeviceToDevice, d->stream));
    d->launches += launch_old_time<D>(G0, d->Wn, d->G, fc, d->stream);
    SULF_CUDA_TRY(cudaMemsetAsync(d->dnorm, 0, sizeof(unsigned long long) * 4, d->stream));
    d->launches += launch_newton_F<D>(G0, d->W, d->G, d->v64[0].rhs, d->v64[0].rhsc, fc, d->dnorm, d->stream);
    if (int rc = read_norms(d, 1)) return rc;
    double fn = bits_to_double(d->hnorm[0]);
    if (!(fn > 0)) fn = 1.0;
    const sulf_solver base = d->solver;
    const int ncyc = 6;
    auto trial = [&](int fuse, int compose, int pdl, double* ms, int occ = -1, int mf = -1) {
        d->solver = base;
        d->solver.fuse_below = fuse;
        d->solver.ghost_compose = compose;
        d->solver.pdl = pdl;
        d->solver.relax_occupancy = occ < 0 ? base.relax_occupancy : occ;
        d->solver.relax_matrix_free = mf < 0 ? base.relax_matrix_free : mf;
        if (int rc = refresh_ghost_ops(d)) return rc;
        return time_solve<D>(d, fn, ncyc, ms);
    };
    sulf_tune_result r{};
    double best = 0;
    if (int rc = trial(-1, 1, 1, &best)) return rc;
    r.ms_per_cycle_default = best;
    r.fuse_below = -1;
    r.ghost_compose = 1;
    r.pdl = 1;
    r.candidates = 1;
    // the fused-level threshold (only V-cycles with red-black sweeps fuse)
    if (base.cycle == 1 && base.smoother != 2) {
        const int fuse[] = {0, 60, 150, 400, 1000, 3000, 10000};
        for (int f : fuse) {
            double ms = 0;
            if (int rc = trial(f, 1, 1, &ms)) return rc;
            r.candidates++;
            if (ms < best) {
                best = ms;
                r.fuse_below = f;
            }
        }
    }
    for (int compose = 0; compose < 2; compose++)
        for (int pdl = 0; pdl < 2; pdl++) {
            if (compose == 1 && pdl == 1) continue;
            double ms = 0;
            if (int rc = trial(r.fuse_below, compose, pdl, &ms)) return rc;
            r.candidates++;
            if (ms < best) {
                best = ms;
                r.ghost_compose = compose;
                r.pdl = pdl;
            }
        }
    r.relax_occupancy = base.relax_occupancy;
    r.relax_matrix_free = base.relax_matrix_free;
    if (base.precision == 0) {
        double ms = 0;
        const int occ = 1 - base.relax_occupancy;
        if (int rc = trial(r.fuse_below, r.ghost_compose, r.pdl, &ms, occ)) return rc;
        r.candidates++;
        if (ms < best) {
            best = ms;
            r.relax_occupancy = occ;
        }
    } else if (base.smoother == 0) {
        for (int mf = 0; mf <= (d->dim == 3 ? 2 : 1); mf++) {
            if (mf == base.relax_matrix_free) continue;
            if (mf == 2)
                if (int rc = ensure_tiles(d)) return rc;
            double ms = 0;
            if (int rc = trial(r.fuse_below, r.ghost_compose, r.pdl, &ms, -1, mf)) return rc;
            r.candidates++;
            if (ms < best) {
                best = ms;
                r.relax_matrix_free = mf;
            }
        }
    }
    r.ms_per_cycle = best;
    d->solver = base;
    d->solver.fuse_below = r.fuse_below;
    d->solver.ghost_compose = r.ghost_compose;
    d->solver.pdl = r.pdl;
    d->solver.relax_occupancy = r.relax_occupancy;
    d->solver.relax_matrix_free = r.relax_matrix_free;
    if (int rc = refresh_ghost_ops(d)) return rc;
    *out = r;
    return SULF_OK;
}

}  // namespace

extern "C" {

int sulf_autotune(sulf_handle h, double dt, int use_cache, sulf_tune_result* out) {
    if (!valid(h) || !(dt > 0)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const TuneKey key = tune_key(h);
    sulf_tune_result r{};
    bool hit = false;
    if (use_cache) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            r = it->second;
            r.cached = 1;
            hit = true;
        }
    }
    if (hit) {
        h->solver.fuse_below = r.fuse_below;
        h->solver.ghost_compose = r.ghost_compose;
        h->solver.pdl = r.pdl;
        h->solver.relax_occupancy = r.relax_occupancy;
        h->solver.relax_matrix_free = r.relax_matrix_free;
        if (r.relax_matrix_free == 2 && h->solver.precision == 1)
            if (int rc = ensure_tiles(h)) return rc;
        if (int rc = refresh_ghost_ops(h)) return rc;
    } else {
        const double dt0 = h->dt;
        int rc = h->dim == 2 ? autotune<2>(h, dt, &r) : autotune<3>(h, dt, &r);
        h->dt = dt0;
        cudaStreamSynchronize(h->stream);
        if (rc) return rc;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = r;
    }
    if (out) *out = r;
    return SULF_OK;
}

int sulf_dbg_cycles(sulf_handle h, double dt, const double* Wc0, const double* rhs, double* x, int ncycles,
                    double* rnorms) {
    if (!valid(h) || !Wc0 || !rhs || !x || ncycles < 1 || !(dt > 0)) return sulf_fail(SULF_EINVAL, "invalid arguments");
    const LevelGeo& G0 = h->geo[0];
    h->dt = dt;
    int rc = copy_in(h, h->W, Wc0, sizeof(double2) * G0.nn);
    if (!rc) rc = copy_in(h, h->v64[0].rhs, rhs, sizeof(double2) * G0.nn);
    if (!rc) h->launches += launch_gather_list(G0, h->v64[0].rhs, h->v64[0].rhsc, h->stream);
    if (rc) return rc;
    // the cycles start from x = 0 inside linear_solve; a nonzero start is
    // folded into the right-hand side: J (x0 + y) = rhs  <=>  J y = rhs - J x0
    std::vector<double> x0(x, x + 2 * G0.nn);
    bool nonzero = false;
    for (double v : x0) nonzero |= v != 0.0;
    if (nonzero) return sulf_fail(SULF_EINVAL, "sulf_dbg_cycles starts from x = 0");
    PdlScope pdl(h->solver.pdl != 0, h->solver.relax_occupancy, h->solver.relax_matrix_free);
    int nc = h->dim == 2 ? linear_solve<2>(h, 1.0, ncycles, 0.0, rnorms) : linear_solve<3>(h, 1.0, ncycles, 0.0, rnorms);
    if (nc < 0) return nc;
    return dbg_copy_out(h, 0, h->v64[0].x, x, false);
}

}  // extern "C"
