// The coarsest levels of a multigrid V-cycle (arXiv:1902.07029, Sec. 3.5) as
// one kernel launch.
//
// On the smallest levels (a few hundred to a few thousand active nodes) every
// phase -- two colours, the ghost passes, residual, band extension,
// restriction, prolongation -- is a chain of dependent loads over a handful of
// nodes: as separate graph nodes each costs a few microseconds of launch and
// latency, ~31 per level and cycle.  Here one CTA walks the levels l0 .. L-1
// down and back up with __syncthreads between phases, on L1-resident data.
// Each phase calls the same per-node stage functions as the per-level kernels
// (mg_stages.cuh), in the same order, so the result is the same.
#include <algorithm>
#include <mutex>

#include "mg_stages.cuh"

namespace sulf {

namespace {

constexpr int kTailThreads = 512;
constexpr int kTailRhs = 512;  // coarsest unknowns whose right-hand side is staged in shared memory

using stages::Lists;

// one level as seen by the fused cycle
template <typename T>
struct TailLevel {
    typedef typename V2<T>::t T2;
    Lists ls;
    int n;
    double h;
    long long st1, st2;
    const int8_t* type;
    stages::GhostTab<T> tab;
    int nb;
    const int* bidx;
    const int* eptr;
    const int* eidx;
    const T* eval;
    int nact;
    const int* act;
    const T* Ainv;
    T2* rhs;
    T2* x;
    T2* res;
    T* gbuf[2];
    const T2* edge[3];
    const T2* Pa;
    const T2* Pb;
    const T2* Ia;
    const T2* Ib;
    const T2* gc;
    const T* gci;
    // composed ghost relaxation (null where the level has none)
    const int* gop_ptr;
    const int* gop_code;
    const T* gop_val;
    int gop_nnz;
};

struct TailParams {
    int l0, L, nu1, nu2, passes, pointwise, bc;
    int compose;     // every fused level relaxes its ghosts by the composed map
    int stage_gop;   // the composed rows are copied into shared memory
    int stage_ainv;  // the coarsest inverse is copied into shared memory
    double tau;
};

// Shared-memory layout of the staged data, the same on host and device: per
// fused level with a composed map its row pointers, codes and weights, then
// the coarsest inverse; every region starts on 16 bytes.
__host__ __device__ inline size_t a16(size_t o) { return (o + 15) & ~size_t(15); }
__host__ __device__ inline size_t gop_stage_bytes(int ng, int nnz, size_t tsize) {
    return a16(4 * (size_t)(ng + 1)) + a16(4 * (size_t)nnz) + a16(tsize * (size_t)nnz);
}
constexpr size_t kTailStageCap = 200 * 1024;

// copy of a byte range in 16-byte pieces (both ends on 16 bytes; the source
// allocation extends to a multiple of 256 bytes) by the whole CTA
__device__ __forceinline__ void stage_copy(void* dst, const void* src, size_t bytes) {
    const size_t n16 = (bytes + 15) / 16;
    for (size_t c = threadIdx.x; c < n16; c += blockDim.x) {
        const unsigned d = (unsigned)__cvta_generic_to_shared((char*)dst + 16 * c);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"((const char*)src + 16 * c) : "memory");
    }
}
__device__ __forceinline__ void stage_wait() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

template <int D, typename T>
__device__ __forceinline__ stages::CoefPtr<D, T> coefs_of(const TailLevel<T>& v) {
    stages::CoefPtr<D, T> c;
    for (int a = 0; a < 3; a++) c.edge[a] = v.edge[a];
    c.Pa = v.Pa;
    c.Pb = v.Pb;
    c.Ia = v.Ia;
    c.Ib = v.Ib;
    c.gc = v.gc;
    c.Pc = nullptr;  // the fused levels read the box-ordered blocks
    c.Ic = nullptr;
    return c;
}

// one relaxation sweep of Sec. 3.5.1 on level v: red, black, ghost passes
template <int D, typename T>
__device__ void tail_relax(const TailLevel<T>& v, const TailParams& pr, int tid, int nthr, const int* gptr,
                           const int* gcode, const T* gval) {
    const long long st[3] = {1, v.st1, v.st2};
    stages::CoefPtr<D, T> cf = coefs_of<D, T>(v);
    for (int colour = 0; colour < 2; colour++) {
        const int* list = colour ? v.ls.l1 : v.ls.l0;
        int cnt = colour ? v.ls.n1 : v.ls.n0;
        for (int t = tid; t < cnt; t += nthr) {
            if (pr.pointwise)
                stages::relax_node<D, T, true, false>(list[t], cf, v.rhs, v.x, st);
            else
                stages::relax_node<D, T, false, false>(list[t], cf, v.rhs, v.x, st);
        }
        // the composed ghost relaxation starts from the ghosts' s, which the
        // inside update does not write
        if (colour == 1 && pr.compose)
            for (int gi = tid; gi < v.ls.ng; gi += nthr)
                v.gbuf[0][gi] = reinterpret_cast<const T*>(v.x + v.ls.lg[gi])[0];
        __syncthreads();
    }
    if (pr.compose) {
        if (pr.stage_gop) stage_wait();  // the rows copied at the start (waits once)
        // kGopLanes threads per ghost row, as in the per-level kernel (the
        // same summation order, so the same bits)
        const int per = nthr / stages::kGopLanes;
        for (int base = 0; base < v.ls.ng; base += per) {
            const int gi = base + tid / stages::kGopLanes;
            stages::gop_group<T>(gi < v.ls.ng, tid % stages::kGopLanes, gi, gptr, gcode, gval, v.ls.lg, v.gc, v.gci,
                                 v.rhs, v.x, v.gbuf[0]);
        }
        __syncthreads();
        return;
    }
    const T tau = (T)(pr.bc ? pr.tau * tail_tau_scale(D, v.h) : pr.tau);
    for (int p = 0; p < pr.passes; p++) {
        bool first = p == 0, last = p == pr.passes - 1 && pr.passes > 1;
        const T* sin = first ? nullptr : v.gbuf[(p - 1) & 1];
        T* sout = v.gbuf[p & 1];
        for (int gi = tid; gi < v.ls.ng; gi += nthr)
            stages::ghost_pass_node<D, T, false>(gi, v.ls.lg, v.tab, v.gc, v.gci, v.rhs, v.x, sin, sout, tau, first,
                                                 last);
        __syncthreads();
    }
    if (pr.passes == 1) {
        for (int gi = tid; gi < v.ls.ng; gi += nthr)
            reinterpret_cast<T*>(v.x + v.ls.lg[gi])[0] = v.gbuf[0][gi];
        __syncthreads();
    }
}

// the fused levels pr.l0 .. pr.L-1 of one instance's cycle, by the whole CTA
template <int D, typename T>
__device__ __forceinline__ void tail_cycle(const TailLevel<T>* __restrict__ lv, const TailParams& pr) {
    typedef typename V2<T>::t T2;
    const int tid = threadIdx.x;
    const int nthr = blockDim.x;
    // the composed ghost rows and the coarsest inverse are fixed during the
    // linear solve: copied into shared memory asynchronously while the first
    // phases run, they take the global-memory latency off later phases
    extern __shared__ __align__(16) unsigned char tail_smem[];
    __shared__ const int* s_gptr[SULF_MAXLEV];
    __shared__ const int* s_gcode[SULF_MAXLEV];
    __shared__ const T* s_gval[SULF_MAXLEV];
    __shared__ const T* s_ainv;
    if (tid == 0) {
        size_t off = 0;
        for (int l = pr.l0; l < pr.L; l++) {
            const TailLevel<T>& v = lv[l];
            s_gptr[l] = v.gop_ptr;
            s_gcode[l] = v.gop_code;
            s_gval[l] = v.gop_val;
            if (pr.stage_gop && v.gop_ptr && v.ls.ng > 0) {
                s_gptr[l] = reinterpret_cast<const int*>(tail_smem + off);
                s_gcode[l] = reinterpret_cast<const int*>(tail_smem + off + a16(4 * (size_t)(v.ls.ng + 1)));
                s_gval[l] = reinterpret_cast<const T*>(tail_smem + off + a16(4 * (size_t)(v.ls.ng + 1)) +
                                                       a16(4 * (size_t)v.gop_nnz));
                off += gop_stage_bytes(v.ls.ng, v.gop_nnz, sizeof(T));
            }
        }
        s_ainv = pr.stage_ainv ? reinterpret_cast<const T*>(tail_smem + off) : lv[pr.L - 1].Ainv;
    }
    __syncthreads();
    for (int l = pr.l0; l < pr.L; l++) {
        const TailLevel<T>& v = lv[l];
        if (s_gptr[l] != v.gop_ptr) {
            stage_copy((void*)s_gptr[l], v.gop_ptr, 4 * (size_t)(v.ls.ng + 1));
            stage_copy((void*)s_gcode[l], v.gop_code, 4 * (size_t)v.gop_nnz);
            stage_copy((void*)s_gval[l], v.gop_val, sizeof(T) * (size_t)v.gop_nnz);
        }
    }
    if (pr.stage_ainv) {
        const int m = 2 * lv[pr.L - 1].nact;
        stage_copy((void*)s_ainv, lv[pr.L - 1].Ainv, sizeof(T) * (size_t)m * m);
    }
    // descent
    for (int l = pr.l0; l < pr.L - 1; l++) {
        const TailLevel<T>& f = lv[l];
        const TailLevel<T>& c = lv[l + 1];
        for (int k = 0; k < pr.nu1; k++) tail_relax<D, T>(f, pr, tid, nthr, s_gptr[l], s_gcode[l], s_gval[l]);
        stages::CoefPtr<D, T> cf = coefs_of<D, T>(f);
        int tot = f.ls.n0 + f.ls.n1 + f.ls.ng;
        for (int t = tid; t < tot; t += nthr)
            stages::residual_node<D, T, false>(t, f.ls, f.tab, cf, f.rhs, f.x, f.res, f.st1, f.st2);
        __syncthreads();
        for (int b = tid; b < f.nb; b += nthr)
            stages::extend_node<T, false>(b, f.eptr, f.eidx, f.eval, f.bidx, f.res);
        __syncthreads();
        int ctot = c.ls.n0 + c.ls.n1 + c.ls.ng;
        for (int t = tid; t < ctot; t += nthr)
            stages::restrict_node<D, T, false>(t, c.ls, c.type, c.n, f.type, f.n, f.res, c.rhs, c.x);
        __syncthreads();
    }
    // coarsest level: x = A^{-1} rhs, one warp per row of the inverse, the
    // right-hand side gathered into shared memory first (when it fits)
    {
        const TailLevel<T>& c = lv[pr.L - 1];
        const int m = 2 * c.nact;
        const int lane = threadIdx.x & 31;
        const int warp = tid >> 5, nwarp = nthr >> 5;
        __shared__ T bsh[kTailRhs];
        const bool staged = m <= kTailRhs;
        if (pr.stage_ainv) stage_wait();
        if (staged) {
            for (int j = tid; j < m; j += nthr) {
                T2 b = c.rhs[c.act[j >> 1]];
                bsh[j] = (j & 1) ? b.y : b.x;
            }
            __syncthreads();
        }
        if (staged) {
            // one thread per row: full warps of multiply-adds and no shuffle
            // reductions (each sub-partition of the SM issues one warp-wide
            // FP64 instruction per 64 cycles)
            for (int r = tid; r < m; r += nthr) {
                const T* row = s_ainv + (long long)r * m;
                T acc = 0;
#pragma unroll 4
                for (int j = 0; j < m; j++) acc = stages::fmadd(row[j], bsh[j], acc);
                reinterpret_cast<T*>(c.x + c.act[r >> 1])[r & 1] = acc;
            }
        } else {
            for (int r = warp; r < m; r += nwarp) {
                const T* row = s_ainv + (long long)r * m;
                T acc = 0;
                for (int j = lane; j < m; j += 32) {
                    T2 b = c.rhs[c.act[j >> 1]];
                    acc += row[j] * ((j & 1) ? b.y : b.x);
                }
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
                if (lane == 0) reinterpret_cast<T*>(c.x + c.act[r >> 1])[r & 1] = acc;
            }
        }
        __syncthreads();
    }
    // ascent
    for (int l = pr.L - 2; l >= pr.l0; l--) {
        const TailLevel<T>& f = lv[l];
        const TailLevel<T>& c = lv[l + 1];
        int tot = f.ls.n0 + f.ls.n1 + f.ls.ng;
        for (int t = tid; t < tot; t += nthr) stages::prolong_node<D, T, false>(t, f.ls, c.type, c.n, c.x, f.n, f.x);
        __syncthreads();
        for (int k = 0; k < pr.nu2; k++) tail_relax<D, T>(f, pr, tid, nthr, s_gptr[l], s_gcode[l], s_gval[l]);
    }
}

template <int D, typename T>
__global__ void __launch_bounds__(kTailThreads, 1) k_tail(const TailLevel<T>* __restrict__ lv, TailParams pr) {
    pdl_enter();
    tail_cycle<D, T>(lv, pr);
}

// the fused levels of many instances (lock-step batching): CTA i runs
// instance i's, unless it is masked
template <int D, typename T>
__global__ void __launch_bounds__(kTailThreads, 1)
    k_tail_batched(const TailLevel<T>* const* __restrict__ lvs, const int* __restrict__ active, TailParams pr) {
    if (!active[blockIdx.x]) return;
    pdl_enter();
    tail_cycle<D, T>(lvs[blockIdx.x], pr);
}

template <typename T>
TailLevel<T> describe(const LevelGeo& G, const LevelVec<T>& V) {
    TailLevel<T> t;
    t.ls = stages::make_lists(G);
    t.n = G.n;
    t.h = G.h;
    t.st1 = G.st[1];
    t.st2 = G.st[2];
    t.type = G.type;
    t.tab = stages::ghost_tab<T>(G);
    t.nb = G.nb;
    t.bidx = G.bidx;
    t.eptr = G.eptr;
    t.eidx = G.eidx;
    t.eval = std::is_same<T, float>::value ? (const T*)G.eval32 : (const T*)G.eval;
    t.nact = G.nact;
    t.act = G.act;
    t.Ainv = V.Ainv;
    t.rhs = V.rhs;
    t.x = V.x;
    t.res = V.res;
    for (int k = 0; k < 2; k++) t.gbuf[k] = V.gbuf[k];
    for (int a = 0; a < 3; a++) t.edge[a] = V.edge[a];
    t.Pa = V.Pa;
    t.Pb = V.Pb;
    t.Ia = V.Ia;
    t.Ib = V.Ib;
    t.gc = V.gc;
    t.gci = V.gci;
    t.gop_ptr = G.gop_on ? G.gop_ptr : nullptr;
    t.gop_code = G.gop_on ? G.gop_code : nullptr;
    t.gop_val = !G.gop_on ? nullptr : std::is_same<T, float>::value ? (const T*)G.gop_val32 : (const T*)G.gop_val;
    t.gop_nnz = G.gop_on ? (int)G.gop_nnz : 0;
    return t;
}

}  // namespace

size_t tail_desc_bytes(int L) { return sizeof(TailLevel<double>) * (size_t)L; }

template <typename T>
int upload_tail_desc(const LevelGeo* G, const LevelVec<T>* V, int L, void* dev, cudaStream_t s) {
    std::vector<TailLevel<T>> h(L);
    for (int l = 0; l < L; l++) h[l] = describe<T>(G[l], V[l]);
    cudaError_t e = cudaMemcpyAsync(dev, h.data(), sizeof(TailLevel<T>) * L, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return sulf_fail_cuda(e, "tail descriptor upload");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return sulf_fail_cuda(e, "tail descriptor upload");
    return SULF_OK;
}

namespace {

TailParams make_params(int l0, int L, const sulf_solver& sv, int bc, bool compose, int D) {
    TailParams pr;
    pr.compose = compose ? 1 : 0;
    pr.stage_gop = 0;
    pr.stage_ainv = 0;
    pr.l0 = l0;
    pr.L = L;
    pr.nu1 = sv.nu1;
    pr.nu2 = sv.nu2;
    pr.passes = sv.ghost_sweeps;
    pr.pointwise = sv.smoother == 1;
    pr.tau = sv.tau_s;
    pr.bc = bc;
    (void)D;
    return pr;
}

}  // namespace

template <int D, typename T>
int launch_tail(const void* dev_desc, const LevelGeo* G, int l0, int L, const sulf_solver& sv, int bc, bool compose,
                cudaStream_t s) {
    TailParams pr = make_params(l0, L, sv, bc, compose, D);
    // what fits in shared memory is staged: the composed rows first, then the
    // coarsest inverse (the same layout rule as the kernel's)
    size_t off = 0;
    if (compose) {
        for (int l = l0; l < L; l++)
            if (G[l].gop_on && G[l].ng > 0) off += gop_stage_bytes(G[l].ng, (int)G[l].gop_nnz, sizeof(T));
        if (off <= kTailStageCap)
            pr.stage_gop = 1;
        else
            off = 0;
    }
    const size_t m = 2 * (size_t)G[L - 1].nact;
    if (off + m * m * sizeof(T) <= kTailStageCap) {
        pr.stage_ainv = 1;
        off += m * m * sizeof(T);
    }
    static std::mutex mu;
    static bool raised[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !raised[dev]) {
            cudaFuncSetAttribute(k_tail<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailStageCap);
            if (dev >= 0 && dev < 64) raised[dev] = true;
        }
    }
    launch_k(k_tail<D, T>, 1, kTailThreads, off, s, (const TailLevel<T>*)dev_desc, pr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sulf_fail_cuda(e, "fused coarse-level cycle launch");
    return SULF_OK;
}

template <int D, typename T>
int launch_tail_batched(const void* const* dev_descs, int K, const int* active, const LevelGeo* const* G, int l0,
                        int L, const sulf_solver& sv, int bc, bool compose, cudaStream_t s) {
    TailParams pr = make_params(l0, L, sv, bc, compose, D);
    // staging as in launch_tail, decided for all instances at once: on where
    // every instance's data fits; the shared memory is the largest need
    size_t gop_max = 0, all_max = 0;
    bool gop_fits = compose, all_fit = true;
    for (int i = 0; i < K; i++) {
        size_t off = 0;
        if (compose)
            for (int l = l0; l < L; l++)
                if (G[i][l].gop_on && G[i][l].ng > 0) off += gop_stage_bytes(G[i][l].ng, (int)G[i][l].gop_nnz, sizeof(T));
        gop_fits = gop_fits && off <= kTailStageCap;
        gop_max = std::max(gop_max, off);
        const size_t m = 2 * (size_t)G[i][L - 1].nact;
        all_fit = all_fit && off + m * m * sizeof(T) <= kTailStageCap;
        all_max = std::max(all_max, off + m * m * sizeof(T));
    }
    size_t smem = 0;
    if (gop_fits) {
        pr.stage_gop = 1;
        smem = gop_max;
        if (all_fit) {
            pr.stage_ainv = 1;
            smem = all_max;
        }
    }
    static std::mutex mu;
    static bool raised[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lock(mu);
        if (dev < 0 || dev >= 64 || !raised[dev]) {
            cudaFuncSetAttribute(k_tail_batched<D, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTailStageCap);
            if (dev >= 0 && dev < 64) raised[dev] = true;
        }
    }
    launch_k(k_tail_batched<D, T>, (unsigned)K, kTailThreads, smem, s, (const TailLevel<T>* const*)dev_descs, active,
             pr);
    return 1;
}

template int upload_tail_desc<double>(const LevelGeo*, const LevelVec<double>*, int, void*, cudaStream_t);
template int upload_tail_desc<float>(const LevelGeo*, const LevelVec<float>*, int, void*, cudaStream_t);
template int launch_tail<2, double>(const void*, const LevelGeo*, int, int, const sulf_solver&, int, bool,
                                    cudaStream_t);
template int launch_tail<2, float>(const void*, const LevelGeo*, int, int, const sulf_solver&, int, bool, cudaStream_t);
template int launch_tail<3, double>(const void*, const LevelGeo*, int, int, const sulf_solver&, int, bool,
                                    cudaStream_t);
template int launch_tail<3, float>(const void*, const LevelGeo*, int, int, const sulf_solver&, int, bool, cudaStream_t);
#define SULF_INST_TAIL_BATCHED(D, T)                                                                            \
    template int launch_tail_batched<D, T>(const void* const*, int, const int*, const LevelGeo* const*, int, int, \
                                           const sulf_solver&, int, bool, cudaStream_t);
SULF_INST_TAIL_BATCHED(2, double)
SULF_INST_TAIL_BATCHED(2, float)
SULF_INST_TAIL_BATCHED(3, double)
SULF_INST_TAIL_BATCHED(3, float)

}  // namespace sulf
