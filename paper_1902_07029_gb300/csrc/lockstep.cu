// Multigrid phases of many domains in one launch (lock-step batching).
//
// Domains of one size class (same dimension, N and levels) advance their
// Newton iterations and multigrid cycles in lock step; each phase of a cycle
// (a colour of the inside relaxation, the composed ghost relaxation, the
// residual, the band extension, the restriction, the prolongation, the
// coarsest solve) is one launch over an (instance, node) work list: CTA b
// belongs to the instance i with pre[i] <= b < pre[i+1] and takes its nodes
// from that instance's level.  An instance whose linear solve has converged
// is masked (its CTAs return at once), so every instance runs exactly the
// cycles it would run alone, with the same per-node stage functions
// (mg_stages.cuh), hence the same results.
#include "lockstep.cuh"

namespace sulf {
namespace {

constexpr int kBT = 256;

__device__ __forceinline__ int find_instance(const int* __restrict__ pre, int K, int b) {
    int lo = 0, hi = K;  // pre[0] = 0 <= b < pre[K]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pre[mid] <= b)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// block-wide max of non-negative doubles held as bit patterns, one atomicMax
__device__ __forceinline__ void block_max_to(unsigned long long v, unsigned long long* out) {
    __shared__ unsigned long long sm[kBT / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
    }
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long m = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) m = sm[k] > m ? sm[k] : m;
        atomicMax(out, m);
    }
}

// one colour of the collective red-black relaxation; the second colour also
// copies the ghosts' s for the composed ghost relaxation
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_relax(const BLev<D, T>* __restrict__ lv, const int* __restrict__ pre, int K,
                                                 const int* __restrict__ active, int colour) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& L = lv[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    const long long st[3] = {1, L.st1, L.st2};
    const int cnt = colour ? L.ls.n1 : L.ls.n0;
    const int* list = colour ? L.ls.l1 : L.ls.l0;
    pdl_enter();
    if (colour == 1 && t < L.ls.ng) L.snap[t] = reinterpret_cast<const T*>(L.x + L.ls.lg[t])[0];
    if (t < cnt) {
        const int tl = (colour ? L.ls.n0 : 0) + t;
        const long long p = list[t];
        const stages::InsideCoef<D, T> k = stages::fetch_inside_at<D, T, false>(p, tl, L.cf, st);
        stages::relax_apply_b<D, T, false, false>(p, k, L.rhsc ? L.rhsc[tl] : L.rhs[p], L.x, st);
    }
}

// the same with the coefficients formed from Wc (FP32): fewer bytes per
// update than the stored coefficient arrays
template <int D>
__global__ void __launch_bounds__(kBT) kb_relax_mf(const BLev<D, float>* __restrict__ lv, const int* __restrict__ pre,
                                                    int K, const int* __restrict__ active, int colour) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, float>& L = lv[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    const long long st[3] = {1, L.st1, L.st2};
    const int cnt = colour ? L.ls.n1 : L.ls.n0;
    const int* list = colour ? L.ls.l1 : L.ls.l0;
    long long p = 0;
    stages::MfCoef<D> k;
    if (t < cnt) {
        p = list[t];
        k = stages::mf_coef<D>(p, L.Wc, L.c, st);
    }
    pdl_enter();
    if (colour == 1 && t < L.ls.ng) L.snap[t] = reinterpret_cast<const float*>(L.x + L.ls.lg[t])[0];
    if (t < cnt) stages::mf_apply<D>(p, k, L.rhs, L.x, st);
}

// the composed ghost relaxation: kGopLanes lanes per ghost row
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_ghost_op(const BLev<D, T>* __restrict__ lv, const int* __restrict__ pre,
                                                    int K, const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& L = lv[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    const int gi = t / stages::kGopLanes, ln = t % stages::kGopLanes;
    pdl_enter();
    stages::gop_group<T>(gi < L.ls.ng, ln, gi, L.gop_ptr, L.gop_code, L.gop_val, L.ls.lg, L.gc, L.gci, L.rhs, L.x,
                         L.snap);
}

// defect rhs - J x on the active nodes; with norms, each instance's max-norm
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_residual(const BLev<D, T>* __restrict__ lv, const int* __restrict__ pre,
                                                    int K, const int* __restrict__ active,
                                                    unsigned long long* norms) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& L = lv[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    unsigned long long nb = 0;
    if (t < L.ls.n0 + L.ls.n1 + L.ls.ng)
        nb = stages::residual_node<D, T, false>(t, L.ls, L.tb, L.cf, L.rhs, L.x, L.res, L.st1, L.st2, L.rhsc);
    if (norms) block_max_to(nb, norms + i);
}

// ghost defects extended into the band (the precomputed operator)
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_extend(const BLev<D, T>* __restrict__ lv, const int* __restrict__ pre,
                                                  int K, const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& L = lv[i];
    const int b = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    if (b < L.nb) stages::extend_node<T, false>(b, L.eptr, L.eidx, L.eval, L.bidx, L.res);
}

// boundary-aware full weighting from fine level f to coarse level c (the
// coarse error starts from zero)
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_restrict(const BLev<D, T>* __restrict__ fl, const BLev<D, T>* __restrict__ cl,
                                                    const int* __restrict__ pre, int K,
                                                    const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& F = fl[i];
    const BLev<D, T>& C = cl[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    if (t < C.ls.n0 + C.ls.n1 + C.ls.ng)
        stages::restrict_node<D, T, false>(t, C.ls, C.type, C.n, F.type, F.n, F.res, C.rhs, C.x, C.rhsc);
}

// (bi/tri)linear interpolation of the coarse error added to the fine one
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_prolong(const BLev<D, T>* __restrict__ fl, const BLev<D, T>* __restrict__ cl,
                                                   const int* __restrict__ pre, int K,
                                                   const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& F = fl[i];
    const BLev<D, T>& C = cl[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    if (t < F.ls.n0 + F.ls.n1 + F.ls.ng) stages::prolong_node<D, T, false>(t, F.ls, C.type, C.n, C.x, F.n, F.x);
}

// coarsest level: x = A^{-1} rhs, one warp per row of the inverse (kBT / 32
// rows per CTA), the right-hand side staged in shared memory
template <int D, typename T>
__global__ void __launch_bounds__(kBT) kb_coarsest(const BLev<D, T>* __restrict__ lv, const int* __restrict__ pre,
                                                    int K, const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, T>& L = lv[i];
    extern __shared__ __align__(16) unsigned char kb_smem[];
    T* b = reinterpret_cast<T*>(kb_smem);
    const int m = 2 * L.nact;
    pdl_enter();
    for (int r = threadIdx.x; r < L.nact; r += kBT) {
        const typename V2<T>::t v = L.rhs[L.act[r]];
        b[2 * r] = v.x;
        b[2 * r + 1] = v.y;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int r = (blockIdx.x - pre[i]) * (kBT / 32) + (threadIdx.x >> 5);
    if (r >= m) return;
    const T* row = L.Ainv + (long long)r * m;
    T acc = 0;
    for (int j = lane; j < m; j += 32) acc += row[j] * b[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) reinterpret_cast<T*>(L.x + L.act[r >> 1])[r & 1] = acc;
}

// zero of the FP32 error at the active nodes, accumulation dW += e and the
// next FP32 right-hand side from the FP64 defect (the mixed form's finest
// level); instance i's FP64 level in l64, FP32 level in l32
template <int D>
__global__ void __launch_bounds__(kBT) kb_zero32(const BLev<D, float>* __restrict__ l32, const int* __restrict__ pre,
                                                  int K, const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, float>& U = l32[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    int kind, gi;
    if (t < U.ls.n0 + U.ls.n1 + U.ls.ng) U.x[stages::list_node(U.ls, t, kind, gi)] = make_float2(0.f, 0.f);
}

template <int D>
__global__ void __launch_bounds__(kBT) kb_accumulate(const BLev<D, double>* __restrict__ l64,
                                                      const BLev<D, float>* __restrict__ l32,
                                                      const int* __restrict__ pre, int K,
                                                      const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, double>& V = l64[i];
    const BLev<D, float>& U = l32[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    int kind, gi;
    if (t < V.ls.n0 + V.ls.n1 + V.ls.ng) {
        const long long p = stages::list_node(V.ls, t, kind, gi);
        const float2 e = U.x[p];
        double2 x = V.x[p];
        x.x += (double)e.x;
        x.y += (double)e.y;
        V.x[p] = x;
    }
}

// the FP64 defect of the mixed form written straight into the FP32
// right-hand side of the next FP32 cycle, with each instance's max-norm
template <int D>
__global__ void __launch_bounds__(kBT) kb_residual_to32(const BLev<D, double>* __restrict__ l64,
                                                         const BLev<D, float>* __restrict__ l32,
                                                         const int* __restrict__ pre, int K,
                                                         const int* __restrict__ active, unsigned long long* norms) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, double>& V = l64[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    unsigned long long nb = 0;
    if (t < V.ls.n0 + V.ls.n1 + V.ls.ng)
        nb = stages::residual_node<D, double, false>(t, V.ls, V.tb, V.cf, V.rhs, V.x, l32[i].rhs, V.st1, V.st2,
                                                     V.rhsc);
    block_max_to(nb, norms + i);
}

template <int D>
__global__ void __launch_bounds__(kBT) kb_to_float(const BLev<D, double>* __restrict__ l64,
                                                    const BLev<D, float>* __restrict__ l32,
                                                    const int* __restrict__ pre, int K,
                                                    const int* __restrict__ active) {
    const int i = find_instance(pre, K, blockIdx.x);
    if (!active[i]) return;
    const BLev<D, double>& V = l64[i];
    const BLev<D, float>& U = l32[i];
    const int t = (blockIdx.x - pre[i]) * kBT + threadIdx.x;
    pdl_enter();
    int kind, gi;
    if (t < V.ls.n0 + V.ls.n1 + V.ls.ng) {
        const long long p = stages::list_node(V.ls, t, kind, gi);
        const double2 r = V.res[p];
        U.rhs[p] = make_float2((float)r.x, (float)r.y);
    }
}

}  // namespace

template <int D, typename T>
int launch_batched(BPhase ph, const BLev<D, T>* lv, const BLev<D, T>* lc, const int* pre, int nblocks, int K,
                   const int* active, int colour, unsigned long long* norms, size_t smem, cudaStream_t s) {
    if (nblocks <= 0) return 0;
    switch (ph) {
        case BPhase::relax:
            launch_k(kb_relax<D, T>, (unsigned)nblocks, kBT, 0, s, lv, pre, K, active, colour);
            break;
        case BPhase::relax_mf:
            if (!std::is_same<T, float>::value) return 0;
            launch_k(kb_relax_mf<D>, (unsigned)nblocks, kBT, 0, s, reinterpret_cast<const BLev<D, float>*>(lv), pre,
                     K, active, colour);
            break;
        case BPhase::ghost_op:
            launch_k(kb_ghost_op<D, T>, (unsigned)nblocks, kBT, 0, s, lv, pre, K, active);
            break;
        case BPhase::residual:
            launch_k(kb_residual<D, T>, (unsigned)nblocks, kBT, 0, s, lv, pre, K, active, norms);
            break;
        case BPhase::extend:
            launch_k(kb_extend<D, T>, (unsigned)nblocks, kBT, 0, s, lv, pre, K, active);
            break;
        case BPhase::restrict_to:
            launch_k(kb_restrict<D, T>, (unsigned)nblocks, kBT, 0, s, lv, lc, pre, K, active);
            break;
        case BPhase::prolong_from:
            launch_k(kb_prolong<D, T>, (unsigned)nblocks, kBT, 0, s, lv, lc, pre, K, active);
            break;
        case BPhase::coarsest:
            launch_k(kb_coarsest<D, T>, (unsigned)nblocks, kBT, smem, s, lv, pre, K, active);
            break;
        default:
            return 0;
    }
    return 1;
}

template <int D>
int launch_batched_mixed(BPhase ph, const BLev<D, double>* l64, const BLev<D, float>* l32, const int* pre,
                         int nblocks, int K, const int* active, cudaStream_t s, unsigned long long* norms) {
    if (nblocks <= 0) return 0;
    switch (ph) {
        case BPhase::residual_to32:
            launch_k(kb_residual_to32<D>, (unsigned)nblocks, kBT, 0, s, l64, l32, pre, K, active, norms);
            break;
        case BPhase::zero32:
            launch_k(kb_zero32<D>, (unsigned)nblocks, kBT, 0, s, l32, pre, K, active);
            break;
        case BPhase::accumulate:
            launch_k(kb_accumulate<D>, (unsigned)nblocks, kBT, 0, s, l64, l32, pre, K, active);
            break;
        case BPhase::to_float:
            launch_k(kb_to_float<D>, (unsigned)nblocks, kBT, 0, s, l64, l32, pre, K, active);
            break;
        default:
            return 0;
    }
    return 1;
}

#define SULF_INST_BATCHED(D, T)                                                                                  \
    template int launch_batched<D, T>(BPhase, const BLev<D, T>*, const BLev<D, T>*, const int*, int, int,         \
                                      const int*, int, unsigned long long*, size_t, cudaStream_t);
SULF_INST_BATCHED(2, double)
SULF_INST_BATCHED(3, double)
SULF_INST_BATCHED(2, float)
SULF_INST_BATCHED(3, float)
template int launch_batched_mixed<2>(BPhase, const BLev<2, double>*, const BLev<2, float>*, const int*, int, int,
                                     const int*, cudaStream_t, unsigned long long*);
template int launch_batched_mixed<3>(BPhase, const BLev<3, double>*, const BLev<3, float>*, const int*, int, int,
                                     const int*, cudaStream_t, unsigned long long*);

}  // namespace sulf
