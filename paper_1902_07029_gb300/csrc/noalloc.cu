// Newton residual without device allocation.
//
// Some callers cannot allocate device memory at the moment they need a
// residual: a host application whose own memory manager has already reserved
// the device memory it may use (cudaMalloc would fail or break its budget),
// or a time-critical loop that must not take the device-wide synchronisation
// a cudaMalloc/cudaFree can imply.  sulf_newton_residual_noalloc lets them
// evaluate F(W; W^n) and |F|_inf on their own device buffers: its only scratch
// memory -- the per-block partial maxima of a two-pass max-norm reduction --
// lives in the file-scope array below, which every GPU that loads this library
// holds until the process exits.
#include <mutex>

#include "sulf_internal.cuh"

namespace {

using namespace sulf;

// partial maxima, one per block of kThreads active nodes (bit patterns of
// non-negative doubles); 65536 entries = 512 KiB
constexpr int kThreads = 256;
constexpr int kMaxBlocks = 65536;
static __device__ __align__(256) unsigned long long g_partial[kMaxBlocks];

// device address of g_partial for the handle's device, looked up on the
// handle's first call with that device current and kept in the handle (a
// handle lives on one device; a handle created after a device reset looks the
// address up again)
std::mutex g_setup_mutex;

int partial_address(sulf_handle h, unsigned long long** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return sulf_fail_cuda(e, "cudaGetDevice");
    if (dev != handle_device(h))
        return sulf_fail(SULF_EINVAL, "sulf_newton_residual_noalloc: the current CUDA device is not the one the "
                                      "handle was created on");
    void** slot = handle_noalloc_slot(h);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!*slot) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_partial);
        if (e != cudaSuccess) return sulf_fail_cuda(e, "cudaGetSymbolAddress");
        *slot = p;
    }
    *out = static_cast<unsigned long long*>(*slot);
    return SULF_OK;
}

struct ResidualArgs {
    const int* l0;
    const int* l1;
    const int* lg;
    int n0, n1, ng;
    const int8_t* gm;
    const double* gw;
    long long st1, st2;
    double alpha, beta, amc, ams, idt, dh2, sb;
};

// gas-equation operator L^s_h(W) at an inside node (Sec. 3.3, flux sum over
// the axis neighbours with the 1/h^2 factor carried in dh2)
template <int D>
__device__ double gas_operator(long long p, const double2* __restrict__ W, const ResidualArgs& a) {
    const long long off[6] = {1, -1, a.st1, -a.st1, a.st2, -a.st2};
    double2 w = W[p];
    double ph = a.alpha * w.y + a.beta;
    double flux = 0.0;
#pragma unroll
    for (int q = 0; q < 2 * D; q++) {
        double2 wq = W[p + off[q]];
        flux += ((a.alpha * wq.y + a.beta) + ph) * (wq.x - w.x);
    }
    return -a.amc * ph * w.x * w.y + a.dh2 * flux;
}

// F of Eqs. FDs, FDc (inside; FDc also at ghosts) and BCs (ghost s rows) for
// every active node, old- and new-time parts evaluated together; each block
// stores the max |F| of its nodes in partial[blockIdx.x]
template <int D>
__global__ void __launch_bounds__(kThreads) k_residual_fused(ResidualArgs a, const double2* __restrict__ W,
                                                             const double2* __restrict__ Wn, double2* __restrict__ F,
                                                             unsigned long long* __restrict__ partial) {
    __shared__ unsigned long long wmax[kThreads / 32];
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long m = 0;
    if (t < a.n0 + a.n1 + a.ng) {
        long long p;
        bool inside = true;
        int gi = 0;
        if (t < a.n0) {
            p = a.l0[t];
        } else if (t < a.n0 + a.n1) {
            p = a.l1[t - a.n0];
        } else {
            gi = t - a.n0 - a.n1;
            p = a.lg[gi];
            inside = false;
        }
        double2 w = W[p], wn = Wn[p];
        double ph = a.alpha * w.y + a.beta, phn = a.alpha * wn.y + a.beta;
        double2 out;
        out.y = (w.y - wn.y) * a.idt + 0.5 * a.ams * (phn * wn.x * wn.y + ph * w.x * w.y);
        if (inside) {
            out.x = (ph * w.x - phn * wn.x) * a.idt - 0.5 * (gas_operator<D>(p, Wn, a) + gas_operator<D>(p, W, a));
        } else {
            // s~(B_g) - s_b: tensor-product weights on the upwind stencil
            const long long st[3] = {1, a.st1, a.st2};
            double acc = 0.0;
            const int K = D == 2 ? 9 : 27;
            for (int kk = 0; kk < K; kk++) {
                int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
                double wt = 1.0;
                long long node = p;
                for (int ax = 0; ax < D; ax++) {
                    wt *= a.gw[(long long)gi * 3 * D + 3 * ax + k[ax]];
                    node -= (long long)a.gm[(long long)gi * D + ax] * k[ax] * st[ax];
                }
                if (wt != 0.0) acc += wt * W[node].x;
            }
            out.x = acc - a.sb;
        }
        F[p] = out;
        unsigned long long b0 = (unsigned long long)__double_as_longlong(fabs(out.x));
        unsigned long long b1 = (unsigned long long)__double_as_longlong(fabs(out.y));
        m = b0 > b1 ? b0 : b1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int k = 0; k < kThreads / 32; k++) b = wmax[k] > b ? wmax[k] : b;
        partial[blockIdx.x] = b;  // every block writes its slot: nothing needs clearing
    }
}

// second pass: max over the nblocks partials into the caller's output
__global__ void __launch_bounds__(1024) k_partial_max(const unsigned long long* __restrict__ partial, int nblocks,
                                                      double* __restrict__ out) {
    __shared__ unsigned long long wmax[32];
    unsigned long long m = 0;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) m = partial[i] > m ? partial[i] : m;
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_down_sync(0xffffffffu, m, o);
        m = v > m ? v : m;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long b = 0;
        for (int k = 0; k < (int)(blockDim.x + 31) / 32; k++) b = wmax[k] > b ? wmax[k] : b;
        *out = __longlong_as_double((long long)b);
    }
}

}  // namespace

extern "C" int sulf_newton_residual_noalloc(sulf_handle h, double dt, const double* W_dev, const double* Wn_dev,
                                            double* F_dev, double* fnorm_dev) {
    const LevelGeo* G = handle_fine_geo(h);
    const sulf_model* m = handle_model(h);
    if (!G || !m || !W_dev || !Wn_dev || !F_dev || !fnorm_dev || !(dt > 0))
        return sulf_fail(SULF_EINVAL, "invalid arguments");
    if (handle_bc(h) != 0)
        return sulf_fail(SULF_EINVAL, "sulf_newton_residual_noalloc evaluates Dirichlet boundary rows only");
    // the kernel moves each node's (s, c) pair with one 16-byte access
    auto misaligned = [](const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) != 0; };
    if (misaligned(W_dev, 16) || misaligned(Wn_dev, 16) || misaligned(F_dev, 16) || misaligned(fnorm_dev, 8))
        return sulf_fail(SULF_EINVAL, "sulf_newton_residual_noalloc: W_dev, Wn_dev and F_dev must be 16-byte "
                                      "aligned and fnorm_dev 8-byte aligned");
    long long nact = (long long)G->nin[0] + G->nin[1] + G->ng;
    long long nblocks = (nact + kThreads - 1) / kThreads;
    if (nblocks > kMaxBlocks)
        return sulf_fail(SULF_EINVAL, "sulf_newton_residual_noalloc: more than 16777216 active nodes (its scratch "
                                      "holds 65536 partial maxima of 256 nodes each)");
    if (nblocks < 1) nblocks = 1;
    unsigned long long* partial = nullptr;
    int rc = partial_address(h, &partial);
    if (rc) return rc;
    ResidualArgs a;
    a.l0 = G->inl[0];
    a.l1 = G->inl[1];
    a.lg = G->gidx;
    a.n0 = G->nin[0];
    a.n1 = G->nin[1];
    a.ng = G->ng;
    a.gm = G->gm;
    a.gw = G->gw;
    a.st1 = G->st[1];
    a.st2 = G->st[2];
    a.alpha = m->alpha;
    a.beta = m->beta;
    a.amc = m->a / m->m_c;
    a.ams = m->a / m->m_s;
    a.idt = 1.0 / dt;
    a.dh2 = m->d / (2.0 * G->h * G->h);
    a.sb = m->s_ext;
    cudaStream_t s = handle_stream(h);
    const double2* W = reinterpret_cast<const double2*>(W_dev);
    const double2* Wn = reinterpret_cast<const double2*>(Wn_dev);
    double2* F = reinterpret_cast<double2*>(F_dev);
    if (G->dim == 2)
        k_residual_fused<2><<<(unsigned)nblocks, kThreads, 0, s>>>(a, W, Wn, F, partial);
    else
        k_residual_fused<3><<<(unsigned)nblocks, kThreads, 0, s>>>(a, W, Wn, F, partial);
    k_partial_max<<<1, 1024, 0, s>>>(partial, (int)nblocks, fnorm_dev);
    handle_count_launches(h, 2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sulf_fail_cuda(e, "sulf_newton_residual_noalloc launch");
    return SULF_OK;
}
