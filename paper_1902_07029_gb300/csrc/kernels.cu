// Newton and multigrid kernels of one Crank-Nicolson step (arXiv:1902.07029,
// Sec. 3.1, 3.4, 3.5), templated on the dimension D (2 or 3) and the precision
// T of the multigrid arithmetic (double, or float inside FP64 defect
// correction).  The Newton residual F and the update always run in FP64.
//
// The Jacobian is stored as stencil coefficients (Eqs. JssI, JscI, JcsI, JccI
// as exact derivatives of F), refreshed once per Newton iteration by k_coefs:
// per node the edge pair (g, e) toward each +axis neighbour and the inverse of
// the 2x2 diagonal block, per ghost its c row.  Each relaxation is then a
// handful of loads and fused multiply-adds per node.  The blocks and the FP64
// right-hand side are also kept in inside-list order, which is the order the
// colour sweeps and the residual visit nodes in.
#include <atomic>
#include <mutex>

#include <cooperative_groups.h>

#include "mg_stages.cuh"

namespace sulf {

using stages::abs_bits;
using stages::coef_ptr;
using stages::CoefPtr;
using stages::GhostTab;
using stages::list_node;
using stages::Lists;
using stages::make_lists;

namespace {
thread_local bool t_pdl = false;
thread_local int t_occ = 0;
thread_local int t_mf = 0;
thread_local std::string t_launch_err;
}  // namespace

void set_launch_pdl(bool on) { t_pdl = on; }
bool launch_pdl() { return t_pdl; }
void set_launch_occupancy(int occ) { t_occ = occ; }
int launch_occupancy() { return t_occ; }
void set_launch_matrix_free(int mf) { t_mf = mf; }
int launch_matrix_free() { return t_mf; }

void note_launch_error(cudaError_t e, unsigned grid, unsigned block, size_t smem) {
    if (!t_launch_err.empty()) return;
    t_launch_err = std::string(cudaGetErrorString(e)) + " (grid " + std::to_string(grid) + ", block " +
                   std::to_string(block) + ", smem " + std::to_string(smem) + (t_pdl ? ", dependent launch)" : ")");
}

std::string take_launch_error() {
    std::string m;
    m.swap(t_launch_err);
    return m;
}

namespace {

constexpr int kT = 256;

// Launch shape of a one-thread-per-node kernel over n nodes.  On this GPU one
// SM issues two FP64 lanes per clock, so a short list in 256-thread CTAs would
// run on a few SMs at their FP64 rate: CTAs shrink (down to one warp) until the
// list covers every SM, and grow to kT threads only for long lists.
int sm_count() {
    static std::atomic<int> cached[64];
    int dev = 0;
    cudaGetDevice(&dev);
    int v = (dev >= 0 && dev < 64) ? cached[dev].load(std::memory_order_relaxed) : 0;
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
    if (dev >= 0 && dev < 64) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

inline unsigned block_for(long long n) {
    const long long sms = sm_count();
    long long per = (n + sms - 1) / sms;
    long long b = (per + 31) / 32 * 32;
    return (unsigned)(b < 32 ? 32 : (b > kT ? kT : b));
}

inline unsigned grid_for(long long n) {
    const unsigned b = block_for(n);
    return (unsigned)((n + b - 1) / b);
}

// max over the block of non-negative doubles held as bit patterns (NaN, whose
// pattern exceeds +inf, propagates), then one atomicMax per block
__device__ __forceinline__ void block_max(unsigned long long v, unsigned long long* out) {
    __shared__ unsigned long long sm[32];
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
        v = v > w ? v : w;
    }
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int nw = (blockDim.x + 31) >> 5;
        v = lane < nw ? sm[lane] : 0ULL;
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
            v = v > w ? v : w;
        }
        if (lane == 0 && v) atomicMax(out, v);
    }
}

template <int D>
struct Offs {
    long long o[2 * D];
};

template <int D>
__host__ __device__ inline Offs<D> make_offs(long long st1, long long st2) {
    Offs<D> f;
    f.o[0] = 1;
    f.o[1] = -1;
    f.o[2] = st1;
    f.o[3] = -st1;
    if (D == 3) {
        f.o[4 % (2 * D)] = st2;
        f.o[5 % (2 * D)] = -st2;
    }
    return f;
}

// stencil coefficients of every active node from Wc: edges toward the +axis
// neighbours, and the 2x2 diagonal block and its inverse (inside; in box order
// and at the node's list position) or the c row (ghost).  Sec. 3.4: J^ss_pp = phi/dt + (a/2m_c) phi c + sum g,
// J^sc_pp = alpha s/dt + (a/2m_c)(alpha s c + phi s) + sum e,
// J^cs_pp = (a/2m_s) phi c, J^cc_pp = 1/dt + (a/2m_s)(alpha s c + phi s).
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_coefs(Lists ls, int n, const typename V2<T>::t* __restrict__ Wc,
                                               typename V2<T>::t* e0, typename V2<T>::t* e1, typename V2<T>::t* e2,
                                               typename V2<T>::t* Pa, typename V2<T>::t* Pb, typename V2<T>::t* Ia,
                                               typename V2<T>::t* Ib, typename V2<T>::t* Pc, typename V2<T>::t* Ic,
                                               typename V2<T>::t* gc, T* gci, Coef<T> c) {
    pdl_enter();
    typedef typename V2<T>::t T2;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi = 0;
    long long p = list_node(ls, t, kind, gi);
    const long long st[3] = {1, n, (long long)n * n};
    int ii[3];
    stages::box_coords<D>(p, n, ii);
    T2* edge[3] = {e0, e1, e2};
    T2 w = Wc[p];
    T s = w.x, cp = w.y;
    T ph = c.alpha * cp + c.beta;
    T sg = 0, se = 0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        if (ii[a] < n - 1) {
            T2 wq = Wc[p + st[a]];
            T2 ge;
            ge.x = c.kap * ((c.alpha * wq.y + c.beta) + ph);
            ge.y = c.kap * c.alpha * (s - wq.x);
            edge[a][p] = ge;
            sg += ge.x;
            se += ge.y;
        }
        if (kind == 1) {  // inside nodes are never on the box edge
            T2 wq = Wc[p - st[a]];
            sg += c.kap * ((c.alpha * wq.y + c.beta) + ph);
            se += c.kap * c.alpha * (s - wq.x);
        }
    }
    T Pcs = c.a2ms * ph * cp;
    T Pcc = c.idt + c.a2ms * (c.alpha * s * cp + ph * s);
    if (kind == 1) {
        T Pss = ph * c.idt + c.a2mc * ph * cp + sg;
        T Psc = c.alpha * s * c.idt + c.a2mc * (c.alpha * s * cp + ph * s) + se;
        T inv = (T)1 / (Pss * Pcc - Psc * Pcs);
        // box order and list order (t is the node's inside-list position)
        T2 v;
        v.x = Pss;
        v.y = Psc;
        Pa[p] = v;
        Pc[2 * (long long)t] = v;
        v.x = Pcs;
        v.y = Pcc;
        Pb[p] = v;
        Pc[2 * (long long)t + 1] = v;
        v.x = Pcc * inv;
        v.y = -Psc * inv;
        Ia[p] = v;
        Ic[2 * (long long)t] = v;
        v.x = -Pcs * inv;
        v.y = Pss * inv;
        Ib[p] = v;
        Ic[2 * (long long)t + 1] = v;
    } else {
        T2 v;
        v.x = Pcs;
        v.y = Pcc;
        gc[gi] = v;
        gci[gi] = (T)1 / Pcc;
    }
}

// ---------------------------------------------------------------------------
// relaxation (Sec. 3.5.1)

// one colour of inside nodes; with snap_n > 0 also the copy of the ghosts' s
// (nodes sidx) into snap that the composed ghost relaxation starts from
// (t0: the position of the colour's list in the concatenated inside lists)
template <int D, typename T, bool PW>
__global__ void __launch_bounds__(kT) k_relax_inside(const int* __restrict__ list, int cnt, int t0, CoefPtr<D, T> cf,
                                                      const typename V2<T>::t* __restrict__ rhs,
                                                      const typename V2<T>::t* __restrict__ rhsc,
                                                      typename V2<T>::t* __restrict__ x, long long st1, long long st2,
                                                      const int* __restrict__ sidx, int snap_n, T* snap) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const long long st[3] = {1, st1, st2};
    // the list and the stencil coefficients are fixed during the linear solve:
    // fetch them while the previous kernel is still running
    long long p = 0;
    stages::InsideCoef<D, T> k;
    if (t < cnt) {
        p = list[t];
        k = stages::fetch_inside_at<D, T, PW>(p, t0 + t, cf, st);
    }
    const int sg = t < snap_n ? sidx[t] : 0;
    pdl_enter();
    if (t < snap_n) snap[t] = reinterpret_cast<const T*>(x + sg)[0];
    if (t >= cnt) return;
    stages::relax_apply_b<D, T, PW, false>(p, k, rhsc ? rhsc[t0 + t] : rhs[p], x, st);
}

// The variant for large levels, where all but the first wave of CTAs start
// after the predecessor has finished anyway: the coefficients are loaded
// after the dependent-launch wait instead of held in registers across it,
// and the register budget is set for six resident CTAs per SM (more warps to
// hide the load latency); sulf_solver::relax_occupancy, FP64 collective only
template <int D, typename T>
__global__ void __launch_bounds__(kT, 6) k_relax_inside_ho(const int* __restrict__ list, int cnt, int t0,
                                                            CoefPtr<D, T> cf, const typename V2<T>::t* __restrict__ rhs,
                                                            const typename V2<T>::t* __restrict__ rhsc,
                                                            typename V2<T>::t* __restrict__ x, long long st1,
                                                            long long st2, const int* __restrict__ sidx, int snap_n,
                                                            T* snap) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const long long st[3] = {1, st1, st2};
    const long long p = t < cnt ? list[t] : 0;
    const int sg = t < snap_n ? sidx[t] : 0;
    pdl_enter();
    if (t < snap_n) snap[t] = reinterpret_cast<const T*>(x + sg)[0];
    if (t >= cnt) return;
    const stages::InsideCoef<D, T> k = stages::fetch_inside_at<D, T, false>(p, t0 + t, cf, st);
    stages::relax_apply_b<D, T, false, false>(p, k, rhsc ? rhsc[t0 + t] : rhs[p], x, st);
}

// lexicographic collective Gauss-Seidel (Sec. 3.5.1, the paper's smoother):
// one CTA walks the wavefronts i+j(+k) = const in increasing order; the
// nodes of one wavefront are independent, and when a node is updated its
// lower axis neighbours (previous wavefront) hold new values and its upper
// ones old values, as in a sweep in box order.  Values written in one
// wavefront are read in the next through L2 (ld.global.cg).
constexpr int kLexThreads = 512;
template <int D, typename T>
__global__ void __launch_bounds__(kLexThreads) k_relax_lex(const int* __restrict__ lex, const int* __restrict__ ptr,
                                                            int nd, CoefPtr<D, T> cf,
                                                            const typename V2<T>::t* __restrict__ rhs,
                                                            typename V2<T>::t* x, long long st1, long long st2,
                                                            const int* __restrict__ sidx, int snap_n, T* snap) {
    const long long st[3] = {1, st1, st2};
    pdl_enter();
    for (int dg = 0; dg < nd; dg++) {
        const int a = ptr[dg], b = ptr[dg + 1];
        for (int i = a + threadIdx.x; i < b; i += blockDim.x)
            stages::relax_node<D, T, false, true>(lex[i], cf, rhs, x, st);
        __syncthreads();
    }
    for (int i = threadIdx.x; i < snap_n; i += blockDim.x) snap[i] = __ldcg(reinterpret_cast<const T*>(x + sidx[i]));
}

// FP32 collective update with the stencil coefficients recomputed from the
// coefficient source Wc, with the expressions and summation order of k_coefs
// (so the same numbers as the stored ones): FP32 arithmetic is plentiful on
// this GPU while bytes are not, and per update this reads the (s, c) and x of
// the node and its axis neighbours and the right-hand side -- no edge, block
// or inverse arrays.  Wc is fixed during the linear solve, so the
// coefficients are formed before the dependent-launch wait.
template <int D>
__global__ void __launch_bounds__(kT) k_relax_mf(const int* __restrict__ list, int cnt,
                                                  const float2* __restrict__ Wc, const float2* __restrict__ rhs,
                                                  float2* __restrict__ x, Coef<float> c, long long st1, long long st2,
                                                  const int* __restrict__ sidx, int snap_n, float* snap) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const long long st[3] = {1, st1, st2};
    long long p = 0;
    stages::MfCoef<D> k;
    if (t < cnt) {
        p = list[t];
        k = stages::mf_coef<D>(p, Wc, c, st);
    }
    const int sg = t < snap_n ? sidx[t] : 0;
    pdl_enter();
    if (t < snap_n) snap[t] = reinterpret_cast<const float*>(x + sg)[0];
    if (t >= cnt) return;
    stages::mf_apply<D>(p, k, rhs, x, st);
}

// ---------------------------------------------------------------------------
// One whole red-black sweep of the FP32 collective smoother (both colours)
// in one kernel, temporally blocked in shared memory (3-D levels of the mixed
// form).  A CTA owns a tile of kTileX x kTileY nodes in (x, y) and kTileZ
// planes in z, and streams through z with a four-plane ring in shared
// memory: plane z+1 is staged (x, the coefficient source (s, c) and the node
// types of the tile and a two-node halo), the red nodes of plane z are
// updated over the tile and a one-node ring (the ring's updates, which the
// neighbouring tile owns, are recomputed here from the old black values so
// that no tile waits for another), then the black nodes of plane z-1 over
// the tile from those red values.  The stencil coefficients are recomputed
// from (s, c) with the expressions and order of k_relax_mf / k_coefs, so every
// update equals the two colour launches'.  x is read from xin and written to
// xout (a neighbour tile may still be reading the old values); ghosts are
// copied across and their s also into snap (the composed ghost relaxation
// starts from it).  Only inside nodes and ghosts of xout are defined after the
// sweep, which is all that any later stage reads.
constexpr int kTileX = 32, kTileY = 8, kTileZ = 16;
constexpr int kTileRX = kTileX + 4, kTileRY = kTileY + 4, kTileRN = kTileRX * kTileRY;
constexpr int kTileThreads = 256;

// the collective update of the node at ring position r of slot sl, its
// neighbour values in X (slots of planes z-1, z, z+1), coefficients from W
__device__ __forceinline__ float2 tile_update(const float2 (*X)[kTileRN], const float2 (*W)[kTileRN], int sl, int r,
                                              int zl, int zh, float2 b, const Coef<float>& c) {
    const float2 w = W[sl][r];
    const float s = w.x, cp = w.y;
    const float ph = c.alpha * cp + c.beta;
    // neighbours in the order +x, -x, +y, -y, +z, -z (as k_relax_mf)
    const int ns[6] = {sl, sl, sl, sl, zh, zl};
    const int nr[6] = {r + 1, r - 1, r + kTileRX, r - kTileRX, r, r};
    float g[6], e[6];
    float sg = 0, se = 0;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const float2 wq = W[ns[q]][nr[q]];
        g[q] = c.kap * ((c.alpha * wq.y + c.beta) + ph);
        e[q] = c.kap * c.alpha * (s - wq.x);
        sg += g[q];
        se += e[q];
    }
    const float Pcs = c.a2ms * ph * cp;
    const float Pcc = c.idt + c.a2ms * (c.alpha * s * cp + ph * s);
    const float Pss = ph * c.idt + c.a2mc * ph * cp + sg;
    const float Psc = c.alpha * s * c.idt + c.a2mc * (c.alpha * s * cp + ph * s) + se;
    const float inv = 1.0f / (Pss * Pcc - Psc * Pcs);
    float r_s = b.x;
#pragma unroll
    for (int q = 0; q < 6; q++) {
        const float2 xq = X[ns[q]][nr[q]];
        r_s = __fmaf_rn(g[q], xq.x, r_s);
        r_s = __fmaf_rn(-e[q], xq.y, r_s);
    }
    float2 out;
    out.x = __fmaf_rn(Pcc * inv, r_s, (-Psc * inv) * b.y);
    out.y = __fmaf_rn(-Pcs * inv, r_s, (Pss * inv) * b.y);
    return out;
}

// the planes' staged data in the dynamic shared memory of k_sweep_tile
struct TileSmem {
    float2 XO[4][kTileRN];  // x before the sweep
    float2 XR[4][kTileRN];  // x after the red half (ring 1 and tile)
    float2 WS[4][kTileRN];  // coefficient source (s, c)
    float2 RH[4][kTileRN];  // right-hand side
    int8_t TS[4][kTileRN];  // node type
};
constexpr int kTilePer = (kTileRN + kTileThreads - 1) / kTileThreads;  // staged nodes per thread

// a thread's share of one plane (region with the two-node halo), fetched one
// iteration ahead of its use
struct TilePlane {
    float2 xo[kTilePer], wc[kTilePer], rh[kTilePer];
    int8_t ty[kTilePer];
};

__device__ __forceinline__ void tile_fetch(TilePlane& f, int zl, int X0, int Y0, int n, long long st1, long long st2,
                                           const int8_t* __restrict__ type, const float2* __restrict__ Wc,
                                           const float2* __restrict__ rhs, const float2* __restrict__ xin) {
#pragma unroll
    for (int k = 0; k < kTilePer; k++) {
        const int t = threadIdx.x + k * kTileThreads;
        const int gx = X0 - 2 + t % kTileRX, gy = Y0 - 2 + t / kTileRX;
        f.xo[k] = make_float2(0.f, 0.f);
        f.wc[k] = make_float2(0.f, 0.f);
        f.rh[k] = make_float2(0.f, 0.f);
        f.ty[k] = T_OUT;
        if (t < kTileRN && zl >= 0 && zl < n && gx >= 0 && gx < n && gy >= 0 && gy < n) {
            // every load issued at once (no dependence on the type): values at
            // inactive nodes are read but never used
            const long long p = gx + gy * st1 + zl * st2;
            f.ty[k] = type[p];
            f.xo[k] = xin[p];
            f.wc[k] = Wc[p];
            f.rh[k] = rhs[p];
        }
    }
}

__global__ void __launch_bounds__(kTileThreads) k_sweep_tile(const int* __restrict__ tiles, int ntx, int nty, int n,
                                                             const int8_t* __restrict__ type,
                                                             const float2* __restrict__ Wc,
                                                             const float2* __restrict__ rhs,
                                                             const float2* __restrict__ xin, float2* __restrict__ xout,
                                                             Coef<float> c, const int* __restrict__ gidx, int ng,
                                                             float* snap) {
    extern __shared__ __align__(16) unsigned char tile_smem[];
    TileSmem& S = *reinterpret_cast<TileSmem*>(tile_smem);
    const int tile = tiles[blockIdx.x];
    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const int X0 = tx * kTileX, Y0 = ty * kTileY, Z0 = tz * kTileZ;
    const long long st1 = n, st2 = (long long)n * n;
    pdl_enter();
    // the ghosts: unchanged by the inside sweep, copied to xout (and their s
    // to snap) by all CTAs together
    for (int gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ng; gi += gridDim.x * blockDim.x) {
        const int g = gidx[gi];
        const float2 v = xin[g];
        xout[g] = v;
        if (snap) snap[gi] = v.x;
    }
    TilePlane f;
    tile_fetch(f, Z0 - 2, X0, Y0, n, st1, st2, type, Wc, rhs, xin);
    for (int z = Z0 - 3; z <= Z0 + kTileZ; z++) {
        // plane z + 1 (fetched during the previous iteration) into its slot,
        // then the fetch of plane z + 2 starts
        {
            const int sl = (z + 1) & 3;
#pragma unroll
            for (int k = 0; k < kTilePer; k++) {
                const int t = threadIdx.x + k * kTileThreads;
                if (t < kTileRN) {
                    S.XO[sl][t] = f.xo[k];
                    S.WS[sl][t] = f.wc[k];
                    S.RH[sl][t] = f.rh[k];
                    S.TS[sl][t] = f.ty[k];
                }
            }
        }
        if (z + 2 <= Z0 + kTileZ + 1) tile_fetch(f, z + 2, X0, Y0, n, st1, st2, type, Wc, rhs, xin);
        __syncthreads();
        // red nodes of plane z over the tile and a one-node ring
        if (z >= Z0 - 1) {
            const int sl = z & 3, zl = (z - 1) & 3, zh = (z + 1) & 3;
            for (int t = threadIdx.x; t < (kTileX + 2) * (kTileY + 2); t += kTileThreads) {
                const int li = 1 + t % (kTileX + 2), lj = 1 + t / (kTileX + 2);
                const int r = li + lj * kTileRX;
                const int gx = X0 - 2 + li, gy = Y0 - 2 + lj;
                float2 v = S.XO[sl][r];
                if (S.TS[sl][r] == T_IN && ((gx + gy + z) & 1) == 0)
                    v = tile_update(S.XO, S.WS, sl, r, zl, zh, S.RH[sl][r], c);
                S.XR[sl][r] = v;
            }
        }
        __syncthreads();
        // black nodes of plane z - 1 over the tile; the tile's inside nodes
        // of that plane go to xout
        const int zb = z - 1;
        if (zb >= Z0 && zb < Z0 + kTileZ && zb < n) {
            const int sl = zb & 3, zl = (zb - 1) & 3, zh = (zb + 1) & 3;
            for (int t = threadIdx.x; t < kTileX * kTileY; t += kTileThreads) {
                const int li = 2 + t % kTileX, lj = 2 + t / kTileX;
                const int r = li + lj * kTileRX;
                const int gx = X0 - 2 + li, gy = Y0 - 2 + lj;
                if (gx >= n || gy >= n || S.TS[sl][r] != T_IN) continue;
                const long long p = gx + gy * st1 + zb * st2;
                float2 v = S.XR[sl][r];
                if (((gx + gy + zb) & 1) == 1) v = tile_update(S.XR, S.WS, sl, r, zl, zh, S.RH[sl][r], c);
                xout[p] = v;
            }
        }
        __syncthreads();
    }
}

// one Jacobi pass of the ghost relaxation of Eq. RelGhost over all ghosts
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_ghost_pass(const int* __restrict__ gidx, GhostTab<T> tb,
                                                    const typename V2<T>::t* __restrict__ gc,
                                                    const T* __restrict__ gci,
                                                    const typename V2<T>::t* __restrict__ rhs,
                                                    typename V2<T>::t* x, const T* sin, T* sout, Coef<T> c, int first,
                                                    int last) {
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = gi < tb.ng;
    // the boundary rows and the ghost c-row coefficients are fixed during the
    // linear solve: fetch them (in 2-D the whole member table of the row) while
    // the previous kernel is still running
    long long g = 0;
    typename V2<T>::t q;
    T qinv;
    stages::Members<T> m;
    if (on) {
        g = gidx[gi];
        q = gc[gi];
        qinv = gci[gi];
        if (D == 2) stages::fetch_members<T>(tb, gi, 0, m);
    }
    pdl_enter();
    if (!on) return;
    stages::ghost_pass_apply<D, T, false>(gi, g, tb, D == 2 ? &m : nullptr, q, qinv, rhs, x, sin, sout, c.tau,
                                          first != 0, last != 0);
}

// The ghost relaxation of one sweep as the composed map (geometry.cu): s_g =
// sum_j val_j u(code_j), u the s of an inside node (x), a ghost's s before the
// passes (snap) or a ghost's right-hand side; then the ghost's c row with the
// new s_g.  kGopLanes lanes share a row: the entries are fetched before the
// wait (they are fixed during the linear solve), so after it only one round of
// gathered loads and a lane reduction remain.
using stages::kGopLanes;
constexpr int kGopPre = 4;

template <typename T>
__global__ void __launch_bounds__(kT) k_ghost_op(int ng, const int* __restrict__ gidx, const int* __restrict__ ptr,
                                                  const int* __restrict__ code, const T* __restrict__ val,
                                                  const typename V2<T>::t* __restrict__ gc,
                                                  const T* __restrict__ gci, const typename V2<T>::t* rhs,
                                                  typename V2<T>::t* x, const T* snap) {
    typedef typename V2<T>::t T2;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int gi = t / kGopLanes, ln = t % kGopLanes;
    const bool on = gi < ng;
    int beg = 0, end = 0, g = 0;
    int cd[kGopPre];
    T w[kGopPre];
    T2 q;
    q.x = 0;
    q.y = 1;
    T qinv = 1;
    if (on) {
        beg = ptr[gi];
        end = ptr[gi + 1];
#pragma unroll
        for (int i = 0; i < kGopPre; i++) {
            const int j = beg + ln + i * kGopLanes;
            cd[i] = j < end ? code[j] : 0;
            w[i] = j < end ? val[j] : (T)0;
        }
        if (ln == 0) {
            g = gidx[gi];
            q = gc[gi];
            qinv = gci[gi];
        }
    }
    pdl_enter();
    auto u = [&](int c) -> T { return stages::gop_input<T>(c, x, rhs, snap); };
    const T by = on && ln == 0 ? reinterpret_cast<const T*>(rhs + g)[1] : (T)0;
    T acc = 0;
    if (on) {
        T v[kGopPre];
#pragma unroll
        for (int i = 0; i < kGopPre; i++) v[i] = beg + ln + i * kGopLanes < end ? u(cd[i]) : (T)0;
#pragma unroll
        for (int i = 0; i < kGopPre; i++) acc = stages::fmadd(w[i], v[i], acc);
        for (int j = beg + ln + kGopPre * kGopLanes; j < end; j += kGopLanes) acc = stages::fmadd(val[j], u(code[j]), acc);
    }
    acc = stages::gop_reduce<T>(acc);
    if (!on || ln != 0) return;
    T2 r;
    r.x = acc;
    r.y = stages::fmadd(-q.x, acc, by) * qinv;
    x[g] = r;
}

template <typename T>
__global__ void k_ghost_scatter(int ng, const int* __restrict__ gidx, const T* __restrict__ sin,
                                typename V2<T>::t* x) {
    pdl_enter();
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    reinterpret_cast<T*>(x + gidx[gi])[0] = sin[gi];
}

// ---------------------------------------------------------------------------
// defect r = rhs - J x on every active node, with its max-norm

// (R2: the element type the defect is stored in; an FP64 defect stored into
// FP32 is the next right-hand side of the mixed form's FP32 cycle)
template <int D, typename T, typename R2>
__global__ void __launch_bounds__(kT) k_residual(Lists ls, GhostTab<T> tb, CoefPtr<D, T> cf,
                                                  const typename V2<T>::t* __restrict__ rhs,
                                                  const typename V2<T>::t* __restrict__ x, R2* __restrict__ res,
                                                  long long st1, long long st2, unsigned long long* norm,
                                                  const typename V2<T>::t* __restrict__ rhsc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = t < ls.n0 + ls.n1 + ls.ng;
    // lists, coefficients and ghost rows are fixed during the linear solve:
    // fetched ahead
    int kind = 0, gi = 0;
    long long p = 0;
    stages::InsideCoef<D, T> k;
    stages::Members<T> m;
    typename V2<T>::t q;
    if (on) p = stages::fetch_residual<D, T>(t, ls, tb, cf, st1, st2, kind, gi, k, m, q);
    pdl_enter();
    unsigned long long nb = 0;
    if (on)
        nb = stages::residual_apply<D, T, false>(p, kind, gi, k, tb, D == 2 ? &m : nullptr, q, rhs, x, res, st1,
                                                 st2, rhsc, t);
    if (norm) block_max(nb, norm);
}

// ---------------------------------------------------------------------------
// extension of the ghost defect into the band along the normal (Sec. 3.5.2),
// the explicit upwind steps applied as one precomputed linear operator

template <typename T>
__global__ void k_extend(int nb, const int* __restrict__ eptr, const int* __restrict__ eidx,
                         const T* __restrict__ eval, const int* __restrict__ bidx, typename V2<T>::t* res) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    stages::ExtRow<T> r;
    if (b < nb) r = stages::fetch_ext<T>(b, eptr, eidx, eval, bidx);  // fixed operator, fetched ahead
    pdl_enter();
    if (b >= nb) return;
    stages::extend_apply<T, false>(r, eidx, eval, res);
}

// ---------------------------------------------------------------------------
// boundary-aware full weighting (Eqs. Fstencil, Fstencilgen, Fig. Neigh):
// inside rule at coarse inside nodes, outside rule (ghost or band) at coarse
// ghosts; per-axis mirrored weights, invalid diagonal weight moved to the
// centre.  Also zeroes the coarse error at the coarse active nodes.
// first_red: the coarse level's first relaxation starts from this zero
// error, and its red half-sweep (which then reads only zeros) is done here
// for the red inside nodes (list positions below ls.n0)
template <int D, typename T, bool PW>
__global__ void __launch_bounds__(kT) k_restrict(Lists ls, const int8_t* __restrict__ ctype, int cn,
                                                  const int8_t* __restrict__ ftype, int fn,
                                                  const typename V2<T>::t* __restrict__ fres,
                                                  typename V2<T>::t* __restrict__ crhs,
                                                  typename V2<T>::t* __restrict__ cx, CoefPtr<D, T> ccf,
                                                  int first_red, typename V2<T>::t* __restrict__ crhsc) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = t < ls.n0 + ls.n1 + ls.ng;
    const bool red = on && first_red && t < ls.n0;
    stages::RestrictGeo<D, T> g;
    stages::InsideCoef<D, T> k;
    if (on) g = stages::fetch_restrict<D, T>(t, ls, ctype, cn, ftype, fn);  // fixed geometry, fetched ahead
    if (red) {
        const long long cst[3] = {1, cn, (long long)cn * cn};
        k = stages::fetch_inside_at<D, T, PW>(g.I, t, ccf, cst);  // fixed coefficients, fetched ahead
    }
    pdl_enter();
    if (!on) return;
    stages::restrict_apply<D, T, false, PW>(g, fn, fres, crhs, cx, red ? &k : nullptr, crhsc, t);
}

// (bi/tri)linear interpolation of the coarse error to every fine active node,
// renormalised over the coarse active nodes (Sec. 3.5.3)
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_prolong(Lists ls, const int8_t* __restrict__ ctype, int cn,
                                                 const typename V2<T>::t* __restrict__ cx, int fn,
                                                 typename V2<T>::t* __restrict__ fx) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool on = t < ls.n0 + ls.n1 + ls.ng;
    stages::ProlongGeo<D, T> g;
    if (on) g = stages::fetch_prolong<D, T>(t, ls, ctype, cn, fn);  // fixed geometry, fetched ahead
    pdl_enter();
    if (!on) return;
    stages::prolong_apply<D, T, false>(g, fn, cx, fx);
}

// coarse Jacobian coefficients by injection of (s, c); a coarse ghost whose
// fine twin is inactive takes the mean over the active fine 3^d neighbourhood
template <int D, typename T>
__global__ void __launch_bounds__(kT) k_inject(Lists ls, int cn, const int8_t* __restrict__ ftype, int fn,
                                                const typename V2<T>::t* __restrict__ fW,
                                                typename V2<T>::t* __restrict__ cW) {
    pdl_enter();
    typedef typename V2<T>::t T2;
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi;
    long long I = list_node(ls, t, kind, gi);
    int ii[3];
    stages::box_coords<D>(I, cn, ii);
    long long fst[3] = {1, fn, (long long)fn * fn};
    long long f = 0;
#pragma unroll
    for (int a = 0; a < D; a++) f += 2LL * ii[a] * fst[a];
    int8_t tf = ftype[f];
    if (tf == T_IN || tf == T_GHOST) {
        cW[I] = fW[f];
        return;
    }
    T ss = 0, sc = 0;
    int cnt = 0;
    const int K = D == 2 ? 9 : 27;
    for (int kk = 0; kk < K; kk++) {
        int k[3] = {kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1};
        bool ok = true;
        long long node = f;
        for (int a = 0; a < D; a++) {
            int ia = 2 * ii[a] + k[a];
            if (ia < 0 || ia > fn - 1) ok = false;
            node += k[a] * fst[a];
        }
        if (!ok) continue;
        int8_t tn = ftype[node];
        if (tn != T_IN && tn != T_GHOST) continue;
        T2 v = fW[node];
        ss += v.x;
        sc += v.y;
        cnt++;
    }
    T2 out;
    out.x = cnt ? ss / (T)cnt : (T)0;
    out.y = cnt ? sc / (T)cnt : (T)0;
    cW[I] = out;
}

// ---------------------------------------------------------------------------
// coarsest level: assemble the Jacobian and invert it by Gauss-Jordan
// elimination with partial pivoting (one CTA, once per Newton iteration); each
// cycle then applies the inverse

template <int D, typename T, bool SMEM>
__global__ void __launch_bounds__(1024) k_coarsest_factor(int nact, const int* __restrict__ act,
                                                          const int* __restrict__ apos, const int8_t* __restrict__ type,
                                                          const int* __restrict__ gpos, GhostTab<T> tb,
                                                          const typename V2<T>::t* __restrict__ Wc, Offs<D> of,
                                                          long long st1, long long st2, Coef<T> c, T* Ag, T* Ainv_g,
                                                          int* singular) {
    pdl_enter();
    typedef typename V2<T>::t T2;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = 2 * nact;
    const long long mm = (long long)m * m;
    // with SMEM the matrix is inverted in shared memory (small coarsest
    // levels) and copied out at the end; otherwise in place in Ag
    T* A = SMEM ? reinterpret_cast<T*>(smem_raw) : Ag;
    T* fac = reinterpret_cast<T*>(smem_raw + (SMEM ? mm * sizeof(T) : 0));  // column k of the current step
    int* piv = reinterpret_cast<int*>(fac + m + 1);                        // row interchanges
    for (long long i = threadIdx.x; i < mm; i += blockDim.x) A[i] = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nact; r += blockDim.x) {
        long long p = act[r];
        T2 w = Wc[p];
        T s = w.x, cp = w.y;
        T ph = c.alpha * cp + c.beta;
        T* rs = A + (long long)(2 * r) * m;
        T* rc = A + (long long)(2 * r + 1) * m;
        if (type[p] == T_IN) {
            T ss = ph * c.idt + c.a2mc * ph * cp;
            T sc = c.alpha * s * c.idt + c.a2mc * (c.alpha * s * cp + ph * s);
            for (int q = 0; q < 2 * D; q++) {
                long long pq = p + of.o[q];
                T2 wq = Wc[pq];
                T g = c.kap * ((c.alpha * wq.y + c.beta) + ph);
                T e = c.kap * c.alpha * (s - wq.x);
                int qc = apos[pq];
                rs[2 * qc] += -g;
                rs[2 * qc + 1] += e;
                ss += g;
                sc += e;
            }
            rs[2 * r] += ss;
            rs[2 * r + 1] += sc;
        } else {
            // the ghost's boundary row from its member table (Dirichlet or Neumann)
            int gi = gpos[p];
            const int K = D == 2 ? 9 : 27;
            for (int kk = 0; kk < K; kk++) {
                const long long o = (long long)kk * tb.ng + gi;
                T wt = tb.w[o];
                if (wt == (T)0) continue;
                rs[2 * apos[tb.node[o]]] += wt;
            }
        }
        rc[2 * r] += c.a2ms * ph * cp;
        rc[2 * r + 1] += c.idt + c.a2ms * (c.alpha * s * cp + ph * s);
    }
    __syncthreads();
    // In-place Gauss-Jordan inversion with partial pivoting (first row of
    // largest |a_ik|, i >= k, as an LU with partial pivoting would choose):
    // step k scales the pivot row by 1/a_kk and eliminates column k from every
    // other row, storing -a_ik/a_kk in column k; this inverts P A, and the
    // column interchanges applied in reverse order at the end give A^{-1}.
    // About m^3 fused multiply-adds (half of eliminating on [A | I]); threads
    // own fixed columns and stride over rows, so the inner loop carries no
    // index division.
    __shared__ int s_piv;
    const int W = m < (int)blockDim.x ? m : (int)blockDim.x;
    const int R = (int)blockDim.x / W;
    const int jt = (int)threadIdx.x % W, rt = (int)threadIdx.x / W;
    __syncthreads();
    for (int k = 0; k < m; k++) {
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            T bv = -1;
            int bi = k;
            for (int i = k + lane; i < m; i += 32) {
                T v = fabs(A[(long long)i * m + k]);
                if (v > bv) {
                    bv = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                T ov = __shfl_down_sync(0xffffffffu, bv, o);
                int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > bv || (ov == bv && oi < bi)) {
                    bv = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                s_piv = bi;
                piv[k] = bi;
                if (!(bv > (T)0)) *singular = 1;
            }
        }
        __syncthreads();
        const int pr = s_piv;
        if (pr != k)
            for (int j = threadIdx.x; j < m; j += blockDim.x) {
                T tmp = A[(long long)k * m + j];
                A[(long long)k * m + j] = A[(long long)pr * m + j];
                A[(long long)pr * m + j] = tmp;
            }
        __syncthreads();
        // the pivot's reciprocal once (every thread dividing would load the
        // FP64 pipe, two lanes per SM per clock)
        if (threadIdx.x == 0) fac[m] = (T)1 / A[(long long)k * m + k];
        for (int i = threadIdx.x; i < m; i += blockDim.x) fac[i] = A[(long long)i * m + k];
        __syncthreads();
        const T inv = fac[m];
        for (int j = threadIdx.x; j < m; j += blockDim.x)
            A[(long long)k * m + j] = j == k ? inv : A[(long long)k * m + j] * inv;
        __syncthreads();
        if (rt < R)
            for (int j = jt; j < m; j += W) {
                if (j == k) continue;
                const T akj = A[(long long)k * m + j];
                for (int i = rt; i < m; i += R) {
                    if (i == k) continue;
                    A[(long long)i * m + j] -= fac[i] * akj;
                }
            }
        __syncthreads();
        for (int i = threadIdx.x; i < m; i += blockDim.x)
            if (i != k) A[(long long)i * m + k] = -fac[i] * inv;
        __syncthreads();
    }
    // undo the row interchanges as column interchanges, last first
    for (int k = m - 1; k >= 0; k--) {
        const int pr = piv[k];
        if (pr != k)
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                T tmp = A[(long long)i * m + k];
                A[(long long)i * m + k] = A[(long long)i * m + pr];
                A[(long long)i * m + pr] = tmp;
            }
        __syncthreads();
    }
    for (long long i = threadIdx.x; i < mm; i += blockDim.x) Ainv_g[i] = A[i];
}

// The same assembly and Gauss-Jordan inversion spread over a thread-block
// cluster: CTA r of C owns the columns j with j % C == r (m rows each, in its
// shared memory).  Step k: the owner of column k finds the pivot row in it and
// writes the column, after the row interchange, and the pivot row index into
// every CTA's shared memory (double-buffered by the parity of k); one cluster
// barrier; then each CTA interchanges, scales and eliminates in its own
// columns.  Every matrix entry sees the operations of the single-CTA kernel in
// the same order.  The inverse is written out with the final column
// permutation applied.
constexpr int kFacCluster = 8;
constexpr int kFacThreads = 512;

template <typename T>
inline size_t factor_cluster_smem(int m) {
    const size_t mc = ((size_t)m + kFacCluster - 1) / kFacCluster;
    return sizeof(T) * ((size_t)m * mc + 2 * ((size_t)m + 1)) + sizeof(int) * 3 * (size_t)m;
}

template <int D, typename T>
__global__ void __launch_bounds__(kFacThreads) k_coarsest_factor_cluster(
    int nact, const int* __restrict__ act, const int* __restrict__ apos, const int8_t* __restrict__ type,
    const int* __restrict__ gpos, GhostTab<T> tb, const typename V2<T>::t* __restrict__ Wc, Offs<D> of, Coef<T> c,
    T* Ainv_g, int* singular) {
    namespace cg = cooperative_groups;
    pdl_enter();
    typedef typename V2<T>::t T2;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int me = (int)cl.block_rank();
    const int m = 2 * nact;
    const int mc = (m + C - 1) / C;  // local column jl is global column jl * C + me
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* A = reinterpret_cast<T*>(smem_raw);  // m x mc, row-major
    T* fac = A + (size_t)m * mc;             // two buffers of m + 1
    int* piv = reinterpret_cast<int*>(fac + 2 * (m + 1));
    int* idx = piv + m;
    int* pos = idx + m;
    for (int i = threadIdx.x; i < m * mc; i += blockDim.x) A[i] = 0;
    __syncthreads();
    auto add = [&](int i, int j, T v) {
        if (j % C == me) A[(size_t)i * mc + j / C] += v;
    };
    for (int r = threadIdx.x; r < nact; r += blockDim.x) {
        long long p = act[r];
        T2 w = Wc[p];
        T s = w.x, cp = w.y;
        T ph = c.alpha * cp + c.beta;
        if (type[p] == T_IN) {
            T ss = ph * c.idt + c.a2mc * ph * cp;
            T sc = c.alpha * s * c.idt + c.a2mc * (c.alpha * s * cp + ph * s);
            for (int q = 0; q < 2 * D; q++) {
                long long pq = p + of.o[q];
                T2 wq = Wc[pq];
                T g = c.kap * ((c.alpha * wq.y + c.beta) + ph);
                T e = c.kap * c.alpha * (s - wq.x);
                int qc = apos[pq];
                add(2 * r, 2 * qc, -g);
                add(2 * r, 2 * qc + 1, e);
                ss += g;
                sc += e;
            }
            add(2 * r, 2 * r, ss);
            add(2 * r, 2 * r + 1, sc);
        } else {
            int gi = gpos[p];
            const int K = D == 2 ? 9 : 27;
            for (int kk = 0; kk < K; kk++) {
                const long long o = (long long)kk * tb.ng + gi;
                T wt = tb.w[o];
                if (wt == (T)0) continue;
                add(2 * r, 2 * apos[tb.node[o]], wt);
            }
        }
        add(2 * r + 1, 2 * r, c.a2ms * ph * cp);
        add(2 * r + 1, 2 * r + 1, c.idt + c.a2ms * (c.alpha * s * cp + ph * s));
    }
    __syncthreads();
    __shared__ int s_piv;
    __shared__ T s_inv;
    for (int k = 0; k < m; k++) {
        T* fb = fac + (size_t)(k & 1) * (m + 1);
        if (k % C == me) {
            const int kl = k / C;
            __syncthreads();  // this CTA's updates of column k in the previous step
            if (threadIdx.x < 32) {
                const int lane = threadIdx.x;
                T bv = -1;
                int bi = k;
                for (int i = k + lane; i < m; i += 32) {
                    T v = fabs(A[(size_t)i * mc + kl]);
                    if (v > bv) {
                        bv = v;
                        bi = i;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    T ov = __shfl_down_sync(0xffffffffu, bv, o);
                    int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ov > bv || (ov == bv && oi < bi)) {
                        bv = ov;
                        bi = oi;
                    }
                }
                if (lane == 0) {
                    s_piv = bi;
                    // the pivot's reciprocal once (every thread dividing
                    // would load the FP64 pipe, two lanes per SM per clock)
                    s_inv = (T)1 / A[(size_t)bi * mc + kl];
                    if (!(bv > (T)0)) *singular = 1;
                }
            }
            __syncthreads();
            const int pr = s_piv;
            for (int t = threadIdx.x; t < m * C; t += blockDim.x) {
                const int rk = t / m, i = t % m;
                const int src = i == k ? pr : (i == pr ? k : i);
                T* dst = cl.map_shared_rank(fb, rk);
                dst[i] = A[(size_t)src * mc + kl];
                if (i == 0) {
                    dst[m] = s_inv;
                    cl.map_shared_rank(piv, rk)[k] = pr;
                }
            }
        }
        cl.sync();  // column k, its reciprocal pivot and the pivot row in every CTA
        const int pr = piv[k];
        const T inv = fb[m];
        // interchange rows k and pr and scale row k, one local column per thread
        for (int jl = threadIdx.x; jl < mc; jl += blockDim.x) {
            const int j = jl * C + me;
            if (j >= m) continue;
            T rowk = A[(size_t)k * mc + jl];
            if (pr != k) {
                const T rowp = A[(size_t)pr * mc + jl];
                A[(size_t)pr * mc + jl] = rowk;
                rowk = rowp;
            }
            A[(size_t)k * mc + jl] = j == k ? inv : rowk * inv;
        }
        __syncthreads();
        // eliminate column k from every other row; column k itself (in its
        // owner) becomes -a_ik / a_kk
        for (int t = threadIdx.x; t < m * mc; t += blockDim.x) {
            const int i = t / mc, jl = t % mc;
            const int j = jl * C + me;
            if (i == k || j >= m) continue;
            if (j == k)
                A[(size_t)i * mc + jl] = -fb[i] * inv;
            else
                A[(size_t)i * mc + jl] -= fb[i] * A[(size_t)k * mc + jl];
        }
        // the next owner synchronises before its pivot search; every other
        // CTA meets the others at the next cluster barrier
    }
    __syncthreads();
    // the row interchanges undone as column interchanges, last first: final
    // column j is column idx[j] of the eliminated matrix
    if (threadIdx.x == 0) {
        for (int j = 0; j < m; j++) idx[j] = j;
        for (int k = m - 1; k >= 0; k--) {
            const int p = piv[k], t = idx[k];
            idx[k] = idx[p];
            idx[p] = t;
        }
        for (int j = 0; j < m; j++) pos[idx[j]] = j;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < m * mc; t += blockDim.x) {
        const int i = t / mc, jl = t % mc;
        const int j = jl * C + me;
        if (j < m) Ainv_g[(size_t)i * m + pos[j]] = A[(size_t)i * mc + jl];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_coarsest_solve(int nact, const int* __restrict__ act, const T* __restrict__ Ainv,
                                                         const typename V2<T>::t* __restrict__ rhs,
                                                         typename V2<T>::t* __restrict__ x) {
    pdl_enter();
    typedef typename V2<T>::t T2;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* b = reinterpret_cast<T*>(smraw);
    const int m = 2 * nact;
    for (int r = threadIdx.x; r < nact; r += blockDim.x) {
        T2 v = rhs[act[r]];
        b[2 * r] = v.x;
        b[2 * r + 1] = v.y;
    }
    __syncthreads();
    // one warp per row of the inverse, lanes over its columns; the rows are
    // spread over several CTAs (each warp-wide FP64 instruction costs 16
    // issue cycles of one SM)
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= m) return;
    const T* row = Ainv + (long long)r * m;
    T acc = 0;
    for (int j = lane; j < m; j += 32) acc += row[j] * b[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) reinterpret_cast<T*>(x + act[r >> 1])[r & 1] = acc;
}

// ---------------------------------------------------------------------------
// Newton residual (Eqs. FDs, FDc, BCs), FP64

template <int D>
__device__ __forceinline__ double Ls_h(long long p, const double2* __restrict__ W, const Offs<D>& of,
                                       const FConst& f, double& ph_out) {
    double2 w = W[p];
    double ph = f.alpha * w.y + f.beta;
    double flux = 0.0;
#pragma unroll
    for (int q = 0; q < 2 * D; q++) {
        double2 wq = W[p + of.o[q]];
        flux += ((f.alpha * wq.y + f.beta) + ph) * (wq.x - w.x);
    }
    ph_out = ph;
    return -f.amc * ph * w.x * w.y + f.dh2 * flux;
}

// old-time part G = -M(W^n)/dt - L(W^n)/2 of the CN step (once per step)
template <int D>
__global__ void __launch_bounds__(kT) k_old_time(Lists ls, const double2* __restrict__ Wn, double2* __restrict__ G,
                                                  Offs<D> of, FConst f) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi;
    long long p = list_node(ls, t, kind, gi);
    double2 w = Wn[p];
    double ph = f.alpha * w.y + f.beta;
    double Lc = -f.ams * ph * w.x * w.y;
    double2 g;
    g.y = -w.y * f.idt - 0.5 * Lc;
    g.x = 0.0;
    if (kind == 1) {
        double phd;
        double Ls = Ls_h<D>(p, Wn, of, f, phd);
        g.x = -ph * w.x * f.idt - 0.5 * Ls;
    }
    if (f.src) {  // manufactured sources: F^s -= (f1o + f1n)/2 inside, F^c -= (f2o + f2n)/2
        double2 q = f.src[p];
        if (kind == 1) g.x -= q.x;
        g.y -= q.y;
    }
    G[p] = g;
}

__global__ void k_average_sources(long long nn, const double* __restrict__ f4, double2* __restrict__ src) {
    pdl_enter();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    src[i] = make_double2(0.5 * (f4[i] + f4[nn + i]), 0.5 * (f4[2 * nn + i] + f4[3 * nn + i]));
}

template <int D>
__global__ void __launch_bounds__(kT) k_newton_F(Lists ls, GhostTab<double> tb, const double2* __restrict__ W, const double2* __restrict__ G,
                                                  double2* __restrict__ F, double2* __restrict__ Fc, Offs<D> of,
                                                  long long st1, long long st2, FConst f, unsigned long long* norm) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nb = 0;
    if (t < ls.n0 + ls.n1 + ls.ng) {
        int kind, gi = 0;
        long long p = list_node(ls, t, kind, gi);
        double2 w = W[p];
        double2 g = G[p];
        double ph = f.alpha * w.y + f.beta;
        double Lc = -f.ams * ph * w.x * w.y;
        double2 out;
        out.y = w.y * f.idt - 0.5 * Lc + g.y;
        if (kind == 1) {
            double phd;
            double Ls = Ls_h<D>(p, W, of, f, phd);
            out.x = ph * w.x * f.idt - 0.5 * Ls + g.x;
        } else {
            out.x = stages::row_dot<D, double, false>(tb, gi, nullptr, W, nullptr, true) - (f.sbg ? f.sbg[gi] : f.sb);
        }
        F[p] = out;
        if (Fc) Fc[t] = out;  // the list-ordered copy
        unsigned long long a0 = abs_bits(out.x), a1 = abs_bits(out.y);
        nb = a0 > a1 ? a0 : a1;
    }
    block_max(nb, norm);
}

// W -= x on active nodes; norms[0] = |x|_inf, norms[1] = |W_old|_inf
__global__ void __launch_bounds__(kT) k_newton_update(Lists ls, double2* __restrict__ W, const double2* __restrict__ x,
                                                      unsigned long long* norms) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nx = 0, nw = 0;
    if (t < ls.n0 + ls.n1 + ls.ng) {
        int kind, gi;
        long long p = list_node(ls, t, kind, gi);
        double2 w = W[p], d = x[p];
        unsigned long long a0 = abs_bits(w.x), a1 = abs_bits(w.y);
        nw = a0 > a1 ? a0 : a1;
        a0 = abs_bits(d.x);
        a1 = abs_bits(d.y);
        nx = a0 > a1 ? a0 : a1;
        w.x -= d.x;
        w.y -= d.y;
        W[p] = w;
    }
    block_max(nx, norms);
    __syncthreads();
    block_max(nw, norms + 1);
}

__global__ void __launch_bounds__(kT) k_norm_active(Lists ls, const double2* __restrict__ v, unsigned long long* norm) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long nb = 0;
    if (t < ls.n0 + ls.n1 + ls.ng) {
        int kind, gi;
        long long p = list_node(ls, t, kind, gi);
        double2 w = v[p];
        unsigned long long a0 = abs_bits(w.x), a1 = abs_bits(w.y);
        nb = a0 > a1 ? a0 : a1;
    }
    block_max(nb, norm);
}

// mixed precision: FP64 values to FP32 on active nodes
__global__ void k_to_float2(Lists ls, const double2* __restrict__ a, float2* __restrict__ b) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi;
    long long p = list_node(ls, t, kind, gi);
    double2 v = a[p];
    b[p] = make_float2((float)v.x, (float)v.y);
}

// x64 += e32 on active nodes
__global__ void k_accumulate(Lists ls, double2* __restrict__ x, const float2* __restrict__ e) {
    pdl_enter();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi;
    long long p = list_node(ls, t, kind, gi);
    double2 v = x[p];
    float2 d = e[p];
    v.x += (double)d.x;
    v.y += (double)d.y;
    x[p] = v;
}

// state import / export over the box
__global__ void k_reset_state(const int8_t* __restrict__ type, long long nn, double2* W, double s0, double c0) {
    pdl_enter();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int8_t t = type[i];
    bool a = t == T_IN || t == T_GHOST;
    W[i] = make_double2(a ? s0 : 0.0, a ? c0 : 0.0);
}

__global__ void k_import_state(const int8_t* __restrict__ type, long long nn, double2* W, const double* __restrict__ sv,
                               const double* __restrict__ cv) {
    pdl_enter();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int8_t t = type[i];
    bool a = t == T_IN || t == T_GHOST;
    W[i] = make_double2(a ? sv[i] : 0.0, a ? cv[i] : 0.0);
}

__global__ void k_export_state(const int8_t* __restrict__ type, long long nn, const double2* __restrict__ W,
                               double* sv, double* cv, int8_t* tv) {
    pdl_enter();
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int8_t t = type[i];
    bool a = t == T_IN || t == T_GHOST;
    double2 w = W[i];
    if (sv) sv[i] = a ? w.x : 0.0;
    if (cv) cv[i] = a ? w.y : 0.0;
    if (tv) tv[i] = a ? t : (int8_t)0;
}

}  // namespace

// ---------------------------------------------------------------------------
// host launchers

template <int D, typename T>
int launch_coefs(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    if (tot == 0) return 0;
    launch_k(k_coefs<D, T>, grid_for(tot), block_for(tot), 0, s, ls, L.n, V.Wc, V.edge[0], V.edge[1], V.edge[2], V.Pa,
             V.Pb, V.Ia, V.Ib, V.Pc, V.Ic, V.gc, V.gci, c);
    return 1;
}

template <int D, typename T>
int launch_relax_inside(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int colour, bool pointwise,
                        T* snap, cudaStream_t s) {
    int cnt = L.nin[colour];
    const int sn = snap ? L.ng : 0;
    const int tot = cnt > sn ? cnt : sn;
    if (tot == 0) return 0;
    CoefPtr<D, T> cf = coef_ptr<D, T>(V);
    if (std::is_same<T, float>::value && !pointwise && launch_matrix_free()) {
        Coef<float> cc;
        cc.alpha = (float)c.alpha;
        cc.beta = (float)c.beta;
        cc.a2mc = (float)c.a2mc;
        cc.a2ms = (float)c.a2ms;
        cc.idt = (float)c.idt;
        cc.kap = (float)c.kap;
        cc.tau = (float)c.tau;
        launch_k(k_relax_mf<D>, grid_for(tot), block_for(tot), 0, s, L.inl[colour], cnt,
                 reinterpret_cast<const float2*>(V.Wc), reinterpret_cast<const float2*>(V.rhs),
                 reinterpret_cast<float2*>(V.x), cc, L.st[1], L.st[2], L.gidx, sn,
                 reinterpret_cast<float*>(snap));
        return 1;
    }
    const int t0 = colour ? L.nin[0] : 0;
    if (pointwise)
        launch_k(k_relax_inside<D, T, true>, grid_for(tot), block_for(tot), 0, s, L.inl[colour], cnt, t0, cf,
                 V.rhs, V.rhsc, V.x, L.st[1], L.st[2], L.gidx, sn, snap);
    else
        launch_k(std::is_same<T, double>::value && launch_occupancy() ? k_relax_inside_ho<D, T>
                                                                       : k_relax_inside<D, T, false>,
                 grid_for(tot), block_for(tot), 0, s, L.inl[colour], cnt, t0, cf,
                 V.rhs, V.rhsc, V.x, L.st[1], L.st[2], L.gidx, sn, snap);
    return 1;
}

template <int D, typename T>
int launch_relax_lex(const LevelGeo& L, const LevelVec<T>& V, T* snap, cudaStream_t s) {
    if (!L.lex) return 0;
    const int sn = snap ? L.ng : 0;
    launch_k(k_relax_lex<D, T>, 1, kLexThreads, 0, s, L.lex, L.lexptr, L.nlexd, coef_ptr<D, T>(V), V.rhs, V.x,
             L.st[1], L.st[2], L.gidx, sn, snap);
    return 1;
}

int launch_sweep_tiled(const LevelGeo& L, const float2* Wc, const float2* rhs, const float2* xin, float2* xout,
                       const Coef<float>& c, float* snap, cudaStream_t s) {
    if (!L.tiles || L.ntiles == 0) return 0;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_sweep_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(TileSmem));
    });
    launch_k(k_sweep_tile, (unsigned)L.ntiles, kTileThreads, sizeof(TileSmem), s, L.tiles, L.tile_nx, L.tile_ny, L.n,
             L.type, Wc, rhs, xin, xout, c, L.gidx, L.ng, snap);
    return 1;
}

template <int D, typename T>
int launch_relax_ghosts(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int passes, bool composed,
                        cudaStream_t s) {
    if (L.ng == 0 || passes < 1) return 0;
    if (composed) {
        const long long nt = (long long)L.ng * kGopLanes;
        const T* val = std::is_same<T, float>::value ? (const T*)L.gop_val32 : (const T*)L.gop_val;
        launch_k(k_ghost_op<T>, grid_for(nt), block_for(nt), 0, s, L.ng, L.gidx, L.gop_ptr, L.gop_code, val, V.gc,
                 V.gci, V.rhs, V.x, V.gbuf[0]);
        return 1;
    }
    int n = 0;
    for (int p = 0; p < passes; p++) {
        bool first = p == 0, last = p == passes - 1 && passes > 1;
        const T* sin = first ? nullptr : V.gbuf[(p - 1) & 1];
        T* sout = V.gbuf[p & 1];
        launch_k(k_ghost_pass<D, T>, grid_for(L.ng), block_for(L.ng), 0, s, L.gidx, stages::ghost_tab<T>(L), V.gc, V.gci,
                 V.rhs, V.x, sin, sout, c, first, last);
        n++;
    }
    if (passes == 1) {
        launch_k(k_ghost_scatter<T>, grid_for(L.ng), block_for(L.ng), 0, s, L.ng, L.gidx, V.gbuf[0], V.x);
        n++;
    }
    return n;
}

template <int D, typename T>
int launch_residual(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, unsigned long long* norm,
                    cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    if (tot == 0) return 0;
    (void)c;
    launch_k(k_residual<D, T, typename V2<T>::t>, grid_for(tot), block_for(tot), 0, s, ls, stages::ghost_tab<T>(L),
             coef_ptr<D, T>(V), V.rhs, V.x, V.res, L.st[1], L.st[2], norm, V.rhsc);
    return 1;
}

template <int D>
int launch_residual_to32(const LevelGeo& L, const LevelVec<double>& V, float2* out, unsigned long long* norm,
                         cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    if (tot == 0) return 0;
    launch_k(k_residual<D, double, float2>, grid_for(tot), block_for(tot), 0, s, ls, stages::ghost_tab<double>(L),
             coef_ptr<D, double>(V), V.rhs, V.x, out, L.st[1], L.st[2], norm, V.rhsc);
    return 1;
}
template int launch_residual_to32<2>(const LevelGeo&, const LevelVec<double>&, float2*, unsigned long long*,
                                     cudaStream_t);
template int launch_residual_to32<3>(const LevelGeo&, const LevelVec<double>&, float2*, unsigned long long*,
                                     cudaStream_t);

template <int D, typename T>
int launch_extend(const LevelGeo& L, const LevelVec<T>& V, cudaStream_t s) {
    if (L.nb == 0) return 0;
    const T* ev = std::is_same<T, float>::value ? (const T*)L.eval32 : (const T*)L.eval;
    launch_k(k_extend<T>, grid_for(L.nb), block_for(L.nb), 0, s, L.nb, L.eptr, L.eidx, ev, L.bidx, V.res);
    return 1;
}

template <int D, typename T>
int launch_restrict(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                    bool first_red, bool pointwise, cudaStream_t s) {
    Lists ls = make_lists(C);
    int tot = ls.n0 + ls.n1 + ls.ng;
    CoefPtr<D, T> ccf = coef_ptr<D, T>(CV);
    if (pointwise)
        launch_k(k_restrict<D, T, true>, grid_for(tot), block_for(tot), 0, s, ls, C.type, C.n, F.type, F.n, FV.res,
                 CV.rhs, CV.x, ccf, first_red ? 1 : 0, CV.rhsc);
    else
        launch_k(k_restrict<D, T, false>, grid_for(tot), block_for(tot), 0, s, ls, C.type, C.n, F.type, F.n, FV.res,
                 CV.rhs, CV.x, ccf, first_red ? 1 : 0, CV.rhsc);
    return 1;
}

// a box-ordered vector gathered into list order (the rhsc copy of rhs)
__global__ void k_gather_list(Lists ls, const double2* __restrict__ box, double2* __restrict__ list) {
    pdl_enter();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ls.n0 + ls.n1 + ls.ng) return;
    int kind, gi;
    list[t] = box[list_node(ls, t, kind, gi)];
}

int launch_gather_list(const LevelGeo& L, const double2* box, double2* list, cudaStream_t s) {
    Lists ls = make_lists(L);
    const int tot = ls.n0 + ls.n1 + ls.ng;
    if (tot == 0 || !list) return 0;
    launch_k(k_gather_list, grid_for(tot), block_for(tot), 0, s, ls, box, list);
    return 1;
}

template <int D, typename T>
int launch_prolong(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                   cudaStream_t s) {
    Lists ls = make_lists(F);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_prolong<D, T>, grid_for(tot), block_for(tot), 0, s, ls, C.type, C.n, CV.x, F.n, FV.x);
    return 1;
}

template <int D, typename T>
int launch_inject(const LevelGeo& F, const LevelVec<T>& FV, const LevelGeo& C, const LevelVec<T>& CV,
                  cudaStream_t s) {
    Lists ls = make_lists(C);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_inject<D, T>, grid_for(tot), block_for(tot), 0, s, ls, C.n, F.type, F.n, FV.Wc, CV.Wc);
    return 1;
}

template <int D, typename T>
int launch_coarsest_factor(const LevelGeo& L, const LevelVec<T>& V, const Coef<T>& c, int* singular,
                           cudaStream_t s) {
    GhostTab<T> tb = stages::ghost_tab<T>(L);
    Offs<D> of = make_offs<D>(L.st[1], L.st[2]);
    const size_t m = 2 * (size_t)L.nact;
    const size_t piv_bytes = sizeof(T) * (m + 1) + sizeof(int) * (m + 1);  // column k and the interchanges
    const size_t smem_cluster = factor_cluster_smem<T>((int)m);
    constexpr size_t kMaxSmem = 220 * 1024;
    if (smem_cluster <= kMaxSmem) {
        auto kern = k_coarsest_factor_cluster<D, T>;
        // The limit is a per-function attribute shared by every thread: set it
        // once to the largest size ever used (a per-launch value would race
        // with other threads' launches of different sizes).
        static std::mutex mu;
        static bool raised[64] = {};
        int dev = 0;
        cudaGetDevice(&dev);
        {
            std::lock_guard<std::mutex> lock(mu);
            if (dev < 0 || dev >= 64 || !raised[dev]) {
                cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
                if (dev >= 0 && dev < 64) raised[dev] = true;
            }
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(kFacCluster);
        cfg.blockDim = dim3(kFacThreads);
        cfg.dynamicSmemBytes = smem_cluster;
        cfg.stream = s;
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = kFacCluster;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[1].val.programmaticStreamSerializationAllowed = launch_pdl() ? 1 : 0;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        cudaError_t e = cudaLaunchKernelEx(&cfg, kern, (int)L.nact, (const int*)L.act, (const int*)L.apos,
                                           (const int8_t*)L.type, (const int*)L.gpos, tb,
                                           (const typename V2<T>::t*)V.Wc, of, c, V.Ainv, singular);
        if (e != cudaSuccess) note_launch_error(e, kFacCluster, kFacThreads, smem_cluster);
    } else {
        launch_k(k_coarsest_factor<D, T, false>, 1, 1024, piv_bytes, s, L.nact, L.act, L.apos, L.type, L.gpos, tb,
                                                                  V.Wc, of, L.st[1], L.st[2], c, V.A, V.Ainv,
                                                                  singular);
    }
    return 1;
}

template <int D, typename T>
int launch_coarsest_solve(const LevelGeo& L, const LevelVec<T>& V, cudaStream_t s) {
    size_t shm = sizeof(T) * (2 * (size_t)L.nact + 2);
    const int m = 2 * L.nact, rows_per_cta = 8;
    launch_k(k_coarsest_solve<T>, (m + rows_per_cta - 1) / rows_per_cta, 32 * rows_per_cta, shm, s, L.nact, L.act,
             V.Ainv, V.rhs, V.x);
    return 1;
}

template <int D>
int launch_old_time(const LevelGeo& L, const double2* Wn, double2* G, const FConst& fc, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_old_time<D>, grid_for(tot), block_for(tot), 0, s, ls, Wn, G, make_offs<D>(L.st[1], L.st[2]), fc);
    return 1;
}

template <int D>
int launch_newton_F(const LevelGeo& L, const double2* W, const double2* G, double2* F, double2* Fc,
                    const FConst& fc, unsigned long long* norm, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_newton_F<D>, grid_for(tot), block_for(tot), 0, s, ls, stages::ghost_tab<double>(L), W, G, F, Fc,
             make_offs<D>(L.st[1], L.st[2]), L.st[1], L.st[2], fc, norm);
    return 1;
}

int launch_newton_update(const LevelGeo& L, double2* W, const double2* x, unsigned long long* norms, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_newton_update, grid_for(tot), block_for(tot), 0, s, ls, W, x, norms);
    return 1;
}

int launch_norm_active(const LevelGeo& L, const double2* v, unsigned long long* norm, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_norm_active, grid_for(tot), block_for(tot), 0, s, ls, v, norm);
    return 1;
}

int launch_average_sources(long long nn, const double* f4, double2* src, cudaStream_t s) {
    launch_k(k_average_sources, grid_for(nn), block_for(nn), 0, s, nn, f4, src);
    return 1;
}

int launch_to_float(const LevelGeo& L, const double2* src, float2* dst, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_to_float2, grid_for(tot), block_for(tot), 0, s, ls, src, dst);
    return 1;
}

// End of one cycle of the device-side linear-solve loop: counts the cycle,
// records its defect norm and sets the enclosing conditional node to run
// another cycle unless the defect met the threshold, is not a number, the
// coarsest Jacobian was singular or the cycle cap is reached.
__global__ void k_cycle_check(cudaGraphConditionalHandle h, const unsigned long long* __restrict__ norm,
                              const int* __restrict__ singular, const double* __restrict__ thr, int max_cycles,
                              int* cycles, double* rnorms) {
    pdl_enter();
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int c = *cycles + 1;
    *cycles = c;
    const double rn = __longlong_as_double((long long)norm[0]);
    rnorms[c - 1] = rn;
    const bool more = *singular == 0 && rn == rn && rn > *thr && c < max_cycles;
    cudaGraphSetConditional(h, more ? 1u : 0u);
}

int launch_cycle_check(cudaGraphConditionalHandle h, const unsigned long long* norm, const int* singular,
                       const double* thr, int max_cycles, int* cycles, double* rnorms, cudaStream_t s) {
    launch_k(k_cycle_check, 1, 32, 0, s, h, norm, singular, thr, max_cycles, cycles, rnorms);
    return 1;
}

int launch_accumulate(const LevelGeo& L, double2* x, const float2* e, cudaStream_t s) {
    Lists ls = make_lists(L);
    int tot = ls.n0 + ls.n1 + ls.ng;
    launch_k(k_accumulate, grid_for(tot), block_for(tot), 0, s, ls, x, e);
    return 1;
}

int launch_reset_state(const LevelGeo& L, double2* W, double s0, double c0, cudaStream_t s) {
    launch_k(k_reset_state, grid_for(L.nn), block_for(L.nn), 0, s, L.type, L.nn, W, s0, c0);
    return 1;
}

int launch_import_state(const LevelGeo& L, double2* W, const double* sv, const double* cv, cudaStream_t s) {
    launch_k(k_import_state, grid_for(L.nn), block_for(L.nn), 0, s, L.type, L.nn, W, sv, cv);
    return 1;
}

int launch_export_state(const LevelGeo& L, const double2* W, double* sv, double* cv, int8_t* tv, cudaStream_t s) {
    launch_k(k_export_state, grid_for(L.nn), block_for(L.nn), 0, s, L.type, L.nn, W, sv, cv, tv);
    return 1;
}

#define SULF_INST(D, T)                                                                                          \
    template int launch_coefs<D, T>(const LevelGeo&, const LevelVec<T>&, const Coef<T>&, cudaStream_t);          \
    template int launch_relax_inside<D, T>(const LevelGeo&, const LevelVec<T>&, const Coef<T>&, int, bool, T*,   \
                                           cudaStream_t);                                                        \
    template int launch_relax_lex<D, T>(const LevelGeo&, const LevelVec<T>&, T*, cudaStream_t);                     \
    template int launch_relax_ghosts<D, T>(const LevelGeo&, const LevelVec<T>&, const Coef<T>&, int, bool,          \
                                           cudaStream_t);                                                        \
    template int launch_residual<D, T>(const LevelGeo&, const LevelVec<T>&, const Coef<T>&, unsigned long long*,  \
                                       cudaStream_t);                                                            \
    template int launch_extend<D, T>(const LevelGeo&, const LevelVec<T>&, cudaStream_t);                         \
    template int launch_restrict<D, T>(const LevelGeo&, const LevelVec<T>&, const LevelGeo&, const LevelVec<T>&, \
                                       bool, bool, cudaStream_t);                                                \
    template int launch_prolong<D, T>(const LevelGeo&, const LevelVec<T>&, const LevelGeo&, const LevelVec<T>&,  \
                                      cudaStream_t);                                                             \
    template int launch_inject<D, T>(const LevelGeo&, const LevelVec<T>&, const LevelGeo&, const LevelVec<T>&,   \
                                     cudaStream_t);                                                              \
    template int launch_coarsest_factor<D, T>(const LevelGeo&, const LevelVec<T>&, const Coef<T>&, int*,         \
                                              cudaStream_t);                                                     \
    template int launch_coarsest_solve<D, T>(const LevelGeo&, const LevelVec<T>&, cudaStream_t);

SULF_INST(2, double)
SULF_INST(2, float)
SULF_INST(3, double)
SULF_INST(3, float)

template int launch_old_time<2>(const LevelGeo&, const double2*, double2*, const FConst&, cudaStream_t);
template int launch_old_time<3>(const LevelGeo&, const double2*, double2*, const FConst&, cudaStream_t);
template int launch_newton_F<2>(const LevelGeo&, const double2*, const double2*, double2*, double2*, const FConst&,
                                unsigned long long*, cudaStream_t);
template int launch_newton_F<3>(const LevelGeo&, const double2*, const double2*, double2*, double2*, const FConst&,
                                unsigned long long*, cudaStream_t);

}  // namespace sulf
