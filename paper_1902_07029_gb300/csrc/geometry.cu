// Level-set geometry of one multigrid level, built once per domain on the GPU.
//
//  * level-set coarsening by injection, phi_2h(I) = phi_h(2I) (Sec. 3.5.3:
//    the coarse operator is rediscretised "with the same technique");
//  * inside / ghost classification (Sec. 3.3, Eq. ghostdef);
//  * ordered stream compaction into index lists (box order);
//  * per-ghost boundary rows (Sec. 3.3): outward normal by central differences
//    (Eq. nij), upwind stencil ST, closest boundary point B by bisection on the
//    tensor-product interpolant of phi along P -> G, and the 1-D weights of
//    Eq. intcoeffsD built dimension by dimension; the row needs every node it
//    weights to be active, else lower per-axis orders are tried, then the
//    identity row;
//  * the band of inactive nodes that receives the ghost defect extended along
//    the normal before restriction (Sec. 3.5.2).
#include <cstdio>
#include <cstring>

#include "sulf_internal.cuh"

namespace sulf {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kChunk = kThreads * kPerThread;

__device__ __forceinline__ void node_coords(long long idx, int n, int dim, int* ii) {
    ii[0] = (int)(idx % n);
    ii[1] = dim > 1 ? (int)((idx / n) % n) : 0;
    ii[2] = dim > 2 ? (int)(idx / ((long long)n * n)) : 0;
}

__device__ __forceinline__ bool is_active(int8_t t) { return t == T_IN || t == T_GHOST; }

__global__ void k_inject_phi(const double* __restrict__ fphi, double* __restrict__ cphi, int cn, int fn, int dim,
                             long long cnn) {
    long long I = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (I >= cnn) return;
    int ii[3];
    node_coords(I, cn, dim, ii);
    long long f = 2LL * ii[0] + 2LL * ii[1] * fn + 2LL * ii[2] * (long long)fn * fn;
    cphi[I] = fphi[f];
}

__global__ void k_classify_inside(const double* __restrict__ phi, int8_t* __restrict__ type, long long nn) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    type[i] = phi[i] < 0.0 ? T_IN : T_OUT;
}

// a non-inside node with an inside axis neighbour is a ghost (Eq. ghostdef)
__global__ void k_classify_ghost(int8_t* __restrict__ type, int n, int dim, long long nn) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    if (type[i] != T_OUT) return;
    int ii[3];
    node_coords(i, n, dim, ii);
    long long st = 1;
    bool g = false;
    for (int a = 0; a < dim; a++) {
        if (ii[a] > 0 && type[i - st] == T_IN) g = true;
        if (ii[a] < n - 1 && type[i + st] == T_IN) g = true;
        st *= n;
    }
    if (g) type[i] = T_GHOST;
}

__global__ void k_check_edge(const int8_t* __restrict__ type, int n, int dim, long long nn, int* flag) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    if (!is_active(type[i])) return;
    int ii[3];
    node_coords(i, n, dim, ii);
    for (int a = 0; a < dim; a++)
        if (ii[a] == 0 || ii[a] == n - 1) atomicOr(flag, 1);
}

// predicates of the compactions
enum { P_IN0 = 0, P_IN1 = 1, P_GHOST = 2, P_BAND = 3, P_ACTIVE = 4 };

__device__ __forceinline__ bool pred(int which, const int8_t* type, long long i, int n, int dim) {
    int8_t t = type[i];
    switch (which) {
        case P_IN0:
        case P_IN1: {
            if (t != T_IN) return false;
            int ii[3];
            node_coords(i, n, dim, ii);
            return ((ii[0] + ii[1] + ii[2]) & 1) == (which == P_IN1 ? 1 : 0);
        }
        case P_GHOST: return t == T_GHOST;
        case P_BAND: return t == T_BAND;
        default: return is_active(t);
    }
}

__global__ void k_compact_count(int which, const int8_t* __restrict__ type, long long nn, int n, int dim,
                                int* __restrict__ blockcnt) {
    __shared__ int wsum[kThreads / 32];
    long long base = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPerThread;
    int c = 0;
    for (int k = 0; k < kPerThread; k++)
        if (base + k < nn && pred(which, type, base + k, n, dim)) c++;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < kThreads / 32; w++) s += wsum[w];
        blockcnt[blockIdx.x] = s;
    }
}

// writes the selected indices of each chunk in box order at the chunk's offset
__global__ void k_compact_write(int which, const int8_t* __restrict__ type, long long nn, int n, int dim,
                                const int* __restrict__ blockoff, int* __restrict__ out) {
    __shared__ int wsum[kThreads / 32];
    long long base = (long long)blockIdx.x * kChunk + (long long)threadIdx.x * kPerThread;
    bool f[kPerThread];
    int c = 0;
    for (int k = 0; k < kPerThread; k++) {
        f[k] = base + k < nn && pred(which, type, base + k, n, dim);
        c += f[k];
    }
    // block-exclusive scan of c
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = c;
    for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < warp; w++) woff += wsum[w];
    int pos = blockoff[blockIdx.x] + woff + incl - c;
    for (int k = 0; k < kPerThread; k++)
        if (f[k]) out[pos++] = (int)(base + k);
}

__global__ void k_scatter_pos(const int* __restrict__ list, int cnt, int* __restrict__ pos) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < cnt) pos[list[t]] = t;
}

// ---- ghost boundary rows ----

__device__ void grad_phi(const double* phi, long long idx, const int* ii, int n, int dim, double h, double* g) {
    long long st = 1;
    for (int a = 0; a < dim; a++) {
        bool hm = ii[a] > 0, hp = ii[a] < n - 1;
        if (hm && hp)
            g[a] = (phi[idx + st] - phi[idx - st]) / (2.0 * h);
        else if (hp)
            g[a] = (phi[idx + st] - phi[idx]) / h;
        else
            g[a] = (phi[idx] - phi[idx - st]) / h;
        st *= n;
    }
}

// 1-D Lagrange basis at local coordinate xi (offset 0 at xi = 1, offset 1 at
// 0, offset 2 at -1): quadratic (Eq. intcoeffsD), linear or constant
__device__ __forceinline__ double basis(int order, int k, double xi) {
    if (order == 0) return k == 0 ? 1.0 : 0.0;
    if (order == 2) {
        if (k == 0) return xi * (1.0 + xi) / 2.0;
        if (k == 1) return (1.0 - xi) * (1.0 + xi);
        return xi * (xi - 1.0) / 2.0;
    }
    if (k == 0) return xi;
    if (k == 1) return 1.0 - xi;
    return 0.0;
}

// derivative of basis with respect to xi: the 1-D first-derivative weights of
// Eq. intcoeffsN (times h) for the quadratic, (1, -1) linear, 0 constant
__device__ __forceinline__ double dbasis(int order, int k, double xi) {
    if (order == 0) return 0.0;
    if (order == 2) {
        if (k == 0) return xi + 0.5;
        if (k == 1) return -2.0 * xi;
        return xi - 0.5;
    }
    if (k == 0) return 1.0;
    if (k == 1) return -1.0;
    return 0.0;
}

// gradient of the tensor interpolant of phi of the given order on the upwind
// stencil of ghost g at the local coordinates xi (Eq. Neumanntilde:
// n~* = grad phi~); d/dX_a = (m_a / h) d/dxi_a
template <int D>
__device__ void grad_interp_phi(const double* phi, int order, long long g, const int* m, const double* xi, int n,
                                double h, double* gr) {
    long long st[3] = {1, n, (long long)n * n};
    for (int a = 0; a < D; a++) gr[a] = 0.0;
    const int K = D == 2 ? 9 : 27;
    for (int kk = 0; kk < K; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        bool skip = false;
        long long node = g;
        for (int a = 0; a < D; a++) {
            if (order == 1 && k[a] == 2) skip = true;
            node -= (long long)m[a] * k[a] * st[a];
        }
        if (skip) continue;
        for (int a = 0; a < D; a++) {
            double t = (m[a] / h) * dbasis(order, k[a], xi[a]);
            for (int b = 0; b < D; b++)
                if (b != a) t *= basis(order, k[b], xi[b]);
            gr[a] += t * phi[node];
        }
    }
}

// weight of stencil member kk of a ghost row: Dirichlet (Eq. JssD) the tensor
// product of the 1-D value weights; Neumann (Eq. JccN built dimension by
// dimension) n~ . grad s~ at B = sum_a n~_a (m_a / h) dbasis_a prod_{b != a} basis_b
template <int D>
__device__ double member_weight(int bc, double h, const int* m, const int* ord, const double* th, const double* nt,
                                int kk) {
    int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
    if (bc == 0) {
        double w = 1.0;
        for (int a = 0; a < D; a++) w *= basis(ord[a], k[a], th[a]);
        return w;
    }
    double w = 0.0;
    for (int a = 0; a < D; a++) {
        double t = nt[a] * (m[a] / h) * dbasis(ord[a], k[a], th[a]);
        for (int b = 0; b < D; b++)
            if (b != a) t *= basis(ord[b], k[b], th[b]);
        w += t;
    }
    return w;
}

// tensor-product interpolant of phi on the upwind stencil of ghost g, at X;
// local coordinate xi_a = 1 - m_a (G_a - X_a) / h
template <int D>
__device__ double interp_phi(const double* phi, int order, long long g, const int* ii, const int* m, const double* X,
                             int n, double lo, double h) {
    double xi[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < D; a++) xi[a] = 1.0 - m[a] * ((lo + ii[a] * h) - X[a]) / h;
    long long st[3] = {1, n, (long long)n * n};
    double acc = 0.0;
    const int K = D == 2 ? 9 : 27;
    for (int kk = 0; kk < K; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        bool skip = false;
        double w = 1.0;
        long long node = g;
        for (int a = 0; a < D; a++) {
            if (order == 1 && k[a] == 2) skip = true;
            w *= basis(order, k[a], xi[a]);
            node -= (long long)m[a] * k[a] * st[a];
        }
        if (!skip) acc += w * phi[node];
    }
    return acc;
}

// every stencil node with a nonzero member weight must be active
template <int D>
__device__ bool weighted_active(const int8_t* type, long long g, const int* m, int bc, double h, const int* ord,
                                const double* th, const double* nt, int n) {
    long long st[3] = {1, n, (long long)n * n};
    const int K = D == 2 ? 9 : 27;
    for (int kk = 0; kk < K; kk++) {
        int k[3] = {kk % 3, (kk / 3) % 3, kk / 9};
        long long node = g;
        for (int a = 0; a < D; a++) node -= (long long)m[a] * k[a] * st[a];
        if (member_weight<D>(bc, h, m, ord, th, nt, kk) != 0.0 && !is_active(type[node])) return false;
    }
    return true;
}

// one thread per ghost: normal (Eq. nij), upwind signs (SIGN(0) = +1), the
// boundary point B by bisection on the quadratic interpolant of phi along
// P -> G with P = G - 2 h n (else the linear one with P = G - h n), then the
// per-axis interpolation orders: all 2 (the paper's row), all 1, then order 0
// on the axis of smallest |n_a|, then on the two smallest; a row needs every
// node it weights to be active, else the identity row
template <int D>
__global__ void k_ghost_geom(const double* __restrict__ phi, const int8_t* __restrict__ type, int n, double lo,
                             double h, const int* __restrict__ gidx, int ng, int bc, int8_t* gkind, int8_t* gm,
                             double* gw, double* gB, int8_t* gord, double* gth, double* gnt) {
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    long long g = gidx[gi];
    int ii[3];
    node_coords(g, n, D, ii);
    double gr[3] = {0, 0, 0}, nv[3] = {0, 0, 0};
    grad_phi(phi, g, ii, n, D, h, gr);
    double nrm = 0.0;
    for (int a = 0; a < D; a++) nrm += gr[a] * gr[a];
    nrm = sqrt(nrm);
    int m[3] = {1, 1, 1};
    if (nrm > 0.0)
        for (int a = 0; a < D; a++) {
            nv[a] = gr[a] / nrm;
            m[a] = nv[a] >= 0.0 ? 1 : -1;
        }
    double wout[9], bout[3], B[3] = {0, 0, 0};
    int border = 0;
    if (nrm > 0.0) {
        for (int order = 2; order >= 1 && !border; order--) {
            bool inbox = true;
            for (int a = 0; a < D; a++) {
                int ia = ii[a] - m[a] * order;
                if (ia < 0 || ia > n - 1) inbox = false;
            }
            if (!inbox) continue;
            double G[3], P[3], X[3];
            for (int a = 0; a < D; a++) {
                G[a] = lo + ii[a] * h;
                P[a] = G[a] - order * h * nv[a];
            }
            if (!(interp_phi<D>(phi, order, g, ii, m, P, n, lo, h) < 0.0)) continue;
            double alo = 0.0, ahi = 1.0;
            for (int it = 0; it < 60 && ahi - alo >= 1e-14; it++) {
                double am = 0.5 * (alo + ahi);
                for (int a = 0; a < D; a++) X[a] = P[a] + am * (G[a] - P[a]);
                if (interp_phi<D>(phi, order, g, ii, m, X, n, lo, h) < 0.0)
                    alo = am;
                else
                    ahi = am;
            }
            double al = 0.5 * (alo + ahi);
            for (int a = 0; a < D; a++) B[a] = P[a] + al * (G[a] - P[a]);
            border = order;
        }
    }
    int kind = 2;
    double nt[3] = {nv[0], nv[1], nv[2]}, thout[3] = {1.0, 1.0, 1.0};
    int ordout[3] = {0, 0, 0};
    if (border) {
        int ax[3] = {0, 1, 2};
        for (int i = 0; i < D; i++)
            for (int j = i + 1; j < D; j++)
                if (fabs(nv[ax[j]]) < fabs(nv[ax[i]])) {
                    int t = ax[i];
                    ax[i] = ax[j];
                    ax[j] = t;
                }
        double th[3] = {0, 0, 0};
        for (int a = 0; a < D; a++) th[a] = 1.0 - m[a] * ((lo + ii[a] * h) - B[a]) / h;
        // unit normal of phi~ at B: quadratic interpolant where its stencil fits
        // in the box, else the linear one, else the node normal
        int q = 0;
        for (int o = 2; o >= 1 && !q; o--) {
            bool inbox = true;
            for (int a = 0; a < D; a++) {
                int ia = ii[a] - m[a] * o;
                if (ia < 0 || ia > n - 1) inbox = false;
            }
            if (inbox) q = o;
        }
        if (q) {
            double gt[3] = {0, 0, 0}, gn = 0.0;
            grad_interp_phi<D>(phi, q, g, m, th, n, h, gt);
            for (int a = 0; a < D; a++) gn += gt[a] * gt[a];
            gn = sqrt(gn);
            if (gn > 0.0)
                for (int a = 0; a < D; a++) nt[a] = gt[a] / gn;
        }
        for (int nzero = 0; nzero < D && kind == 2; nzero++)
            for (int top = border; top >= 1 && kind == 2; top--) {
                int ord[3] = {top, top, top};
                for (int z = 0; z < nzero; z++) ord[ax[z]] = 0;
                if (weighted_active<D>(type, g, m, bc, h, ord, th, nt, n)) {
                    kind = (nzero == 0 && top == 2) ? 0 : 1;
                    for (int a = 0; a < D; a++) {
                        for (int k = 0; k < 3; k++) wout[3 * a + k] = basis(ord[a], k, th[a]);
                        bout[a] = B[a];
                        ordout[a] = ord[a];
                        thout[a] = th[a];
                    }
                }
            }
    }
    if (kind == 2)
        for (int a = 0; a < D; a++) {
            wout[3 * a + 0] = 1.0;
            wout[3 * a + 1] = 0.0;
            wout[3 * a + 2] = 0.0;
            bout[a] = lo + ii[a] * h;
        }
    gkind[gi] = (int8_t)kind;
    for (int a = 0; a < D; a++) {
        gm[(long long)gi * D + a] = (int8_t)m[a];
        gB[(long long)gi * D + a] = bout[a];
        gord[(long long)gi * D + a] = (int8_t)ordout[a];
        gth[(long long)gi * D + a] = thout[a];
        gnt[(long long)gi * D + a] = nt[a];
        for (int k = 0; k < 3; k++) gw[(long long)gi * 3 * D + 3 * a + k] = wout[3 * a + k];
    }
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long long cnt) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < cnt) b[i] = (float)a[i];
}

// member table of the ghost rows: the tensor weights of Eq. JssD multiplied
// out per stencil member (the same products, in the same order, the row
// evaluation used to form on the fly), the member's box node and ghost index
template <int D>
__global__ void k_ghost_members(int ng, const int* __restrict__ gidx, const int8_t* __restrict__ gm,
                                const double* __restrict__ gw, const float* __restrict__ gw32,
                                const int* __restrict__ gpos, long long st1, long long st2, int bc, double h,
                                const int8_t* __restrict__ gkind, const int8_t* __restrict__ gord,
                                const double* __restrict__ gth, const double* __restrict__ gnt, double* wk,
                                float* wk32, int* node, int* src) {
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    const int K = D == 2 ? 9 : 27;
    const long long g = gidx[gi];
    int m[3] = {1, 1, 1}, ord[3] = {0, 0, 0};
    double th[3] = {1, 1, 1}, nt[3] = {0, 0, 0};
    for (int a = 0; a < D; a++) {
        m[a] = gm[(long long)gi * D + a];
        ord[a] = gord[(long long)gi * D + a];
        th[a] = gth[(long long)gi * D + a];
        nt[a] = gnt[(long long)gi * D + a];
    }
    for (int kk = 0; kk < K; kk++) {
        const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = kk / 9;
        const double* w = gw + (long long)gi * 3 * D;
        const float* w32 = gw32 + (long long)gi * 3 * D;
        double wd = w[k0] * w[3 + k1];
        float wf = w32[k0] * w32[3 + k1];
        if (D == 3) {
            wd = wd * w[6 + k2];
            wf = wf * w32[6 + k2];
        }
        if (bc == 1) {
            // Neumann row (Eq. JccN); the identity fallback is s_g / h
            wd = gkind[gi] == 2 ? (kk == 0 ? 1.0 / h : 0.0) : member_weight<D>(1, h, m, ord, th, nt, kk);
            wf = (float)wd;
        }
        long long nd = g - m[0] * k0 - m[1] * k1 * st1;
        if (D == 3) nd -= m[2] * k2 * st2;
        const long long o = (long long)kk * ng + gi;
        wk[o] = wd;
        wk32[o] = wf;
        const bool on = wd != 0.0 || wf != 0.0f;
        node[o] = on ? (int)nd : (int)g;
        src[o] = on ? gpos[nd] : -1;
    }
}

// ---- band extension operator (Sec. 3.5.2) ----
// kExtSteps explicit upwind Euler steps of dr/dtau + n.grad r = 0 from zero
// band values are linear in the ghost defects with coefficients fixed by the
// geometry: with S_b the sum of |n_a| over b's upwind references,
//   v_{k+1}(b) = (1 - cfl S_b) v_k(b) + cfl sum_a |n_a| u_k(ref_a),
// u the band value (v_k) or the ghost defect at the reference.  Expanding the
// recursion, each band node's final value is a short weighted sum of ghost
// defects; the weights are accumulated over the paths of the recursion.
constexpr int kExtSteps = 4;
constexpr int kExtCap = 32;

template <int D>
__device__ int ext_row(int b, const int* __restrict__ bref, const double* __restrict__ ban, double cfl, int* gnode,
                       double* coef) {
    struct Item {
        int node, k;
        double scale;
    };
    Item st[1 + kExtSteps * (D + 1)];
    int sp = 0, n = 0;
    st[sp++] = Item{b, kExtSteps, 1.0};
    while (sp > 0) {
        Item e = st[--sp];
        if (e.k == 0) continue;  // band values start at zero
        double S = 0.0;
        for (int a = 0; a < D; a++)
            if (bref[(long long)e.node * D + a] != -1) S += ban[(long long)e.node * D + a];
        st[sp++] = Item{e.node, e.k - 1, e.scale * (1.0 - cfl * S)};
        for (int a = 0; a < D; a++) {
            const int r = bref[(long long)e.node * D + a];
            if (r == -1) continue;
            const double w = e.scale * (cfl * ban[(long long)e.node * D + a]);
            if (r >= 0) {
                st[sp++] = Item{r, e.k - 1, w};
            } else {
                const int g = -r - 2;
                int j = 0;
                while (j < n && gnode[j] != g) j++;
                if (j == n) {
                    if (n == kExtCap) return -1;
                    gnode[n] = g;
                    coef[n] = 0.0;
                    n++;
                }
                coef[j] += w;
            }
        }
    }
    return n;
}

template <int D>
__global__ void k_ext_count(int nb, const int* __restrict__ bref, const double* __restrict__ ban, double cfl,
                            int* cnt) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int gnode[kExtCap];
    double coef[kExtCap];
    cnt[b] = ext_row<D>(b, bref, ban, cfl, gnode, coef);
}

template <int D>
__global__ void k_ext_fill(int nb, const int* __restrict__ bref, const double* __restrict__ ban, double cfl,
                           const int* __restrict__ eptr, int* eidx, double* eval, float* eval32) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    int gnode[kExtCap];
    double coef[kExtCap];
    int n = ext_row<D>(b, bref, ban, cfl, gnode, coef);
    const int o = eptr[b];
    for (int j = 0; j < n; j++) {
        eidx[o + j] = gnode[j];
        eval[o + j] = coef[j];
        eval32[o + j] = (float)coef[j];
    }
}

// ---- band of inactive nodes near the ghosts ----

__global__ void k_band_mark(const int8_t* __restrict__ type, int8_t* __restrict__ mark, int n, int dim, long long nn,
                            int layer) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    if (type[i] != T_OUT || mark[i] != 0) return;
    int ii[3];
    node_coords(i, n, dim, ii);
    long long st[3] = {1, n, (long long)n * n};
    const int K = dim == 2 ? 9 : 27;
    for (int kk = 0; kk < K; kk++) {
        int kd[3] = {kk % 3 - 1, (kk / 3) % 3 - 1, kk / 9 - 1};
        bool ok = true;
        long long node = i;
        for (int a = 0; a < dim; a++) {
            int ia = ii[a] + kd[a];
            if (ia < 0 || ia > n - 1) ok = false;
            node += kd[a] * st[a];
        }
        if (!ok || node == i) continue;
        if ((layer == 1 && type[node] == T_GHOST) || (layer == 2 && mark[node] == 1)) {
            mark[i] = (int8_t)layer;
            return;
        }
    }
}

__global__ void k_band_set(int8_t* __restrict__ type, const int8_t* __restrict__ mark, long long nn) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn && mark[i]) type[i] = T_BAND;
}

__global__ void k_band_info(const double* __restrict__ phi, const int8_t* __restrict__ type, int n, int dim, double h,
                            const int* __restrict__ bidx, int nb, const int* __restrict__ bpos, int* bref,
                            double* ban) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    long long i = bidx[b];
    int ii[3];
    node_coords(i, n, dim, ii);
    double gr[3] = {0, 0, 0};
    grad_phi(phi, i, ii, n, dim, h, gr);
    double nrm = 0.0;
    for (int a = 0; a < dim; a++) nrm += gr[a] * gr[a];
    nrm = sqrt(nrm);
    long long st = 1;
    for (int a = 0; a < dim; a++) {
        double na = nrm > 0.0 ? gr[a] / nrm : 0.0;
        int m = na >= 0.0 ? 1 : -1;
        int ia = ii[a] - m;
        int ref = -1;
        if (ia >= 0 && ia <= n - 1) {
            long long up = i - m * st;
            if (type[up] == T_GHOST) ref = -(int)(up + 2);
            else if (type[up] == T_BAND) ref = bpos[up];
        }
        bref[(long long)b * dim + a] = ref;
        ban[(long long)b * dim + a] = fabs(na);
        st *= n;
    }
}

inline int nblk(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

// ---- composed ghost relaxation (Eq. RelGhost) ----
// One pass updates every ghost from the previous pass's values,
//   s_g^{k+1} = s_g^k + tau (b_g - sum_j w_gj u_j^k),
// u_j^k the s of member j: a fixed inside value, or ghost h's s_h^k.  The
// passes are affine in the ghosts' s before the first pass, their right-hand
// sides and the inside members' values, with coefficients fixed by the rows
// and tau, so after P passes s_g is one short weighted sum.  It is expanded
// pass by pass backwards from s_g^P, merging the terms that reach the same
// ghost at the same pass (the frontier) and accumulating the fixed inputs.
constexpr int kGopRowCap = 256;   // entries of one composed row
constexpr int kGopFront = 64;     // ghosts of one frontier
constexpr int kGopMaxPasses = 8;

// per-thread workspace of the row expansion, in shared memory (4.5 KB a
// thread; as local arrays it would make the driver reserve that much stack for
// every resident thread of the device)
struct GopWork {
    double coef[kGopRowCap];
    double ca[kGopFront], cb[kGopFront];
    int code[kGopRowCap];
    int fa[kGopFront], fb[kGopFront];
};
constexpr int kGopBuildThreads = 8;  // 36 KB of workspace per CTA

template <int D>
__device__ int gop_row(int gi, int passes, double tau, int ng, const int* __restrict__ gidx,
                       const double* __restrict__ wk, const int* __restrict__ node, const int* __restrict__ src,
                       GopWork& ws) {
    const int K = D == 2 ? 9 : 27;
    int* code = ws.code;
    double* coef = ws.coef;
    int *fa = ws.fa, *fb = ws.fb;
    double *ca = ws.ca, *cb = ws.cb;
    int nf = 1, n = 0;
    fa[0] = gi;
    ca[0] = 1.0;
    auto out = [&](int c, double v) -> bool {
        int j = 0;
        while (j < n && code[j] != c) j++;
        if (j == n) {
            if (n == kGopRowCap) return false;
            code[n] = c;
            coef[n] = 0.0;
            n++;
        }
        coef[j] += v;
        return true;
    };
    for (int k = passes; k > 0; k--) {
        int nn = 0;
        auto front = [&](int h, double v) -> bool {
            int j = 0;
            while (j < nn && fb[j] != h) j++;
            if (j == nn) {
                if (nn == kGopFront) return false;
                fb[nn] = h;
                cb[nn] = 0.0;
                nn++;
            }
            cb[j] += v;
            return true;
        };
        for (int i = 0; i < nf; i++) {
            const int h = fa[i];
            const double a = ca[i];
            if (!front(h, a)) return -1;
            if (!out(~(2 * gidx[h] + 1), tau * a)) return -1;
            for (int kk = 0; kk < K; kk++) {
                const long long o = (long long)kk * ng + h;
                const double w = wk[o];
                if (w == 0.0) continue;
                const double v = -tau * w * a;
                const int sr = src[o];
                if (sr >= 0) {
                    if (!front(sr, v)) return -1;
                } else if (!out(node[o], v)) {
                    return -1;
                }
            }
        }
        for (int i = 0; i < nn; i++) {
            fa[i] = fb[i];
            ca[i] = cb[i];
        }
        nf = nn;
    }
    for (int i = 0; i < nf; i++)
        if (!out(~(2 * fa[i]), ca[i])) return -1;
    return n;
}

template <int D>
__global__ void k_gop_count(int ng, int passes, double tau, const int* __restrict__ gidx,
                            const double* __restrict__ wk, const int* __restrict__ node,
                            const int* __restrict__ src, int* cnt) {
    extern __shared__ GopWork gop_ws[];
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    cnt[gi] = gop_row<D>(gi, passes, tau, ng, gidx, wk, node, src, gop_ws[threadIdx.x]);
}

template <int D>
__global__ void k_gop_fill(int ng, int passes, double tau, const int* __restrict__ gidx,
                           const double* __restrict__ wk, const int* __restrict__ node, const int* __restrict__ src,
                           const int* __restrict__ ptr, int* gcode, double* gval, float* gval32) {
    extern __shared__ GopWork gop_ws[];
    int gi = blockIdx.x * blockDim.x + threadIdx.x;
    if (gi >= ng) return;
    GopWork& ws = gop_ws[threadIdx.x];
    const int n = gop_row<D>(gi, passes, tau, ng, gidx, wk, node, src, ws);
    const int o = ptr[gi];
    for (int j = 0; j < n; j++) {
        gcode[o + j] = ws.code[j];
        gval[o + j] = ws.coef[j];
        gval32[o + j] = (float)ws.coef[j];
    }
}


// ordered compaction: returns the count, fills out (allocated by the caller
// after a first counting pass when out == nullptr)
int compact(int which, const LevelGeo& L, int*& out, DevMem& mem, cudaStream_t s, std::string& err,
            long long& launches) {
    long long nchunks = (L.nn + kChunk - 1) / kChunk;
    int* dcnt = (int*)mem.get(sizeof(int) * (nchunks + 1));
    if (!dcnt) {
        err = "out of device memory";
        return -1;
    }
    k_compact_count<<<(unsigned)nchunks, kThreads, 0, s>>>(which, L.type, L.nn, L.n, L.dim, dcnt);
    launches++;
    std::vector<int> cnt(nchunks), off(nchunks);
    if (cudaMemcpyAsync(cnt.data(), dcnt, sizeof(int) * nchunks, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = "compaction count failed";
        return -1;
    }
    long long tot = 0;
    for (long long b = 0; b < nchunks; b++) {
        off[b] = (int)tot;
        tot += cnt[b];
    }
    out = (int*)mem.get(sizeof(int) * (tot + 1));
    if (!out) {
        err = "out of device memory";
        return -1;
    }
    if (tot > 0) {
        cudaMemcpyAsync(dcnt, off.data(), sizeof(int) * nchunks, cudaMemcpyHostToDevice, s);
        k_compact_write<<<(unsigned)nchunks, kThreads, 0, s>>>(which, L.type, L.nn, L.n, L.dim, dcnt, out);
        launches++;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            err = "compaction failed";
            return -1;
        }
    }
    return (int)tot;
}

}  // namespace

int build_ghost_op(LevelGeo& L, double tau, int passes, int bc, DevMem& mem, cudaStream_t s, std::string& err,
                   long long& launches) {
    L.gop_on = false;
    L.gop_tau = tau;
    L.gop_passes = passes;
    L.gop_bc = bc;
    // the codes hold 2 * node + 1 in 31 bits
    if (L.ng == 0 || passes < 1 || passes > kGopMaxPasses || L.nn >= (1LL << 30)) return SULF_OK;
    if (!L.gop_ptr) {
        L.gop_ptr = (int*)mem.get(sizeof(int) * (L.ng + 1));
        if (!L.gop_ptr) {
            err = "out of device memory";
            return SULF_ENOMEM;
        }
    }
    const int bt = kGopBuildThreads;
    const size_t shm = sizeof(GopWork) * bt;
    if (L.dim == 2)
        k_gop_count<2><<<nblk(L.ng, bt), bt, shm, s>>>(L.ng, passes, tau, L.gidx, L.gwk, L.gnode, L.gsrc, L.gop_ptr);
    else
        k_gop_count<3><<<nblk(L.ng, bt), bt, shm, s>>>(L.ng, passes, tau, L.gidx, L.gwk, L.gnode, L.gsrc, L.gop_ptr);
    launches++;
    std::vector<int> cnt(L.ng + 1, 0);
    if (cudaMemcpyAsync(cnt.data(), L.gop_ptr, sizeof(int) * L.ng, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        err = "ghost relaxation map failed";
        return SULF_EDEVICE;
    }
    long long tot = 0;
    for (int g = 0; g < L.ng; g++) {
        if (cnt[g] < 0) return SULF_OK;  // a row too long: passes one by one
        const int c = cnt[g];
        cnt[g] = (int)tot;
        tot += c;
    }
    cnt[L.ng] = (int)tot;
    if (tot > (long long)(L.dim == 2 ? kGopAvg2 : kGopAvg3) * L.ng) return SULF_OK;
    if (tot + 1 > L.gop_cap) {
        L.gop_code = (int*)mem.get(sizeof(int) * (tot + 1));
        L.gop_val = (double*)mem.get(sizeof(double) * (tot + 1));
        L.gop_val32 = (float*)mem.get(sizeof(float) * (tot + 1));
        if (!L.gop_code || !L.gop_val || !L.gop_val32) {
            L.gop_cap = 0;
            err = "out of device memory";
            return SULF_ENOMEM;
        }
        L.gop_cap = tot + 1;
    }
    if (cudaMemcpyAsync(L.gop_ptr, cnt.data(), sizeof(int) * (L.ng + 1), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        err = "ghost relaxation map failed";
        return SULF_EDEVICE;
    }
    if (L.dim == 2)
        k_gop_fill<2><<<nblk(L.ng, bt), bt, shm, s>>>(L.ng, passes, tau, L.gidx, L.gwk, L.gnode, L.gsrc, L.gop_ptr,
                                                      L.gop_code, L.gop_val, L.gop_val32);
    else
        k_gop_fill<3><<<nblk(L.ng, bt), bt, shm, s>>>(L.ng, passes, tau, L.gidx, L.gwk, L.gnode, L.gsrc, L.gop_ptr,
                                                      L.gop_code, L.gop_val, L.gop_val32);
    launches++;
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        err = "ghost relaxation map failed";
        return SULF_EDEVICE;
    }
    L.gop_nnz = tot;
    L.gop_on = true;
    return SULF_OK;
}

int build_ghost_rows(LevelGeo& L, int bc, bool finest, cudaStream_t s, std::string& err, long long& launches) {
    if (L.ng == 0) return SULF_OK;
    const int D = L.dim;
    if (D == 2)
        k_ghost_geom<2><<<nblk(L.ng, 128), 128, 0, s>>>(L.phi, L.type, L.n, L.lo, L.h, L.gidx, L.ng, bc, L.gkind,
                                                        L.gm, L.gw, L.gB, L.gord, L.gth, L.gnt);
    else
        k_ghost_geom<3><<<nblk(L.ng, 128), 128, 0, s>>>(L.phi, L.type, L.n, L.lo, L.h, L.gidx, L.ng, bc, L.gkind,
                                                        L.gm, L.gw, L.gB, L.gord, L.gth, L.gnt);
    k_to_float<<<nblk(L.ng * 3LL * D), kThreads, 0, s>>>(L.gw, L.gw32, L.ng * 3LL * D);
    if (D == 2)
        k_ghost_members<2><<<nblk(L.ng, 128), 128, 0, s>>>(L.ng, L.gidx, L.gm, L.gw, L.gw32, L.gpos, L.st[1], L.st[2],
                                                           bc, L.h, L.gkind, L.gord, L.gth, L.gnt, L.gwk, L.gwk32,
                                                           L.gnode, L.gsrc);
    else
        k_ghost_members<3><<<nblk(L.ng, 128), 128, 0, s>>>(L.ng, L.gidx, L.gm, L.gw, L.gw32, L.gpos, L.st[1], L.st[2],
                                                           bc, L.h, L.gkind, L.gord, L.gth, L.gnt, L.gwk, L.gwk32,
                                                           L.gnode, L.gsrc);
    launches += 3;
    std::vector<int8_t> kinds(L.ng);
    cudaMemcpyAsync(kinds.data(), L.gkind, L.ng, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        err = "ghost geometry failed";
        return SULF_EDEVICE;
    }
    for (int k = 0; k < 3; k++) L.kinds[k] = 0;
    for (int8_t k : kinds) L.kinds[(int)k]++;
    if (finest && L.kinds[2] > 0) {
        char buf[128];
        snprintf(buf, sizeof buf, "%d finest-level ghost(s) have no usable boundary stencil: refine the grid",
                 L.kinds[2]);
        err = buf;
        return SULF_EGEOM;
    }
    return SULF_OK;
}

int build_level_geometry(LevelGeo& L, const LevelGeo* finer, bool finest, bool coarsest, DevMem& mem,
                         cudaStream_t s, std::string& err, long long& launches) {
    const long long nn = L.nn;
    if (!L.phi) {
        L.phi = (double*)mem.get(sizeof(double) * nn);
        if (!L.phi) {
            err = "out of device memory";
            return SULF_ENOMEM;
        }
    }
    if (finer) {
        k_inject_phi<<<nblk(nn), kThreads, 0, s>>>(finer->phi, L.phi, L.n, finer->n, L.dim, nn);
        launches++;
    }
    L.type = (int8_t*)mem.get(nn);
    if (!L.type) {
        err = "out of device memory";
        return SULF_ENOMEM;
    }
    k_classify_inside<<<nblk(nn), kThreads, 0, s>>>(L.phi, L.type, nn);
    k_classify_ghost<<<nblk(nn), kThreads, 0, s>>>(L.type, L.n, L.dim, nn);
    launches += 2;
    if (finest) {
        int* dflag = (int*)mem.get(sizeof(int));
        cudaMemsetAsync(dflag, 0, sizeof(int), s);
        k_check_edge<<<nblk(nn), kThreads, 0, s>>>(L.type, L.n, L.dim, nn, dflag);
        launches++;
        int hflag = 0;
        cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            err = "geometry kernels failed";
            return SULF_EDEVICE;
        }
        if (hflag) {
            err = "an active node lies on the box edge: enlarge the box";
            return SULF_EINVAL;
        }
    }
    for (int c = 0; c < 2; c++) {
        L.nin[c] = compact(c == 0 ? P_IN0 : P_IN1, L, L.inl[c], mem, s, err, launches);
        if (L.nin[c] < 0) return SULF_EDEVICE;
    }
    if (L.nin[0] + L.nin[1] == 0) {
        char buf[96];
        snprintf(buf, sizeof buf, "no inside node at level N=%d", L.N);
        err = buf;
        return SULF_EINVAL;
    }
    L.ng = compact(P_GHOST, L, L.gidx, mem, s, err, launches);
    if (L.ng < 0) return SULF_EDEVICE;
    const int D = L.dim;
    long long ng1 = L.ng + 1;
    L.gpos = (int*)mem.get(sizeof(int) * nn);
    L.gkind = (int8_t*)mem.get(ng1);
    L.gm = (int8_t*)mem.get(ng1 * D);
    L.gw = (double*)mem.get(sizeof(double) * ng1 * D * 3);
    L.gw32 = (float*)mem.get(sizeof(float) * ng1 * D * 3);
    L.gB = (double*)mem.get(sizeof(double) * ng1 * D);
    const long long K = D == 2 ? 9 : 27;
    L.gwk = (double*)mem.get(sizeof(double) * ng1 * K);
    L.gwk32 = (float*)mem.get(sizeof(float) * ng1 * K);
    L.gnode = (int*)mem.get(sizeof(int) * ng1 * K);
    L.gsrc = (int*)mem.get(sizeof(int) * ng1 * K);
    L.gord = (int8_t*)mem.get(ng1 * D);
    L.gth = (double*)mem.get(sizeof(double) * ng1 * D);
    L.gnt = (double*)mem.get(sizeof(double) * ng1 * D);
    if (!L.gpos || !L.gkind || !L.gm || !L.gw || !L.gw32 || !L.gB || !L.gwk || !L.gwk32 || !L.gnode || !L.gsrc ||
        !L.gord || !L.gth || !L.gnt) {
        err = "out of device memory";
        return SULF_ENOMEM;
    }
    cudaMemsetAsync(L.gpos, 0xff, sizeof(int) * nn, s);
    if (L.ng > 0) {
        k_scatter_pos<<<nblk(L.ng), kThreads, 0, s>>>(L.gidx, L.ng, L.gpos);
        launches++;
    }
    {
        int rc = build_ghost_rows(L, 0, finest, s, err, launches);
        if (rc) return rc;
    }
    // band: inactive nodes within Chebyshev distance 2 of a ghost
    int8_t* mark = (int8_t*)mem.get(nn);
    if (!mark) {
        err = "out of device memory";
        return SULF_ENOMEM;
    }
    cudaMemsetAsync(mark, 0, nn, s);
    k_band_mark<<<nblk(nn), kThreads, 0, s>>>(L.type, mark, L.n, D, nn, 1);
    k_band_mark<<<nblk(nn), kThreads, 0, s>>>(L.type, mark, L.n, D, nn, 2);
    k_band_set<<<nblk(nn), kThreads, 0, s>>>(L.type, mark, nn);
    launches += 3;
    L.nb = compact(P_BAND, L, L.bidx, mem, s, err, launches);
    if (L.nb < 0) return SULF_EDEVICE;
    long long nb1 = L.nb + 1;
    L.bref = (int*)mem.get(sizeof(int) * nb1 * D);
    L.ban = (double*)mem.get(sizeof(double) * nb1 * D);
    L.ban32 = (float*)mem.get(sizeof(float) * nb1 * D);
    int* bpos = (int*)mem.get(sizeof(int) * nn);
    if (!L.bref || !L.ban || !L.ban32 || !bpos) {
        err = "out of device memory";
        return SULF_ENOMEM;
    }
    if (L.nb > 0) {
        cudaMemsetAsync(bpos, 0xff, sizeof(int) * nn, s);
        k_scatter_pos<<<nblk(L.nb), kThreads, 0, s>>>(L.bidx, L.nb, bpos);
        k_band_info<<<nblk(L.nb), kThreads, 0, s>>>(L.phi, L.type, L.n, D, L.h, L.bidx, L.nb, bpos, L.bref, L.ban);
        k_to_float<<<nblk(L.nb * (long long)D), kThreads, 0, s>>>(L.ban, L.ban32, L.nb * (long long)D);
        launches += 3;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        err = "band construction failed";
        return SULF_EDEVICE;
    }
    // the band extension operator: per-node entry counts, host scan, fill
    {
        const double cfl = D == 2 ? 0.5 : 1.0 / 3.0;
        L.eptr = (int*)mem.get(sizeof(int) * nb1);
        if (!L.eptr) {
            err = "out of device memory";
            return SULF_ENOMEM;
        }
        std::vector<int> cnt(L.nb + 1, 0);
        if (L.nb > 0) {
            if (D == 2)
                k_ext_count<2><<<nblk(L.nb, 128), 128, 0, s>>>(L.nb, L.bref, L.ban, cfl, L.eptr);
            else
                k_ext_count<3><<<nblk(L.nb, 128), 128, 0, s>>>(L.nb, L.bref, L.ban, cfl, L.eptr);
            launches++;
            if (cudaMemcpyAsync(cnt.data(), L.eptr, sizeof(int) * L.nb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess) {
                err = "band extension operator failed";
                return SULF_EDEVICE;
            }
        }
        std::vector<int> ptr(L.nb + 1, 0);
        long long tot = 0;
        for (int b = 0; b < L.nb; b++) {
            if (cnt[b] < 0) {
                err = "band extension reaches more ghosts than supported";
                return SULF_EGEOM;
            }
            ptr[b] = (int)tot;
            tot += cnt[b];
        }
        ptr[L.nb] = (int)tot;
        L.ne = tot;
        L.eidx = (int*)mem.get(sizeof(int) * (tot + 1));
        L.eval = (double*)mem.get(sizeof(double) * (tot + 1));
        L.eval32 = (float*)mem.get(sizeof(float) * (tot + 1));
        if (!L.eidx || !L.eval || !L.eval32) {
            err = "out of device memory";
            return SULF_ENOMEM;
        }
        if (cudaMemcpyAsync(L.eptr, ptr.data(), sizeof(int) * (L.nb + 1), cudaMemcpyHostToDevice, s) != cudaSuccess) {
            err = "band extension operator failed";
            return SULF_EDEVICE;
        }
        if (L.nb > 0) {
            if (D == 2)
                k_ext_fill<2><<<nblk(L.nb, 128), 128, 0, s>>>(L.nb, L.bref, L.ban, cfl, L.eptr, L.eidx, L.eval,
                                                              L.eval32);
            else
                k_ext_fill<3><<<nblk(L.nb, 128), 128, 0, s>>>(L.nb, L.bref, L.ban, cfl, L.eptr, L.eidx, L.eval,
                                                              L.eval32);
            launches++;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            err = "band extension operator failed";
            return SULF_EDEVICE;
        }
    }
    if (coarsest) {
        L.nact = compact(P_ACTIVE, L, L.act, mem, s, err, launches);
        if (L.nact < 0) return SULF_EDEVICE;
        L.apos = (int*)mem.get(sizeof(int) * nn);
        if (!L.apos) {
            err = "out of device memory";
            return SULF_ENOMEM;
        }
        cudaMemsetAsync(L.apos, 0xff, sizeof(int) * nn, s);
        k_scatter_pos<<<nblk(L.nact), kThreads, 0, s>>>(L.act, L.nact, L.apos);
        launches++;
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            err = "coarsest-level lists failed";
            return SULF_EDEVICE;
        }
    }
    return SULF_OK;
}

}  // namespace sulf
