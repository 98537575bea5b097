// Per-node stages of the multigrid cycle (arXiv:1902.07029, Sec. 3.5), shared
// by the per-level kernels (kernels.cu) and the fused coarse-level cycle
// (tail.cu), so each stage's arithmetic has one definition.
//
// Load policy CG: when true, data that the same kernel may have written in an
// earlier phase (x, rhs, res, ghost and band buffers) is read with
// ld.global.cg, i.e. from L2, never from a possibly stale L1 line of another
// SM; the per-level kernels use plain loads.
#pragma once

#include "sulf_internal.cuh"

namespace sulf {
namespace stages {

template <bool CG, typename V>
__device__ __forceinline__ V ldx(const V* p) {
    if (CG) return __ldcg(p);
    return *p;
}

// box coordinates of node p on a grid of n nodes per axis: node indices fit
// in 32 bits, and unsigned 32-bit division costs a small fraction of the
// 64-bit one
template <int D>
__device__ __forceinline__ void box_coords(long long p, int n, int* ii) {
    const unsigned u = (unsigned)p, un = (unsigned)n;
    const unsigned q = u / un;
    ii[0] = (int)(u - q * un);
    if (D == 3) {
        const unsigned r = q / un;
        ii[1] = (int)(q - r * un);
        ii[2] = (int)r;
    } else {
        ii[1] = (int)q;
        ii[2] = 0;
    }
}

template <typename T>
__device__ __forceinline__ unsigned long long abs_bits(T v) {
    double d = fabs((double)v);
    return (unsigned long long)__double_as_longlong(d);
}

// node of list position t in the concatenation (inside colour 0, inside
// colour 1, ghosts); kind 1 inside, 2 ghost
struct Lists {
    const int* l0;
    const int* l1;
    const int* lg;
    int n0, n1, ng;
};

__device__ __forceinline__ long long list_node(const Lists& L, int t, int& kind, int& gi) {
    if (t < L.n0) {
        kind = 1;
        return L.l0[t];
    }
    t -= L.n0;
    if (t < L.n1) {
        kind = 1;
        return L.l1[t];
    }
    t -= L.n1;
    kind = 2;
    gi = t;
    return L.lg[t];
}

inline Lists make_lists(const LevelGeo& L) {
    Lists l;
    l.l0 = L.inl[0];
    l.l1 = L.inl[1];
    l.lg = L.gidx;
    l.n0 = L.nin[0];
    l.n1 = L.nin[1];
    l.ng = L.ng;
    return l;
}

// pointers of the stencil coefficients of a level
template <int D, typename T>
struct CoefPtr {
    typedef typename V2<T>::t T2;
    const T2* edge[3];
    const T2* Pa;
    const T2* Pb;
    const T2* Ia;
    const T2* Ib;
    const T2* gc;
    // (Pa, Pb) and (Ia, Ib) per inside-list position (null: read the box arrays)
    const T2* Pc;
    const T2* Ic;
};

template <int D, typename T>
inline CoefPtr<D, T> coef_ptr(const LevelVec<T>& V) {
    CoefPtr<D, T> c;
    for (int a = 0; a < 3; a++) c.edge[a] = V.edge[a];
    c.Pa = V.Pa;
    c.Pb = V.Pb;
    c.Ia = V.Ia;
    c.Ib = V.Ib;
    c.gc = V.gc;
    c.Pc = V.Pc;
    c.Ic = V.Ic;
    return c;
}

__device__ __forceinline__ double fmadd(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// b_s minus the off-diagonal part of the s row of inside node p applied to x
// (Eq. JssI and Eq. JscI as exact derivatives): over the axis neighbours q,
// J^ss_pq = -g and J^sc_pq = +-e, so b_s - sum_q (J^ss_pq x^s_q + J^sc_pq x^c_q)
// is one chain of 4 fused multiply-adds per axis.  FP64 issue rate is the
// scarce resource on this GPU, so the chain is written out explicitly.
template <int D, typename T, bool CG>
__device__ __forceinline__ T s_defect(T bs, long long p, const typename V2<T>::t* ge, const typename V2<T>::t* gw,
                                      const typename V2<T>::t* x, const long long* st) {
    typedef typename V2<T>::t T2;
    T r = bs;
#pragma unroll
    for (int a = 0; a < D; a++) {
        T2 xe = ldx<CG>(x + p + st[a]);
        T2 xw = ldx<CG>(x + p - st[a]);
        r = fmadd(ge[a].x, xe.x, r);
        r = fmadd(-ge[a].y, xe.y, r);
        r = fmadd(gw[a].x, xw.x, r);
        r = fmadd(gw[a].y, xw.y, r);
    }
    return r;
}

// The coefficients an inside-node update needs, all fixed during a linear
// solve: the edge pairs toward the +axis neighbours (ge) and from the -axis
// neighbours (gw), and the rows of P^{-1} (collective) or of P (pointwise).
template <int D, typename T>
struct InsideCoef {
    typedef typename V2<T>::t T2;
    T2 ge[D], gw[D];
    T2 m0, m1;
};

template <int D, typename T, bool PW>
__device__ __forceinline__ InsideCoef<D, T> fetch_inside(long long p, const CoefPtr<D, T>& cf, const long long* st) {
    InsideCoef<D, T> k;
#pragma unroll
    for (int a = 0; a < D; a++) {
        k.ge[a] = cf.edge[a][p];
        k.gw[a] = cf.edge[a][p - st[a]];
    }
    k.m0 = PW ? cf.Pa[p] : cf.Ia[p];
    k.m1 = PW ? cf.Pb[p] : cf.Ib[p];
    return k;
}

// the same for the inside node p at position t of the inside lists, the 2x2
// block (or its inverse) read from the list-ordered copy where there is one
template <int D, typename T, bool PW>
__device__ __forceinline__ InsideCoef<D, T> fetch_inside_at(long long p, int t, const CoefPtr<D, T>& cf,
                                                            const long long* st) {
    InsideCoef<D, T> k;
#pragma unroll
    for (int a = 0; a < D; a++) {
        k.ge[a] = cf.edge[a][p];
        k.gw[a] = cf.edge[a][p - st[a]];
    }
    const typename V2<T>::t* c = PW ? cf.Pc : cf.Ic;
    if (c) {
        k.m0 = c[2 * (long long)t];
        k.m1 = c[2 * (long long)t + 1];
    } else {
        k.m0 = PW ? cf.Pa[p] : cf.Ia[p];
        k.m1 = PW ? cf.Pb[p] : cf.Ib[p];
    }
    return k;
}

// collective (Eq. matrixP) or pointwise (Eq. matrixPclassical) update of the
// inside node p from its fetched coefficients: x_p <- P^{-1} (b - (J - P) x),
// resp. the diagonal of P
template <int D, typename T, bool PW, bool CG>
__device__ __forceinline__ void relax_apply_b(long long p, const InsideCoef<D, T>& k, typename V2<T>::t b,
                                              typename V2<T>::t* x, const long long* st) {
    typedef typename V2<T>::t T2;
    T r = s_defect<D, T, CG>(b.x, p, k.ge, k.gw, x, st);
    T2 out;
    if (PW) {
        T2 xp = ldx<CG>(x + p);
        out.x = fmadd(-k.m0.y, xp.y, r) / k.m0.x;
        out.y = fmadd(-k.m1.x, xp.x, b.y) / k.m1.y;
    } else {
        out.x = fmadd(k.m0.x, r, k.m0.y * b.y);
        out.y = fmadd(k.m1.x, r, k.m1.y * b.y);
    }
    x[p] = out;
}

// the same with b = rhs(p)
template <int D, typename T, bool PW, bool CG>
__device__ __forceinline__ void relax_apply(long long p, const InsideCoef<D, T>& k, const typename V2<T>::t* rhs,
                                            typename V2<T>::t* x, const long long* st) {
    relax_apply_b<D, T, PW, CG>(p, k, ldx<CG>(rhs + p), x, st);
}

// Matrix-free FP32 collective update (Eq. matrixP with the Jacobian entries
// of Eqs. JssI, JscI, JcsI, JccI formed from Wc on the fly): the stencil
// coefficients of inside node p and the inverse of its 2x2 block, from the
// (s, c) of the node and its axis neighbours (neighbour order +a, -a per axis)
template <int D>
struct MfCoef {
    float g[2 * D], e[2 * D];
    float i00, i01, i10, i11;
};

template <int D>
__device__ __forceinline__ MfCoef<D> mf_coef(long long p, const float2* Wc, const Coef<float>& c, const long long* st) {
    MfCoef<D> k;
    const float2 w = Wc[p];
    const float s = w.x, cp = w.y;
    const float ph = c.alpha * cp + c.beta;
    float sg = 0, se = 0;
#pragma unroll
    for (int a = 0; a < D; a++) {
#pragma unroll
        for (int dir = 0; dir < 2; dir++) {
            const float2 wq = Wc[dir ? p - st[a] : p + st[a]];
            const float gq = c.kap * ((c.alpha * wq.y + c.beta) + ph);
            const float eq = c.kap * c.alpha * (s - wq.x);
            k.g[2 * a + dir] = gq;
            k.e[2 * a + dir] = eq;
            sg += gq;
            se += eq;
        }
    }
    const float Pcs = c.a2ms * ph * cp;
    const float Pcc = c.idt + c.a2ms * (c.alpha * s * cp + ph * s);
    const float Pss = ph * c.idt + c.a2mc * ph * cp + sg;
    const float Psc = c.alpha * s * c.idt + c.a2mc * (c.alpha * s * cp + ph * s) + se;
    const float inv = 1.0f / (Pss * Pcc - Psc * Pcs);
    k.i00 = Pcc * inv;
    k.i01 = -Psc * inv;
    k.i10 = -Pcs * inv;
    k.i11 = Pss * inv;
    return k;
}

// x_p <- P^{-1} (b - (J - P) x) from the coefficients of mf_coef
template <int D>
__device__ __forceinline__ void mf_apply(long long p, const MfCoef<D>& k, const float2* rhs, float2* x,
                                         const long long* st) {
    const float2 b = rhs[p];
    float r = b.x;
#pragma unroll
    for (int a = 0; a < D; a++) {
        const float2 xe = x[p + st[a]];
        const float2 xw = x[p - st[a]];
        r = __fmaf_rn(k.g[2 * a], xe.x, r);
        r = __fmaf_rn(-k.e[2 * a], xe.y, r);
        r = __fmaf_rn(k.g[2 * a + 1], xw.x, r);
        r = __fmaf_rn(-k.e[2 * a + 1], xw.y, r);
    }
    float2 out;
    out.x = __fmaf_rn(k.i00, r, k.i01 * b.y);
    out.y = __fmaf_rn(k.i10, r, k.i11 * b.y);
    x[p] = out;
}

// relax_value when every x is zero (the coarse-grid error right after
// restriction): the same operations with zero operands, so the same bits
template <int D, typename T, bool PW>
__device__ __forceinline__ typename V2<T>::t relax_value_zero(typename V2<T>::t b, const InsideCoef<D, T>& k) {
    typedef typename V2<T>::t T2;
    const T z = 0;
    T r = b.x;
#pragma unroll
    for (int a = 0; a < D; a++) {
        r = fmadd(k.ge[a].x, z, r);
        r = fmadd(-k.ge[a].y, z, r);
        r = fmadd(k.gw[a].x, z, r);
        r = fmadd(k.gw[a].y, z, r);
    }
    T2 out;
    if (PW) {
        out.x = fmadd(-k.m0.y, z, r) / k.m0.x;
        out.y = fmadd(-k.m1.x, z, b.y) / k.m1.y;
    } else {
        out.x = fmadd(k.m0.x, r, k.m0.y * b.y);
        out.y = fmadd(k.m1.x, r, k.m1.y * b.y);
    }
    return out;
}

template <int D, typename T, bool PW, bool CG>
__device__ __forceinline__ void relax_node(long long p, const CoefPtr<D, T>& cf, const typename V2<T>::t* rhs,
                                           typename V2<T>::t* x, const long long* st) {
    InsideCoef<D, T> k = fetch_inside<D, T, PW>(p, cf, st);
    relax_apply<D, T, PW, CG>(p, k, rhs, x, st);
}

// the same for the node at position t of the inside lists
template <int D, typename T, bool PW, bool CG>
__device__ __forceinline__ void relax_node_at(long long p, int t, const CoefPtr<D, T>& cf,
                                              const typename V2<T>::t* rhs, typename V2<T>::t* x,
                                              const long long* st) {
    InsideCoef<D, T> k = fetch_inside_at<D, T, PW>(p, t, cf, st);
    relax_apply<D, T, PW, CG>(p, k, rhs, x, st);
}

// Ghost boundary rows s~(B) (Eq. JssD) as member tables built once per level:
// member kk of the upwind 3^D stencil of ghost gi has weight w (the tensor
// product of the 1-D weights, 0 when absent), box node and ghost index (or -1),
// stored member-major (kk * ng + gi) so a warp's loads of a member coalesce.
template <typename T>
struct GhostTab {
    const T* w;
    const int* node;
    const int* src;
    int ng;
};

template <typename T>
inline GhostTab<T> ghost_tab(const LevelGeo& L) {
    GhostTab<T> t;
    t.w = std::is_same<T, float>::value ? (const T*)L.gwk32 : (const T*)L.gwk;
    t.node = L.gnode;
    t.src = L.gsrc;
    t.ng = L.ng;
    return t;
}

// nine members of one row
template <typename T>
struct Members {
    T w[9];
    int node[9];
    int src[9];
};

template <typename T>
__device__ __forceinline__ void fetch_members(const GhostTab<T>& tb, int gi, int k0, Members<T>& m) {
#pragma unroll
    for (int j = 0; j < 9; j++) {
        const long long o = (long long)(k0 + j) * tb.ng + gi;
        m.w[j] = tb.w[o];
        m.node[j] = tb.node[o];
        m.src[j] = tb.src[o];
    }
}

// acc plus nine members of the row applied to the s component.  Ghost members
// come from the previous relaxation pass (sin) unless from_x.  Every load is
// issued before any value is used, then the terms are summed in member order.
template <typename T, bool CG>
__device__ __forceinline__ T members_dot(const Members<T>& m, const typename V2<T>::t* x, const T* sin, bool from_x,
                                         T acc) {
    T v[9];
#pragma unroll
    for (int j = 0; j < 9; j++) {
        const T* a = reinterpret_cast<const T*>(x + m.node[j]);
        if (!from_x && m.src[j] >= 0) a = sin + m.src[j];
        v[j] = m.w[j] != (T)0 ? ldx<CG>(a) : (T)0;
    }
#pragma unroll
    for (int j = 0; j < 9; j++)
        if (m.w[j] != (T)0) acc += m.w[j] * v[j];
    return acc;
}

// the whole row: in 2-D from the members fetched ahead (pre), in 3-D fetched
// here nine at a time
template <int D, typename T, bool CG>
__device__ __forceinline__ T row_dot(const GhostTab<T>& tb, int gi, const Members<T>* pre,
                                     const typename V2<T>::t* x, const T* sin, bool from_x) {
    if (D == 2 && pre) return members_dot<T, CG>(*pre, x, sin, from_x, (T)0);
    const int K = D == 2 ? 9 : 27;
    T acc = 0;
#pragma unroll 1
    for (int c0 = 0; c0 < K; c0 += 9) {
        Members<T> m;
        fetch_members<T>(tb, gi, c0, m);
        acc = members_dot<T, CG>(m, x, sin, from_x, acc);
    }
    return acc;
}

// one Jacobi pass of the ghost relaxation (Eq. RelGhost) for ghost gi at node
// g: s_g += tau (r_g - row . x) from the previous pass's values, then the ghost
// c row J^cs_gg s_g + J^cc_gg c_g = r^c_g solved for c_g with the fresh s_g
// (q = (J^cs_gg, J^cc_gg), qinv = 1 / J^cc_gg)
template <int D, typename T, bool CG>
__device__ __forceinline__ void ghost_pass_apply(int gi, long long g, const GhostTab<T>& tb, const Members<T>* pre,
                                                 typename V2<T>::t q, T qinv, const typename V2<T>::t* rhs,
                                                 typename V2<T>::t* x, const T* sin, T* sout, T tau, bool first,
                                                 bool last) {
    typedef typename V2<T>::t T2;
    T acc = row_dot<D, T, CG>(tb, gi, pre, x, sin, first);
    T2 xg = ldx<CG>(x + g);
    T s_old = first ? xg.x : ldx<CG>(sin + gi);
    T2 b = ldx<CG>(rhs + g);
    T s_new = s_old + tau * (b.x - acc);
    T c_new = fmadd(-q.x, s_new, b.y) * qinv;
    T* xs = reinterpret_cast<T*>(x + g);
    xs[1] = c_new;
    if (last)
        xs[0] = s_new;
    else
        sout[gi] = s_new;
}

template <int D, typename T, bool CG>
__device__ __forceinline__ void ghost_pass_node(int gi, const int* gidx, const GhostTab<T>& tb,
                                                const typename V2<T>::t* gc, const T* gci,
                                                const typename V2<T>::t* rhs, typename V2<T>::t* x, const T* sin,
                                                T* sout, T tau, bool first, bool last) {
    Members<T> m;
    const Members<T>* pre = nullptr;
    if (D == 2) {
        fetch_members<T>(tb, gi, 0, m);
        pre = &m;
    }
    ghost_pass_apply<D, T, CG>(gi, gidx[gi], tb, pre, gc[gi], gci[gi], rhs, x, sin, sout, tau, first, last);
}

// The composed ghost relaxation (all passes of a sweep as one affine map per
// ghost, built in geometry.cu).  An entry's code names its input: the s of box
// node code (code >= 0, an inside member), else with u = ~code the s of ghost
// u >> 1 before the passes (u even, from the copy snap) or the right-hand side
// of box node u >> 1 (u odd).
constexpr int kGopLanes = 8;

template <typename T>
__device__ __forceinline__ T gop_input(int code, const typename V2<T>::t* x, const typename V2<T>::t* rhs,
                                       const T* snap) {
    if (code >= 0) return reinterpret_cast<const T*>(x + code)[0];
    const unsigned u = ~(unsigned)code;
    return (u & 1u) ? reinterpret_cast<const T*>(rhs + (u >> 1))[0] : snap[u >> 1];
}

// The lanes of a group of kGopLanes (aligned within a warp) share one row:
// lane k sums the entries beg + k, beg + k + kGopLanes, ... (one FMA chain
// from zero), then the lane sums are combined by xor shuffles (lane 0 with 4,
// then 2, then 1).  Every lane of the warp must call it.
template <typename T>
__device__ __forceinline__ T gop_reduce(T acc) {
#pragma unroll
    for (int o = kGopLanes / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// the row of ghost gi by the kGopLanes lanes of its group (lane ln; on:
// whether the group has a row), then lane 0 solves the ghost's c row with the
// new s_g (as in ghost_pass_apply); every lane of the warp must call it
// the row of ghost gi by the kGopLanes lanes of its group (lane ln; on:
// whether the group has a row), then lane 0 solves the ghost's c row with the
// new s_g (as in ghost_pass_apply; gci = 1 / J^cc_gg); every lane of the warp
// must call it
template <typename T>
__device__ __forceinline__ void gop_group(bool on, int ln, int gi, const int* ptr, const int* code, const T* val,
                                          const int* gidx, const typename V2<T>::t* gc, const T* gci,
                                          const typename V2<T>::t* rhs, typename V2<T>::t* x, const T* snap) {
    T acc = 0;
    if (on)
        for (int j = ptr[gi] + ln; j < ptr[gi + 1]; j += kGopLanes)
            acc = fmadd(val[j], gop_input<T>(code[j], x, rhs, snap), acc);
    acc = gop_reduce<T>(acc);
    if (!on || ln != 0) return;
    const long long g = gidx[gi];
    const typename V2<T>::t q = gc[gi];
    typename V2<T>::t r;
    r.x = acc;
    r.y = fmadd(-q.x, acc, reinterpret_cast<const T*>(rhs + g)[1]) * gci[gi];
    x[g] = r;
}

// defect r = rhs - J x at node p of kind 1 (inside, coefficients k) or 2
// (ghost gi, its row and c-row q); returns max(|r_s|, |r_c|) as bits
// the defect stored in res's element type (an FP64 defect into FP32: the
// next right-hand side of the mixed form's FP32 cycle, rounded to nearest)
__device__ __forceinline__ void store_res(double2* res, long long p, double2 r) { res[p] = r; }
__device__ __forceinline__ void store_res(float2* res, long long p, float2 r) { res[p] = r; }
__device__ __forceinline__ void store_res(float2* res, long long p, double2 r) {
    res[p] = make_float2((float)r.x, (float)r.y);
}

// (rhsc: the list-ordered copy of rhs, read at list position t, or null)
template <int D, typename T, bool CG, typename R2>
__device__ __forceinline__ unsigned long long residual_apply(long long p, int kind, int gi, const InsideCoef<D, T>& k,
                                                             const GhostTab<T>& tb, const Members<T>* pre,
                                                             typename V2<T>::t q, const typename V2<T>::t* rhs,
                                                             const typename V2<T>::t* x, R2* res,
                                                             long long st1, long long st2,
                                                             const typename V2<T>::t* rhsc = nullptr, int t = 0) {
    typedef typename V2<T>::t T2;
    T2 b = rhsc ? rhsc[t] : ldx<CG>(rhs + p);
    T2 xp = ldx<CG>(x + p);
    T2 r;
    if (kind == 1) {
        const long long st[3] = {1, st1, st2};
        T rs = s_defect<D, T, CG>(b.x, p, k.ge, k.gw, x, st);
        r.x = fmadd(-k.m0.y, xp.y, fmadd(-k.m0.x, xp.x, rs));
        r.y = fmadd(-k.m1.y, xp.y, fmadd(-k.m1.x, xp.x, b.y));
    } else {
        T acc = row_dot<D, T, CG>(tb, gi, pre, x, nullptr, true);
        r.x = b.x - acc;
        r.y = b.y - (q.x * xp.x + q.y * xp.y);
    }
    store_res(res, p, r);
    unsigned long long a0 = abs_bits(r.x), a1 = abs_bits(r.y);
    return a0 > a1 ? a0 : a1;
}

// the fixed data of the defect at list position t (in 2-D a ghost's members)
template <int D, typename T>
__device__ __forceinline__ long long fetch_residual(int t, const Lists& ls, const GhostTab<T>& tb,
                                                   const CoefPtr<D, T>& cf, long long st1, long long st2, int& kind,
                                                   int& gi, InsideCoef<D, T>& k, Members<T>& m,
                                                   typename V2<T>::t& q) {
    gi = 0;
    long long p = list_node(ls, t, kind, gi);
    if (kind == 1) {
        const long long st[3] = {1, st1, st2};
        k = fetch_inside_at<D, T, true>(p, t, cf, st);
    } else {
        if (D == 2) fetch_members<T>(tb, gi, 0, m);
        q = cf.gc[gi];
    }
    return p;
}

template <int D, typename T, bool CG, typename R2>
__device__ __forceinline__ unsigned long long residual_node(int t, const Lists& ls, const GhostTab<T>& tb,
                                                            const CoefPtr<D, T>& cf, const typename V2<T>::t* rhs,
                                                            const typename V2<T>::t* x, R2* res, long long st1,
                                                            long long st2, const typename V2<T>::t* rhsc = nullptr) {
    int kind, gi;
    InsideCoef<D, T> k;
    Members<T> m;
    typename V2<T>::t q;
    long long p = fetch_residual<D, T>(t, ls, tb, cf, st1, st2, kind, gi, k, m, q);
    return residual_apply<D, T, CG>(p, kind, gi, k, tb, D == 2 ? &m : nullptr, q, rhs, x, res, st1, st2, rhsc, t);
}

// The ghost defect extended into the band along the normal (Sec. 3.5.2): the
// explicit upwind steps are linear in the ghost defects, so the extended value
// at band node b is a precomputed weighted sum of ghost defects (CSR row b of
// eptr/eidx/eval, built with the geometry).  Ghost nodes are never band nodes,
// so all band nodes update at once.
template <typename T>
struct ExtRow {
    static constexpr int kAhead = 8;  // entries fetched ahead of the wait
    int j0, j1, node;
    int idx[kAhead];
    T w[kAhead];
};

template <typename T>
__device__ __forceinline__ ExtRow<T> fetch_ext(int b, const int* eptr, const int* eidx, const T* eval,
                                               const int* bidx) {
    ExtRow<T> r;
    r.j0 = eptr[b];
    r.j1 = eptr[b + 1];
    r.node = bidx[b];
#pragma unroll
    for (int j = 0; j < ExtRow<T>::kAhead; j++) {
        const bool on = r.j0 + j < r.j1;
        r.idx[j] = on ? eidx[r.j0 + j] : 0;
        r.w[j] = on ? eval[r.j0 + j] : (T)0;
    }
    return r;
}

template <typename T, bool CG>
__device__ __forceinline__ void extend_apply(const ExtRow<T>& r, const int* eidx, const T* eval,
                                             typename V2<T>::t* res) {
    typedef typename V2<T>::t T2;
    T2 v[ExtRow<T>::kAhead];
#pragma unroll
    for (int j = 0; j < ExtRow<T>::kAhead; j++) {
        v[j].x = 0;
        v[j].y = 0;
        if (r.j0 + j < r.j1) v[j] = ldx<CG>(res + r.idx[j]);
    }
    T sx = 0, sy = 0;
#pragma unroll
    for (int j = 0; j < ExtRow<T>::kAhead; j++) {
        if (r.j0 + j >= r.j1) break;
        sx += r.w[j] * v[j].x;
        sy += r.w[j] * v[j].y;
    }
    for (int j = r.j0 + ExtRow<T>::kAhead; j < r.j1; j++) {
        T2 u = ldx<CG>(res + eidx[j]);
        T w = eval[j];
        sx += w * u.x;
        sy += w * u.y;
    }
    T2 out;
    out.x = sx;
    out.y = sy;
    res[r.node] = out;
}

template <typename T, bool CG>
__device__ __forceinline__ void extend_node(int b, const int* eptr, const int* eidx, const T* eval, const int* bidx,
                                            typename V2<T>::t* res) {
    ExtRow<T> r = fetch_ext<T>(b, eptr, eidx, eval, bidx);
    extend_apply<T, CG>(r, eidx, eval, res);
}

__device__ __forceinline__ bool valid_for(int8_t rule, int8_t t) {
    return rule == T_IN ? t == T_IN : (t == T_GHOST || t == T_BAND);
}

// The fixed part of the boundary-aware full weighting (Eqs. Fstencil,
// Fstencilgen, Fig. Neigh) at coarse node I: the fine twin f, the per-axis
// mirrored 1-D weights times 4 -- (1,2,1), (2,2,0), (0,2,2) or (0,4,0) --, the
// members that hold a value of the rule's kind (bit kk), and the weight moved
// to the centre (the centre's own plus that of every member without a value).
// A member's weight is the product of its axes' weights over 4^D: a power of
// two, built from its exponent with integer operations, so the weights cost
// no FP64 instruction (FP64 issues at two lanes per SM and clock on this GPU)
// and are exactly the products the paper's per-axis rule gives.
template <int D, typename T>
struct RestrictGeo {
    long long I, f;
    unsigned char e1[3][3];  // per-axis weight times 4 as log2 + 1 (0: weight 0)
    unsigned valid;
    int iwc;                 // centre weight times 4^D
    bool full;               // (1,2,1) on every axis and every member valid
};

// 2^(e - 2D) in T for a member whose per-axis exponents sum to e
template <int D, typename T>
__device__ __forceinline__ T pow2_weight(int e);
template <>
__device__ __forceinline__ double pow2_weight<2, double>(int e) {
    return __longlong_as_double((long long)(1023 + e - 4) << 52);
}
template <>
__device__ __forceinline__ double pow2_weight<3, double>(int e) {
    return __longlong_as_double((long long)(1023 + e - 6) << 52);
}
template <>
__device__ __forceinline__ float pow2_weight<2, float>(int e) {
    return __int_as_float((127 + e - 4) << 23);
}
template <>
__device__ __forceinline__ float pow2_weight<3, float>(int e) {
    return __int_as_float((127 + e - 6) << 23);
}

template <int D, typename T>
__device__ __forceinline__ RestrictGeo<D, T> fetch_restrict(int t, const Lists& ls, const int8_t* ctype, int cn,
                                                            const int8_t* ftype, int fn) {
    RestrictGeo<D, T> g;
    int kind, gi;
    g.I = list_node(ls, t, kind, gi);
    const long long I = g.I;
    int8_t rule = ctype[I];
    int ii[3];
    box_coords<D>(I, cn, ii);
    const long long fst[3] = {1, fn, (long long)fn * fn};
    long long f = 0;
#pragma unroll
    for (int a = 0; a < D; a++) f += 2LL * ii[a] * fst[a];
    g.f = f;
    bool std_axes = true;
#pragma unroll
    for (int a = 0; a < D; a++) {
        bool vl = ii[a] > 0 && valid_for(rule, ftype[f - fst[a]]);
        bool vr = 2 * ii[a] < fn - 1 && valid_for(rule, ftype[f + fst[a]]);
        // log2(weight * 4) + 1: 1 -> 1, 2 -> 2, 4 -> 3, 0 -> 0
        unsigned char l = 1, m = 2, r = 1;
        if (vl && !vr) {
            l = 2; m = 2; r = 0;
        } else if (!vl && vr) {
            l = 0; m = 2; r = 2;
        } else if (!vl && !vr) {
            l = 0; m = 3; r = 0;
        }
        std_axes = std_axes && vl && vr;
        g.e1[a][0] = l;
        g.e1[a][1] = m;
        g.e1[a][2] = r;
    }
    const int K = D == 2 ? 9 : 27;
    g.valid = 0;
    g.iwc = 0;
#pragma unroll
    for (int kk = 0; kk < K; kk++) {
        const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = kk / 9;
        const int e0 = g.e1[0][k0], ea = g.e1[1][k1], eb = D == 3 ? g.e1[2][k2] : 1;
        if (e0 == 0 || ea == 0 || eb == 0) continue;
        const int iw = 1 << (e0 + ea + eb - 3);  // weight times 4^D
        bool centre = k0 == 1 && k1 == 1 && (D == 2 || k2 == 1);
        long long node = f + (k0 - 1) * fst[0] + (k1 - 1) * fst[1];
        if (D == 3) node += (k2 - 1) * fst[2];
        if (centre || !valid_for(rule, ftype[node]))
            g.iwc += iw;
        else
            g.valid |= 1u << kk;
    }
    const unsigned all = (D == 2 ? 0x1ffu : 0x7ffffffu) & ~(1u << (D == 2 ? 4 : 13));
    g.full = std_axes && g.valid == all;
    return g;
}

// the weighting applied to the fine defect (members in box order, then the
// centre with the weight moved to it); also zeroes the coarse error, or, for a
// red inside node whose coefficients red holds, sets it to the first red
// relaxation from zero (relax_value_zero)
// (crhsc: the coarse level's list-ordered copy of its right-hand side, or
// null; t: the coarse node's list position)
template <int D, typename T, bool CG, bool PW = false>
__device__ __forceinline__ void restrict_apply(const RestrictGeo<D, T>& g, int fn, const typename V2<T>::t* fres,
                                               typename V2<T>::t* crhs, typename V2<T>::t* cx,
                                               const InsideCoef<D, T>* red = nullptr,
                                               typename V2<T>::t* crhsc = nullptr, int t = 0) {
    typedef typename V2<T>::t T2;
    const long long fst[3] = {1, fn, (long long)fn * fn};
    const int K = D == 2 ? 9 : 27;
    T as = 0, ac = 0;
    T2 vc = ldx<CG>(fres + g.f);
#pragma unroll
    for (int c0 = 0; c0 < K; c0 += 9) {
        T2 v[9];
#pragma unroll
        for (int j = 0; j < 9; j++) {
            const int kk = c0 + j;
            const int k0 = kk % 3 - 1, k1 = (kk / 3) % 3 - 1, k2 = kk / 9 - 1;
            long long node = g.f + k0 * fst[0] + k1 * fst[1];
            if (D == 3) node += k2 * fst[2];
            v[j].x = 0;
            v[j].y = 0;
            if ((g.valid >> kk) & 1u) v[j] = ldx<CG>(fres + node);
        }
        if (g.full) {
            // interior: the standard full weighting, weights known at compile time
#pragma unroll
            for (int j = 0; j < 9; j++) {
                const int kk = c0 + j;
                const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = kk / 9;
                if (k0 == 1 && k1 == 1 && (D == 2 || k2 == 1)) continue;
                const int e = (k0 == 1) + (k1 == 1) + (D == 3 ? (k2 == 1) : 0);
                const T w = (T)(1 << e) / (T)(D == 2 ? 16 : 64);
                as += w * v[j].x;
                ac += w * v[j].y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 9; j++) {
                const int kk = c0 + j;
                if (!((g.valid >> kk) & 1u)) continue;
                const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = kk / 9;
                const int e = g.e1[0][k0] + g.e1[1][k1] + (D == 3 ? g.e1[2][k2] : 1) - 3;
                const T w = pow2_weight<D, T>(e);
                as += w * v[j].x;
                ac += w * v[j].y;
            }
        }
    }
    const T wc = g.full ? (T)(1 << D) / (T)(D == 2 ? 16 : 64) : (T)g.iwc / (T)(D == 2 ? 16 : 64);
    T2 out;
    out.x = as + wc * vc.x;
    out.y = ac + wc * vc.y;
    crhs[g.I] = out;
    if (crhsc) crhsc[t] = out;
    T2 z;
    z.x = 0;
    z.y = 0;
    cx[g.I] = red ? relax_value_zero<D, T, PW>(out, *red) : z;  // the coarse-grid error starts from zero
}

template <int D, typename T, bool CG>
__device__ __forceinline__ void restrict_node(int t, const Lists& ls, const int8_t* ctype, int cn,
                                              const int8_t* ftype, int fn, const typename V2<T>::t* fres,
                                              typename V2<T>::t* crhs, typename V2<T>::t* cx,
                                              typename V2<T>::t* crhsc = nullptr) {
    RestrictGeo<D, T> g = fetch_restrict<D, T>(t, ls, ctype, cn, ftype, fn);
    restrict_apply<D, T, CG>(g, fn, fres, crhs, cx, nullptr, crhsc, t);
}

// The fixed part of the (bi/tri)linear interpolation to fine active node i
// (Sec. 3.5.3): the coarse corners that are active (bit cc) with their nodes.
// Every corner of a fine node carries the same weight 2^-k (k its odd
// coordinates), so the weights renormalised over the active corners are
// 1/n each (n of them): the interpolated value is the corners' sum times the
// correctly rounded 1/n -- the same number the weighted sum divided by the
// summed weights gives, without FP64 multiplies or a division.
template <int D, typename T>
struct ProlongGeo {
    long long i;
    long long node[1 << D];
    unsigned use;
};

template <int D>
__device__ __forceinline__ long long corner_node(const int* ii, int cc, const long long* cst, bool& dup) {
    long long node = 0;
    dup = false;
#pragma unroll
    for (int a = 0; a < D; a++) {
        int pick = (cc >> a) & 1;
        int lo = ii[a] >> 1, hi = (ii[a] + 1) >> 1;
        if (lo == hi) {
            if (pick) dup = true;
            node += lo * cst[a];
        } else {
            node += (pick ? hi : lo) * cst[a];
        }
    }
    return node;
}

template <int D, typename T>
__device__ __forceinline__ ProlongGeo<D, T> fetch_prolong(int t, const Lists& ls, const int8_t* ctype, int cn,
                                                          int fn) {
    ProlongGeo<D, T> g;
    int kind, gi;
    g.i = list_node(ls, t, kind, gi);
    const long long i = g.i;
    int ii[3];
    box_coords<D>(i, fn, ii);
    const long long cst[3] = {1, cn, (long long)cn * cn};
    g.use = 0;
    const int NC = 1 << D;
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        bool dup;
        g.node[cc] = corner_node<D>(ii, cc, cst, dup);
        if (dup) continue;
        int8_t tc = ctype[g.node[cc]];
        if (tc != T_IN && tc != T_GHOST) continue;
        g.use |= 1u << cc;
    }
    return g;
}

// 1/n correctly rounded in T, n = 1..8 (constants folded at compile time)
template <typename T>
__device__ __forceinline__ T inv_count(int n) {
    switch (n) {
        case 1: return (T)1;
        case 2: return (T)1 / (T)2;
        case 3: return (T)1 / (T)3;
        case 4: return (T)1 / (T)4;
        case 5: return (T)1 / (T)5;
        case 6: return (T)1 / (T)6;
        case 7: return (T)1 / (T)7;
        default: return (T)1 / (T)8;
    }
}

template <int D, typename T, bool CG>
__device__ __forceinline__ void prolong_apply(const ProlongGeo<D, T>& g, int fn, const typename V2<T>::t* cx,
                                              typename V2<T>::t* fx) {
    typedef typename V2<T>::t T2;
    if (!g.use) return;
    const int NC = 1 << D;
    T2 v[1 << D];
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        v[cc].x = 0;
        v[cc].y = 0;
        if ((g.use >> cc) & 1u) v[cc] = ldx<CG>(cx + g.node[cc]);
    }
    T2 xf = ldx<CG>(fx + g.i);
    T as = 0, ac = 0;
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        if (!((g.use >> cc) & 1u)) continue;
        as += v[cc].x;
        ac += v[cc].y;
    }
    const T r = inv_count<T>(__popc(g.use));
    xf.x = fmadd(as, r, xf.x);
    xf.y = fmadd(ac, r, xf.y);
    fx[g.i] = xf;
}

template <int D, typename T, bool CG>
__device__ __forceinline__ void prolong_node(int t, const Lists& ls, const int8_t* ctype, int cn,
                                             const typename V2<T>::t* cx, int fn, typename V2<T>::t* fx) {
    ProlongGeo<D, T> g = fetch_prolong<D, T>(t, ls, ctype, cn, fn);
    prolong_apply<D, T, CG>(g, fn, cx, fx);
}

}  // namespace stages
}  // namespace sulf
