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
    return c;
}

// off-diagonal part of the s row of an inside node applied to x (Eq. JssI and
// Eq. JscI as exact derivatives): sum over the axis neighbours q of
// J^ss_pq x^s_q + J^sc_pq x^c_q with J^ss_pq = -g and J^sc_pq = +-e
template <int D, typename T, bool CG>
__device__ __forceinline__ T offdiag_s(long long p, const CoefPtr<D, T>& cf, const typename V2<T>::t* x,
                                       const long long* st) {
    typedef typename V2<T>::t T2;
    T acc = 0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        T2 ge = cf.edge[a][p];
        T2 xe = ldx<CG>(x + p + st[a]);
        T2 gw = cf.edge[a][p - st[a]];
        T2 xw = ldx<CG>(x + p - st[a]);
        acc += (ge.y * xe.y - ge.x * xe.x) - (gw.x * xw.x + gw.y * xw.y);
    }
    return acc;
}

// collective (Eq. matrixP) or pointwise (Eq. matrixPclassical) update of the
// inside node p: x_p <- P^{-1} (b - (J - P) x), resp. the diagonal of P
template <int D, typename T, bool PW, bool CG>
__device__ __forceinline__ void relax_node(long long p, const CoefPtr<D, T>& cf, const typename V2<T>::t* rhs,
                                           typename V2<T>::t* x, const long long* st) {
    typedef typename V2<T>::t T2;
    T off = offdiag_s<D, T, CG>(p, cf, x, st);
    T2 b = ldx<CG>(rhs + p);
    T2 out;
    if (PW) {
        T2 xp = ldx<CG>(x + p);
        T2 pa = cf.Pa[p], pb = cf.Pb[p];
        out.x = (b.x - off - pa.y * xp.y) / pa.x;
        out.y = (b.y - pb.x * xp.x) / pb.y;
    } else {
        T2 ia = cf.Ia[p], ib = cf.Ib[p];
        T r = b.x - off;
        out.x = ia.x * r + ia.y * b.y;
        out.y = ib.x * r + ib.y * b.y;
    }
    x[p] = out;
}

// boundary row s~(B) of ghost gi applied to the s component: tensor-product
// weights on the upwind stencil (Eq. JssD).  Ghost members come from the
// previous relaxation pass (sin) unless from_x.
template <int D, typename T, bool CG>
__device__ __forceinline__ T ghost_dot(int gi, long long g, const int8_t* gm, const T* gw, const int* gpos,
                                       const typename V2<T>::t* x, const T* sin, bool from_x, long long st1,
                                       long long st2) {
    T wa[3][3];
    int m[3] = {1, 1, 1};
#pragma unroll
    for (int a = 0; a < D; a++) {
        m[a] = gm[(long long)gi * D + a];
#pragma unroll
        for (int k = 0; k < 3; k++) wa[a][k] = gw[(long long)gi * 3 * D + 3 * a + k];
    }
    const long long st[3] = {1, st1, st2};
    const int K = D == 2 ? 9 : 27;
    T acc = 0;
#pragma unroll
    for (int kk = 0; kk < K; kk++) {
        const int k0 = kk % 3, k1 = (kk / 3) % 3, k2 = kk / 9;
        T w = wa[0][k0] * wa[1][k1];
        if (D == 3) w = w * wa[2][k2];
        if (w == (T)0) continue;
        long long node = g - m[0] * k0 * st[0] - m[1] * k1 * st[1];
        if (D == 3) node -= m[2] * k2 * st[2];
        T v;
        if (from_x) {
            v = ldx<CG>(x + node).x;
        } else {
            int gp = gpos[node];
            v = gp >= 0 ? ldx<CG>(sin + gp) : ldx<CG>(x + node).x;
        }
        acc += w * v;
    }
    return acc;
}

// one Jacobi pass of the ghost relaxation (Eq. RelGhost) for ghost gi:
// s_g += tau (r_g - row . x) from the previous pass's values, then the ghost c
// row relaxed by its diagonal with the fresh s_g
template <int D, typename T, bool CG>
__device__ __forceinline__ void ghost_pass_node(int gi, const int* gidx, const int* gpos, const int8_t* gm,
                                                const T* gw, const typename V2<T>::t* gc,
                                                const typename V2<T>::t* rhs, typename V2<T>::t* x, const T* sin,
                                                T* sout, long long st1, long long st2, T tau, bool first,
                                                bool last) {
    typedef typename V2<T>::t T2;
    long long g = gidx[gi];
    T acc = ghost_dot<D, T, CG>(gi, g, gm, gw, gpos, x, sin, first, st1, st2);
    T2 xg = ldx<CG>(x + g);
    T s_old = first ? xg.x : ldx<CG>(sin + gi);
    T2 b = ldx<CG>(rhs + g);
    T s_new = s_old + tau * (b.x - acc);
    T2 q = gc[gi];  // (J^cs_gg, J^cc_gg)
    T c_new = xg.y + (b.y - (q.x * s_new + q.y * xg.y)) / q.y;
    T* xs = reinterpret_cast<T*>(x + g);
    xs[1] = c_new;
    if (last)
        xs[0] = s_new;
    else
        sout[gi] = s_new;
}

// defect r = rhs - J x at list position t; returns max(|r_s|, |r_c|) as bits
template <int D, typename T, bool CG>
__device__ __forceinline__ unsigned long long residual_node(int t, const Lists& ls, const int8_t* gm, const T* gw,
                                                            const CoefPtr<D, T>& cf, const typename V2<T>::t* rhs,
                                                            const typename V2<T>::t* x, typename V2<T>::t* res,
                                                            long long st1, long long st2) {
    typedef typename V2<T>::t T2;
    int kind, gi = 0;
    long long p = list_node(ls, t, kind, gi);
    T2 b = ldx<CG>(rhs + p);
    T2 xp = ldx<CG>(x + p);
    T2 r;
    if (kind == 1) {
        const long long st[3] = {1, st1, st2};
        T off = offdiag_s<D, T, CG>(p, cf, x, st);
        T2 pa = cf.Pa[p], pb = cf.Pb[p];
        r.x = b.x - (pa.x * xp.x + pa.y * xp.y + off);
        r.y = b.y - (pb.x * xp.x + pb.y * xp.y);
    } else {
        T acc = ghost_dot<D, T, CG>(gi, p, gm, gw, nullptr, x, nullptr, true, st1, st2);
        T2 q = cf.gc[gi];
        r.x = b.x - acc;
        r.y = b.y - (q.x * xp.x + q.y * xp.y);
    }
    res[p] = r;
    unsigned long long a0 = abs_bits(r.x), a1 = abs_bits(r.y);
    return a0 > a1 ? a0 : a1;
}

// one explicit upwind Euler step of dr/dtau + n.grad r = 0 at band node b
// (Sec. 3.5.2); band values start at 0
template <int D, typename T, bool CG>
__device__ __forceinline__ void extend_node(int b, const int* bidx, const int* bref, const T* ban,
                                            typename V2<T>::t* res, const typename V2<T>::t* bin,
                                            typename V2<T>::t* bout, T cfl, bool first, bool last) {
    typedef typename V2<T>::t T2;
    T2 v;
    if (first) {
        v.x = 0;
        v.y = 0;
    } else {
        v = ldx<CG>(bin + b);
    }
    T ax = 0, ay = 0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        int ref = bref[(long long)b * D + a];
        if (ref == -1) continue;
        T2 u;
        if (ref >= 0) {
            if (first) {
                u.x = 0;
                u.y = 0;
            } else {
                u = ldx<CG>(bin + ref);
            }
        } else {
            u = ldx<CG>(res + (-(long long)ref - 2));
        }
        T an = ban[(long long)b * D + a];
        ax += an * (v.x - u.x);
        ay += an * (v.y - u.y);
    }
    T2 nv;
    nv.x = v.x - cfl * ax;
    nv.y = v.y - cfl * ay;
    if (last)
        res[bidx[b]] = nv;
    else
        bout[b] = nv;
}

__device__ __forceinline__ bool valid_for(int8_t rule, int8_t t) {
    return rule == T_IN ? t == T_IN : (t == T_GHOST || t == T_BAND);
}

// boundary-aware full weighting at the coarse node of list position t (Eqs.
// Fstencil, Fstencilgen, Fig. Neigh); also zeroes the coarse error there
template <int D, typename T, bool CG>
__device__ __forceinline__ void restrict_node(int t, const Lists& ls, const int8_t* ctype, int cn,
                                              const int8_t* ftype, int fn, const typename V2<T>::t* fres,
                                              typename V2<T>::t* crhs, typename V2<T>::t* cx) {
    typedef typename V2<T>::t T2;
    int kind, gi;
    long long I = list_node(ls, t, kind, gi);
    int8_t rule = ctype[I];
    int ii[3] = {0, 0, 0};
    ii[0] = (int)(I % cn);
    ii[1] = (int)((I / cn) % cn);
    if (D == 3) ii[2] = (int)(I / ((long long)cn * cn));
    const long long fst[3] = {1, fn, (long long)fn * fn};
    long long f = 0;
#pragma unroll
    for (int a = 0; a < D; a++) f += 2LL * ii[a] * fst[a];
    T w1[3][3];
#pragma unroll
    for (int a = 0; a < D; a++) {
        bool vl = ii[a] > 0 && valid_for(rule, ftype[f - fst[a]]);
        bool vr = 2 * ii[a] < fn - 1 && valid_for(rule, ftype[f + fst[a]]);
        T l = 1, m = 2, r = 1;
        if (vl && !vr) {
            l = 2; m = 2; r = 0;
        } else if (!vl && vr) {
            l = 0; m = 2; r = 2;
        } else if (!vl && !vr) {
            l = 0; m = 4; r = 0;
        }
        w1[a][0] = l / (T)4;
        w1[a][1] = m / (T)4;
        w1[a][2] = r / (T)4;
    }
    const int K = D == 2 ? 9 : 27;
    T as = 0, ac = 0, wc = 0;
#pragma unroll
    for (int kk = 0; kk < K; kk++) {
        const int k0 = kk % 3 - 1, k1 = (kk / 3) % 3 - 1, k2 = kk / 9 - 1;
        T w = w1[0][k0 + 1] * w1[1][k1 + 1];
        if (D == 3) w = w * w1[2][k2 + 1];
        if (w == (T)0) continue;
        bool centre = k0 == 0 && k1 == 0 && (D == 2 || k2 == 0);
        if (centre) {
            wc += w;
            continue;
        }
        long long node = f + k0 * fst[0] + k1 * fst[1];
        if (D == 3) node += k2 * fst[2];
        if (!valid_for(rule, ftype[node])) {
            wc += w;
            continue;
        }
        T2 v = ldx<CG>(fres + node);
        as += w * v.x;
        ac += w * v.y;
    }
    T2 vc = ldx<CG>(fres + f);
    T2 out;
    out.x = as + wc * vc.x;
    out.y = ac + wc * vc.y;
    crhs[I] = out;
    T2 z;
    z.x = 0;
    z.y = 0;
    cx[I] = z;  // the coarse-grid error starts from zero
}

// (bi/tri)linear interpolation of the coarse error to the fine active node of
// list position t, renormalised over the coarse active nodes (Sec. 3.5.3)
template <int D, typename T, bool CG>
__device__ __forceinline__ void prolong_node(int t, const Lists& ls, const int8_t* ctype, int cn,
                                             const typename V2<T>::t* cx, int fn, typename V2<T>::t* fx) {
    typedef typename V2<T>::t T2;
    int kind, gi;
    long long i = list_node(ls, t, kind, gi);
    int ii[3] = {0, 0, 0};
    ii[0] = (int)(i % fn);
    ii[1] = (int)((i / fn) % fn);
    if (D == 3) ii[2] = (int)(i / ((long long)fn * fn));
    const long long cst[3] = {1, cn, (long long)cn * cn};
    T ws = 0, as = 0, ac = 0;
    const int NC = 1 << D;
#pragma unroll
    for (int cc = 0; cc < NC; cc++) {
        long long node = 0;
        T w = 1;
        bool dup = false;
#pragma unroll
        for (int a = 0; a < D; a++) {
            int pick = (cc >> a) & 1;
            int lo = ii[a] >> 1, hi = (ii[a] + 1) >> 1;
            if (lo == hi) {
                if (pick) dup = true;
                node += lo * cst[a];
            } else {
                w *= (T)0.5;
                node += (pick ? hi : lo) * cst[a];
            }
        }
        if (dup) continue;
        int8_t tc = ctype[node];
        if (tc != T_IN && tc != T_GHOST) continue;
        T2 v = ldx<CG>(cx + node);
        ws += w;
        as += w * v.x;
        ac += w * v.y;
    }
    if (ws > (T)0) {
        T2 xf = ldx<CG>(fx + i);
        xf.x += as / ws;
        xf.y += ac / ws;
        fx[i] = xf;
    }
}

}  // namespace stages
}  // namespace sulf
