// Lock-step batching: the data of one instance's level as the batched
// multigrid kernels read it, and their launchers (lockstep.cu).
#pragma once

#include "mg_stages.cuh"

namespace sulf {

// everything a batched phase reads of instance i's level (device copy, one
// entry per instance, built once per batch and level)
template <int D, typename T>
struct BLev {
    typedef typename V2<T>::t T2;
    stages::Lists ls;            // inside colour 0, colour 1, ghosts
    stages::GhostTab<T> tb;      // boundary rows (residual)
    stages::CoefPtr<D, T> cf;    // stencil coefficients
    Coef<T> c;                   // the level's constants (matrix-free FP32 relaxation)
    const typename V2<T>::t* Wc; // the (s, c) the coefficients are formed from
    T2* rhs;
    T2* rhsc;  // rhs per list position (FP64 levels; null for FP32)
    T2* x;
    T2* res;
    const int8_t* type;
    int n;
    long long st1, st2;
    // composed ghost relaxation and the copy of the ghosts' s it starts from
    const int* gop_ptr;
    const int* gop_code;
    const T* gop_val;
    const T2* gc;
    const T* gci;
    T* snap;
    // band extension
    int nb;
    const int* eptr;
    const int* eidx;
    const int* bidx;
    const T* eval;
    // coarsest level
    int nact;
    const int* act;
    const T* Ainv;
};

enum class BPhase { relax, relax_mf, ghost_op, residual, extend, restrict_to, prolong_from, coarsest, zero32,
                    accumulate, to_float, residual_to32 };

// one launch of phase ph over the instances' work lists: CTA b serves the
// instance i with pre[i] <= b < pre[i+1]; masked instances (active[i] == 0)
// are skipped.  lc: the coarse level of a restriction / prolongation (lv is
// the fine one); colour: of a relaxation; norms: per-instance max-norm slots
// of a residual (or NULL); smem: dynamic shared memory of the coarsest solve.
// relax_mf (FP32 only): the relaxation with the coefficients formed from Wc.
template <int D, typename T>
int launch_batched(BPhase ph, const BLev<D, T>* lv, const BLev<D, T>* lc, const int* pre, int nblocks, int K,
                   const int* active, int colour, unsigned long long* norms, size_t smem, cudaStream_t s);
// the mixed form's per-cycle steps on the finest level (zero the FP32 error,
// accumulate it into the FP64 update, next FP32 right-hand side from the FP64
// defect: to_float converts a stored one, residual_to32 computes it with the
// max-norms into norms)
template <int D>
int launch_batched_mixed(BPhase ph, const BLev<D, double>* l64, const BLev<D, float>* l32, const int* pre,
                         int nblocks, int K, const int* active, cudaStream_t s, unsigned long long* norms = nullptr);

}  // namespace sulf
