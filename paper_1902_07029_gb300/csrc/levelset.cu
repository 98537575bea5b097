// Level-set preprocessing (arXiv:1902.07029, Sec. 2): reinitialization of a
// generic level set toward the signed distance, and the provisional level set
// of a binary mask (a scanned shape).  Run once before sulf_create_domain;
// not part of the time step.
//
// Both march explicit steps over the whole box, one thread per node, ping-pong
// between two device arrays; the device memory is taken from the
// stream-ordered pool on a private stream and returned before the call ends.
#include <cmath>

#include "sulf_internal.cuh"

namespace sulf {
namespace {

constexpr int kLsThreads = 256;

inline unsigned blocks_for(long long n) { return (unsigned)((n + kLsThreads - 1) / kLsThreads); }

template <int D>
__device__ __forceinline__ void box_coords(long long i, int n, int* ii) {
    ii[0] = (int)(i % n);
    ii[1] = (int)((i / n) % n);
    ii[2] = D == 3 ? (int)(i / ((long long)n * n)) : 0;
}

// one explicit Euler step of d phi_d / d mu = sgn(phi0) (1 - |grad phi_d|):
// smoothed sign phi0 / sqrt(phi0^2 + h^2), Godunov's upwind |grad| from the
// one-sided differences (a missing box-edge side counts as zero)
template <int D>
__global__ void k_reinit_step(long long nn, int n, double h, double dmu, const double* __restrict__ phi0,
                              const double* __restrict__ a, double* __restrict__ b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int ii[3];
    box_coords<D>(i, n, ii);
    const long long st[3] = {1, n, (long long)n * n};
    const double p0 = phi0[i];
    const double ai = a[i];
    const double sg = p0 / sqrt(p0 * p0 + h * h);
    double g2 = 0.0;
#pragma unroll
    for (int ax = 0; ax < D; ax++) {
        const double dm = ii[ax] > 0 ? (ai - a[i - st[ax]]) / h : 0.0;
        const double dp = ii[ax] < n - 1 ? (a[i + st[ax]] - ai) / h : 0.0;
        double l, r;
        if (p0 > 0.0) {
            l = dm > 0.0 ? dm : 0.0;
            r = dp < 0.0 ? dp : 0.0;
        } else {
            l = dm < 0.0 ? dm : 0.0;
            r = dp > 0.0 ? dp : 0.0;
        }
        g2 += l * l > r * r ? l * l : r * r;
    }
    b[i] = p0 == 0.0 ? ai : ai - dmu * sg * (sqrt(g2) - 1.0);
}

__global__ void k_mask_init(long long nn, const uint8_t* __restrict__ mask, double* __restrict__ a) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn) a[i] = mask[i] ? -1.0 : 1.0;
}

// one explicit heat step phi += lambda sum_q (phi_q - phi) over the axis
// neighbours present in the box
template <int D>
__global__ void k_heat_step(long long nn, int n, double lam, const double* __restrict__ a, double* __restrict__ b) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int ii[3];
    box_coords<D>(i, n, ii);
    const long long st[3] = {1, n, (long long)n * n};
    const double ai = a[i];
    double acc = 0.0;
#pragma unroll
    for (int ax = 0; ax < D; ax++) {
        if (ii[ax] > 0) acc += a[i - st[ax]] - ai;
        if (ii[ax] < n - 1) acc += a[i + st[ax]] - ai;
    }
    b[i] = ai + lam * acc;
}

// device buffers of one call, returned to the pool at the end
struct Scratch {
    cudaStream_t s = nullptr;
    double* p[3] = {nullptr, nullptr, nullptr};
    uint8_t* m = nullptr;
    ~Scratch() {
        if (s) {
            for (double* q : p)
                if (q) cudaFreeAsync(q, s);
            if (m) cudaFreeAsync(m, s);
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    }
};

bool box_size(int dim, int N, long long* nn) {
    if ((dim != 2 && dim != 3) || N < 2 || N > (dim == 2 ? 65535 : 2047)) return false;
    long long n = N + 1;
    *nn = dim == 2 ? n * n : n * n * n;
    return true;
}

}  // namespace
}  // namespace sulf

using namespace sulf;

extern "C" int sulf_reinit_levelset(const double* phi_in, int dim, int N, double h, int steps, double* phi_out) {
    long long nn = 0;
    if (!phi_in || !phi_out || !box_size(dim, N, &nn) || !(h > 0) || steps < 0)
        return sulf_fail(SULF_EINVAL, "invalid arguments");
    Scratch sc;
    SULF_CUDA_TRY(cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking));
    for (double*& q : sc.p) SULF_CUDA_TRY(cudaMallocAsync((void**)&q, sizeof(double) * nn, sc.s));
    SULF_CUDA_TRY(cudaMemcpyAsync(sc.p[0], phi_in, sizeof(double) * nn, cudaMemcpyHostToDevice, sc.s));
    SULF_CUDA_TRY(cudaMemcpyAsync(sc.p[1], sc.p[0], sizeof(double) * nn, cudaMemcpyDeviceToDevice, sc.s));
    const double dmu = h / dim;
    double *a = sc.p[1], *b = sc.p[2];
    for (int k = 0; k < steps; k++) {
        if (dim == 2)
            k_reinit_step<2><<<blocks_for(nn), kLsThreads, 0, sc.s>>>(nn, N + 1, h, dmu, sc.p[0], a, b);
        else
            k_reinit_step<3><<<blocks_for(nn), kLsThreads, 0, sc.s>>>(nn, N + 1, h, dmu, sc.p[0], a, b);
        double* t = a;
        a = b;
        b = t;
    }
    SULF_CUDA_TRY(cudaGetLastError());
    SULF_CUDA_TRY(cudaMemcpyAsync(phi_out, a, sizeof(double) * nn, cudaMemcpyDeviceToHost, sc.s));
    SULF_CUDA_TRY(cudaStreamSynchronize(sc.s));
    return SULF_OK;
}

extern "C" int sulf_levelset_from_mask(const uint8_t* mask, int dim, int N, int steps, double* phi_out) {
    long long nn = 0;
    if (!mask || !phi_out || !box_size(dim, N, &nn) || steps < 0) return sulf_fail(SULF_EINVAL, "invalid arguments");
    Scratch sc;
    SULF_CUDA_TRY(cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking));
    for (int k = 0; k < 2; k++) SULF_CUDA_TRY(cudaMallocAsync((void**)&sc.p[k], sizeof(double) * nn, sc.s));
    SULF_CUDA_TRY(cudaMallocAsync((void**)&sc.m, (size_t)nn, sc.s));
    SULF_CUDA_TRY(cudaMemcpyAsync(sc.m, mask, (size_t)nn, cudaMemcpyHostToDevice, sc.s));
    k_mask_init<<<blocks_for(nn), kLsThreads, 0, sc.s>>>(nn, sc.m, sc.p[0]);
    const double lam = 1.0 / (4.0 * dim);
    double *a = sc.p[0], *b = sc.p[1];
    for (int k = 0; k < steps; k++) {
        if (dim == 2)
            k_heat_step<2><<<blocks_for(nn), kLsThreads, 0, sc.s>>>(nn, N + 1, lam, a, b);
        else
            k_heat_step<3><<<blocks_for(nn), kLsThreads, 0, sc.s>>>(nn, N + 1, lam, a, b);
        double* t = a;
        a = b;
        b = t;
    }
    SULF_CUDA_TRY(cudaGetLastError());
    SULF_CUDA_TRY(cudaMemcpyAsync(phi_out, a, sizeof(double) * nn, cudaMemcpyDeviceToHost, sc.s));
    SULF_CUDA_TRY(cudaStreamSynchronize(sc.s));
    return SULF_OK;
}

// ---------------------------------------------------------------------------
// Linear extrapolation of initial data from the inside nodes (the PDE approach
// the paper cites for the ICs on the ghosts, Sec. 3.3): u_n = n . grad u where
// the central stencil is inside, u_n extended by Jacobi steps of
// d q / d tau + n . grad q = 0, then u by Jacobi steps of
// d u / d tau + n . grad u = u_n; upwind differences toward the inside,
// d tau = h / 2, n the central-difference unit normal of phi.

namespace sulf {
namespace {

template <int D>
__device__ __forceinline__ void unit_normal(const double* phi, long long i, const int* ii, int n, double h,
                                            double* nv) {
    const long long st[3] = {1, n, (long long)n * n};
    double g[3] = {0, 0, 0}, gn = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        const bool lo = ii[a] > 0, hi = ii[a] < n - 1;
        if (lo && hi)
            g[a] = (phi[i + st[a]] - phi[i - st[a]]) / (2.0 * h);
        else if (hi)
            g[a] = (phi[i + st[a]] - phi[i]) / h;
        else
            g[a] = (phi[i] - phi[i - st[a]]) / h;
        gn += g[a] * g[a];
    }
    gn = sqrt(gn);
#pragma unroll
    for (int a = 0; a < D; a++) nv[a] = gn > 0.0 ? g[a] / gn : 0.0;
}

// u_n at inside nodes whose axis neighbours are all inside, else 0 (unknown)
template <int D>
__global__ void k_xn_init(long long nn, int n, double h, const double* __restrict__ phi,
                          const int8_t* __restrict__ type, const double* __restrict__ u, double* __restrict__ q) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int ii[3];
    box_coords<D>(i, n, ii);
    const long long st[3] = {1, n, (long long)n * n};
    bool ok = type[i] == T_IN;
#pragma unroll
    for (int a = 0; a < D; a++)
        if (ii[a] == 0 || ii[a] == n - 1 || type[i - st[a]] != T_IN || type[i + st[a]] != T_IN) ok = false;
    double un = 0.0;
    if (ok) {
        double nv[3];
        unit_normal<D>(phi, i, ii, n, h, nv);
#pragma unroll
        for (int a = 0; a < D; a++) un += nv[a] * (u[i + st[a]] - u[i - st[a]]) / (2.0 * h);
    }
    q[i] = un;
}

template <int D>
__device__ __forceinline__ bool un_known(const int8_t* type, long long i, const int* ii, int n) {
    const long long st[3] = {1, n, (long long)n * n};
    if (type[i] != T_IN) return false;
#pragma unroll
    for (int a = 0; a < D; a++)
        if (ii[a] == 0 || ii[a] == n - 1 || type[i - st[a]] != T_IN || type[i + st[a]] != T_IN) return false;
    return true;
}

// one Jacobi step: q (source = 0, known nodes fixed) or u (source q, inside
// nodes fixed)
template <int D, bool FOR_U>
__global__ void k_x_step(long long nn, int n, double h, const double* __restrict__ phi,
                         const int8_t* __restrict__ type, const double* __restrict__ src,
                         const double* __restrict__ v, double* __restrict__ w) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= nn) return;
    int ii[3];
    box_coords<D>(i, n, ii);
    const bool fixed = FOR_U ? type[i] == T_IN : un_known<D>(type, i, ii, n);
    if (fixed) {
        w[i] = v[i];
        return;
    }
    const long long st[3] = {1, n, (long long)n * n};
    double nv[3];
    unit_normal<D>(phi, i, ii, n, h, nv);
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < D; a++) {
        long long up = -1;
        if (nv[a] > 0.0 && ii[a] > 0) up = i - st[a];
        if (nv[a] < 0.0 && ii[a] < n - 1) up = i + st[a];
        if (up < 0) continue;
        acc += fabs(nv[a]) * (v[i] - v[up]);
    }
    const double dtau = 0.5 * h;
    w[i] = FOR_U ? v[i] - dtau * (acc / h - src[i]) : v[i] - (dtau / h) * acc;
}

__global__ void k_x_zero_outside(long long nn, const int8_t* __restrict__ type, double* __restrict__ u) {
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < nn && type[i] != T_IN) u[i] = 0.0;
}

}  // namespace

// u (device, box of the finest level) extended from the inside nodes; work
// arrays q, q2, u2 of nn doubles each
int launch_extrapolate(const LevelGeo& L, double* u, double* q, double* q2, double* u2, int iters, cudaStream_t s) {
    const long long nn = L.nn;
    const int n = L.n;
    const unsigned g = blocks_for(nn);
    int launches = 0;
    if (L.dim == 2)
        k_xn_init<2><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, u, q);
    else
        k_xn_init<3><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, u, q);
    launches++;
    double *a = q, *b = q2;
    for (int k = 0; k < iters; k++) {
        if (L.dim == 2)
            k_x_step<2, false><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, nullptr, a, b);
        else
            k_x_step<3, false><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, nullptr, a, b);
        double* t = a;
        a = b;
        b = t;
        launches++;
    }
    k_x_zero_outside<<<g, kLsThreads, 0, s>>>(nn, L.type, u);
    launches++;
    double *v = u, *w = u2;
    for (int k = 0; k < iters; k++) {
        if (L.dim == 2)
            k_x_step<2, true><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, a, v, w);
        else
            k_x_step<3, true><<<g, kLsThreads, 0, s>>>(nn, n, L.h, L.phi, L.type, a, v, w);
        double* t = v;
        v = w;
        w = t;
        launches++;
    }
    if (v != u) {
        cudaMemcpyAsync(u, v, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s);
    }
    return launches;
}

}  // namespace sulf
