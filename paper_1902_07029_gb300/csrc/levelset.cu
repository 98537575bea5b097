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
