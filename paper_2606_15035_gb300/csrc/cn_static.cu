// pic_cn_update_static: the Crank--Nicolson potential update with no device allocation.
//
// For callers that cannot allocate device memory at the point of use: code running under
// a fixed, pre-committed memory budget, host threads that must not enter the CUDA
// allocator (it can synchronise the device), or plugins whose host application owns all
// device allocations.  They pass device buffers for the inputs and outputs only; the
// working storage (right-hand sides, Chebyshev iterates and directions) lives in one
// file-scope __device__ array of fixed size, which every device that loads this library
// holds until the process exits.
#include <cmath>

#include "pic_internal.h"

namespace {

constexpr int64_t STATIC_MAX_CELLS = PIC_STATIC_MAX_CELLS;
constexpr int STATIC_MAX_STEPS = 1024;   // Chebyshev steps one call may run

// rhs | x (2 buffers) | d, 4 fields each.
static __device__ __align__(256) double g_cn_scratch[4 * 4 * STATIC_MAX_CELLS];

struct Dims {
    int n[3];
    int64_t N;
    double invH[3];
};

__device__ __forceinline__ int wrap_index(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

__device__ __forceinline__ int64_t at(const Dims& d, int ix, int iy, int iz) {
    return (int64_t)wrap_index(ix, d.n[0]) + (int64_t)d.n[0] * ((int64_t)wrap_index(iy, d.n[1]) +
                                                                 (int64_t)d.n[1] * wrap_index(iz, d.n[2]));
}

// Delta_h f = sum_a (f[+2] - 2 f + f[-2]) / (4 H_a^2) at node (ix, iy, iz).
__device__ __forceinline__ double lap_at(const double* __restrict__ f, const Dims& d, int ix, int iy, int iz) {
    const double c = f[at(d, ix, iy, iz)];
    return 0.25 * d.invH[0] * d.invH[0] * (f[at(d, ix + 2, iy, iz)] - 2.0 * c + f[at(d, ix - 2, iy, iz)]) +
           0.25 * d.invH[1] * d.invH[1] * (f[at(d, ix, iy + 2, iz)] - 2.0 * c + f[at(d, ix, iy - 2, iz)]) +
           0.25 * d.invH[2] * d.invH[2] * (f[at(d, ix, iy, iz + 2)] - 2.0 * c + f[at(d, ix, iy, iz - 2)]);
}

struct Fields4 {
    const double* f[4];
};

// rhs_f = (I + a Delta_h) F_f + dt W_f + c_f src_f and the warm start x_f = F_f.
__global__ void k_static_rhs(Dims d, Fields4 F, Fields4 W, Fields4 src, double a, double dt, double c_rho, double c_J,
                             double* __restrict__ rhs, double* __restrict__ x) {
    const int f = blockIdx.y;
    const double cf = f == 0 ? c_rho : c_J;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.N; g += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(g % d.n[0]);
        const int64_t t = g / d.n[0];
        const int iy = (int)(t % d.n[1]), iz = (int)(t / d.n[1]);
        const double u = F.f[f][g];
        rhs[f * d.N + g] = u + a * lap_at(F.f[f], d, ix, iy, iz) + dt * W.f[f][g] + cf * src.f[f][g];
        x[f * d.N + g] = u;
    }
}

// One Chebyshev step of (I - a Delta_h) x = rhs (the recurrence of the library's solver).
__global__ void k_static_cheb(Dims d, const double* __restrict__ x, double* __restrict__ xout, double* __restrict__ dir,
                              const double* __restrict__ rhs, double a, double alpha, double beta) {
    const int64_t off = blockIdx.y * d.N;
    const double* xf = x + off;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.N; g += (int64_t)gridDim.x * blockDim.x) {
        const int ix = (int)(g % d.n[0]);
        const int64_t t = g / d.n[0];
        const int iy = (int)(t % d.n[1]), iz = (int)(t / d.n[1]);
        const double r = rhs[off + g] - (xf[g] - a * lap_at(xf, d, ix, iy, iz));
        const double dn = (alpha == 0.0 ? 0.0 : alpha * dir[off + g]) + beta * r;
        dir[off + g] = dn;
        xout[off + g] = xf[g] + dn;
    }
}

// F1_f = x_f and W1_f = 2 (F1_f - F0_f) / dt - W0_f.
__global__ void k_static_backsub(Dims d, Fields4 F, Fields4 W, const double* __restrict__ x, double dt, double* phi1,
                                 double* psi1, double* A1, double* U1) {
    const int f = blockIdx.y;
    double* Fo = f == 0 ? phi1 : A1 + (int64_t)(f - 1) * d.N;
    double* Wo = f == 0 ? psi1 : U1 + (int64_t)(f - 1) * d.N;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.N; g += (int64_t)gridDim.x * blockDim.x) {
        const double u1 = x[f * d.N + g];
        Fo[g] = u1;
        Wo[g] = 2.0 * (u1 - F.f[f][g]) / dt - W.f[f][g];
    }
}

double sin2_max(int n) {
    double mx = 0.0;
    for (int m = 0; m < n; ++m) {
        const double s = std::sin(2.0 * M_PI * m / n);
        mx = std::fmax(mx, s * s);
    }
    return mx;
}

}  // namespace

extern "C" pic_status pic_cn_update_static(const int32_t n[3], const double L[3], double dt, double kappa,
                                           double sigma1, double sigma2, double helmholtz_tol, const double* phi,
                                           const double* psi, const double* A, const double* U,
                                           const double* rho_half, const double* J, double* phi1, double* psi1,
                                           double* A1, double* U1, void* stream) {
    if (!n || !L || !phi || !psi || !A || !U || !rho_half || !J || !phi1 || !psi1 || !A1 || !U1) return PIC_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (n[a] < 1 || !(L[a] > 0.0)) return PIC_ERR_ARG;
    const int64_t N = (int64_t)n[0] * n[1] * n[2];
    if (N > STATIC_MAX_CELLS) return PIC_ERR_ARG;     // beyond the fixed working storage
    if (!(dt > 0.0) || !(kappa > 0.0) || !(sigma1 > 0.0) || !(sigma2 > 0.0) || !(helmholtz_tol > 0.0))
        return PIC_ERR_ARG;
    Dims d;
    d.N = N;
    double lmax = 1.0;
    const double a = 0.25 * kappa * kappa * dt * dt;
    for (int ax = 0; ax < 3; ++ax) {
        d.n[ax] = n[ax];
        const double H = L[ax] / n[ax];
        d.invH[ax] = 1.0 / H;
        lmax += a * sin2_max(n[ax]) * d.invH[ax] * d.invH[ax];
    }
    // Chebyshev schedule on the spectrum [1, lmax] of I - a Delta_h, the library's own
    // (pic::cheb_schedule): the fewest steps whose error bound is below helmholtz_tol.
    if (pic::cheb_steps(1.0, lmax, helmholtz_tol) > STATIC_MAX_STEPS) return PIC_ERR_ARG;
    double alpha[STATIC_MAX_STEPS], beta[STATIC_MAX_STEPS];
    const int iters = pic::cheb_schedule(1.0, lmax, helmholtz_tol, alpha, beta, STATIC_MAX_STEPS);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    // The host-side name g_cn_scratch is a stand-in, not a device address.  Its address on the
    // current device is looked up on every call, so that it is never stale (a device reset or
    // a new primary context can move the module).
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_cn_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    double* scratch = static_cast<double*>(p);
    double* rhs = scratch;
    double* xa = scratch + 4 * STATIC_MAX_CELLS;
    double* xb = scratch + 8 * STATIC_MAX_CELLS;
    double* dir = scratch + 12 * STATIC_MAX_CELLS;

    cudaStream_t s = (cudaStream_t)stream;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t nb = (N + 255) / 256;
    if (nb > (int64_t)sms * 8) nb = (int64_t)sms * 8;
    const dim3 grid((unsigned)nb, 4);
    Fields4 F = {{phi, A, A + N, A + 2 * N}};
    Fields4 W = {{psi, U, U + N, U + 2 * N}};
    Fields4 src = {{rho_half, J, J + N, J + 2 * N}};
    const double c_rho = 0.5 * dt * dt * kappa * kappa * sigma1;
    const double c_J = 0.5 * dt * dt * kappa * kappa * sigma2;
    k_static_rhs<<<grid, 256, 0, s>>>(d, F, W, src, a, dt, c_rho, c_J, rhs, xa);
    double* x = xa;
    double* spare = xb;
    for (int k = 0; k < iters; ++k) {
        k_static_cheb<<<grid, 256, 0, s>>>(d, x, spare, dir, rhs, a, alpha[k], beta[k]);
        double* t = x;
        x = spare;
        spare = t;
    }
    k_static_backsub<<<grid, 256, 0, s>>>(d, F, W, x, dt, phi1, psi1, A1, U1);
    if (cudaGetLastError() != cudaSuccess) return PIC_ERR_CUDA;
    return PIC_OK;
}
