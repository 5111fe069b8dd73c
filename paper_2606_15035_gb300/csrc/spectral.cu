// Spectral mesh operators (the paper's choice, §3.3) for the PIC step (FP64, sm_103a).
//
// With ops = PIC_OPS_SPECTRAL the first derivative D_a has the Fourier symbol i k_a,
// k_a = 2 pi m_a / L_a, with the Nyquist symbol (2 |m_a| = n_a) set to zero so that D_a stays
// real and skew-adjoint; Delta_h = sum_a D_a D_a has the symbol -|k|^2 and the same 8 null
// modes as the central difference.  The Crank--Nicolson update (§3.2, Eq. (cn-field-update))
// is then diagonal: per mode, with b = dt kappa^2 lambda / 2 and lambda = -|k|^2,
//     [ 1     -dt/2 ] [u1]   [ u0 + dt/2 w0                  ]
//     [ -b      1   ] [w1] = [ w0 + b u0 + dt kappa^2 c src   ],
// solved exactly (no iteration), with src = rho^{n+1/2} (c = sigma1) for (phi, psi) and
// src = J_c^{n+1/2} (c = sigma2) for (A_c, U_c); continuity (Eq. (cn-continuity)) is
// rho^{n+1} = rho^n - dt D . J in the same basis.
//
// Transforms: a batched, mixed-radix (2 and 3) Stockham FFT of complex FP64 lines, one line
// per block in shared memory, applied along x, y and z; unnormalised forward transform and
// a 1/N scale on the way back to real space.  Mesh sizes n_a = 2^p 3^q <= 1024.
#include <cmath>
#include <vector>

#include "pic_internal.h"

namespace pic {
namespace {

struct FftAxis {
    int axis, n, nst;
    int64_t stride;              // element stride of a line along this axis
    int radix[FFT_MAX_STAGES];
    const double2* tw;           // exp(-2 pi i t / n), t = 0 .. n-1
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// First element of line l along the axis.
__device__ __forceinline__ int64_t line_base(int axis, int64_t l, const MeshDims& m) {
    if (axis == 0) return l * m.n[0];
    if (axis == 1) return (l % m.n[0]) + (int64_t)m.n[0] * m.n[1] * (l / m.n[0]);
    return l;
}

// In-place 1D transforms of every line of field blockIdx.y along one axis (fields N apart).
// Stockham autosort: stage s of radix R, with L = product of the previous radices, takes
// v_r = x[j + r n/R] (j < n/R, k = j mod L), twiddles v_r by exp(-+2 pi i k r / (L R)),
// applies the radix-R DFT and stores output s at (j div L) L R + k + s L.
// A block transforms `lb` lines whose first elements are adjacent in memory (lines l0 .. l0 +
// lb - 1 along y or z start at consecutive x, or consecutive x-y positions), so that the loads
// and stores of a strided axis read lb consecutive complex values at a time; along x (stride 1)
// lb is 1.  Shared memory holds the lb lines twice (ping-pong), line j at j n.
__global__ void k_fft_axis(double2* __restrict__ data, MeshDims m, FftAxis ax, int inverse, int lb) {
    extern __shared__ double2 sbuf[];
    const int n = ax.n;
    const int64_t nlines = m.ncell / n;
    const int64_t ngroups = nlines / lb;
    double2* field = data + (int64_t)blockIdx.y * m.ncell;
    const double sgn = inverse ? 1.0 : -1.0;
    const double s3 = sgn * 0.86602540378443864676;   // sin(2 pi / 3) with the transform's sign
    const int tot = lb * n;
    for (int64_t gr = blockIdx.x; gr < ngroups; gr += gridDim.x) {
        double2* x = sbuf;
        double2* y = sbuf + tot;
        double2* first = field + line_base(ax.axis, gr * lb, m);
        // element t of line j sits at first + j + t stride (lb > 1 only where lines are adjacent)
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int j = e % lb, t = e / lb;
            x[j * n + t] = lb > 1 ? first[j + (int64_t)t * ax.stride] : first[(int64_t)t * ax.stride];
        }
        __syncthreads();
        int L = 1;
        for (int st = 0; st < ax.nst; ++st) {
            const int R = ax.radix[st];
            const int nb = n / R, tstep = n / (L * R);
            for (int e = threadIdx.x; e < lb * nb; e += blockDim.x) {
                const int line = e / nb, j = e - line * nb;
                const double2* xl = x + line * n;
                double2* yl = y + line * n;
                const int k = j % L;
                const int out = (j / L) * L * R + k;
                double2 v0 = xl[j], v1 = xl[j + nb];
                double2 t1 = ax.tw[k * tstep];
                if (inverse) t1.y = -t1.y;
                v1 = cmul(v1, t1);
                if (R == 2) {
                    yl[out] = cadd(v0, v1);
                    yl[out + L] = csub(v0, v1);
                } else {
                    double2 v2 = xl[j + 2 * nb];
                    double2 t2 = ax.tw[2 * k * tstep];
                    if (inverse) t2.y = -t2.y;
                    v2 = cmul(v2, t2);
                    const double2 sum = cadd(v1, v2), dif = csub(v1, v2);
                    const double2 mid = make_double2(v0.x - 0.5 * sum.x, v0.y - 0.5 * sum.y);
                    yl[out] = cadd(v0, sum);
                    yl[out + L] = make_double2(mid.x - s3 * dif.y, mid.y + s3 * dif.x);        // + i s3 dif
                    yl[out + 2 * L] = make_double2(mid.x + s3 * dif.y, mid.y - s3 * dif.x);    // - i s3 dif
                }
            }
            __syncthreads();
            double2* t = x;
            x = y;
            y = t;
            L *= R;
        }
        for (int e = threadIdx.x; e < tot; e += blockDim.x) {
            const int j = e % lb, t = e / lb;
            if (lb > 1) first[j + (int64_t)t * ax.stride] = x[j * n + t];
            else first[(int64_t)t * ax.stride] = x[j * n + t];
        }
        __syncthreads();
    }
}

struct SpecParams {
    MeshDims m;
    double kscale[3];   // 2 pi / L_a
    double dt, kappa2, sigma1, sigma2, dV, invN;
};

// Wavenumber of index i on an axis of n nodes (fftfreq order), 0 at the Nyquist index.
__device__ __forceinline__ double kwave(int i, int n, double scale) {
    const int mm = i <= (n - 1) / 2 ? i : i - n;
    return 2 * (mm < 0 ? -mm : mm) == n ? 0.0 : mm * scale;
}

__device__ __forceinline__ void mode_k(const SpecParams& p, int64_t g, double k[3]) {
    const int ix = (int)(g % p.m.n[0]);
    const int64_t t = g / p.m.n[0];
    const int iy = (int)(t % p.m.n[1]), iz = (int)(t / p.m.n[1]);
    k[0] = kwave(ix, p.m.n[0], p.kscale[0]);
    k[1] = kwave(iy, p.m.n[1], p.kscale[1]);
    k[2] = kwave(iz, p.m.n[2], p.kscale[2]);
}

// i k z
__device__ __forceinline__ double2 ik(double k, double2 z) { return make_double2(-k * z.y, k * z.x); }

#define SPEC_LOOP(g, N) for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (N); g += (int64_t)gridDim.x * blockDim.x)

__global__ void k_r2c(const double* __restrict__ in, double2* __restrict__ out, int64_t n) {
    SPEC_LOOP(i, n) out[i] = make_double2(in[i], 0.0);
}

__global__ void k_c2r(const double2* __restrict__ in, double* __restrict__ out, int64_t n, double scale) {
    SPEC_LOOP(i, n) out[i] = in[i].x * scale;
}

// Continuity and the CN update per mode.  In: J^ (3), level n: [phi, A (3) | psi, U (3) | rho].
// Out: level n+1 [phi, A | psi, U | rho] and D phi^{n+1/2} (3).
__global__ void k_spec_cn(SpecParams p, const double2* __restrict__ Jh, const double2* __restrict__ S0,
                          double2* __restrict__ S1) {
    const int64_t N = p.m.ncell;
    const double hdt = 0.5 * p.dt;
    SPEC_LOOP(g, N) {
        double k[3];
        mode_k(p, g, k);
        const double lam = -(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
        const double b = hdt * p.kappa2 * lam, det = 1.0 - hdt * b;
        const double2 J[3] = {Jh[g], Jh[N + g], Jh[2 * N + g]};
        double2 divJ = cadd(cadd(ik(k[0], J[0]), ik(k[1], J[1])), ik(k[2], J[2]));
        const double2 r0 = S0[8 * N + g];
        const double2 r1 = make_double2(r0.x - p.dt * divJ.x, r0.y - p.dt * divJ.y);
        S1[8 * N + g] = r1;
        const double2 rh = make_double2(0.5 * (r0.x + r1.x), 0.5 * (r0.y + r1.y));
        double2 phi1 = make_double2(0.0, 0.0);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const double2 u0 = S0[f * N + g], w0 = S0[(4 + f) * N + g];
            const double2 src = f == 0 ? rh : J[f - 1];
            const double cs = p.dt * p.kappa2 * (f == 0 ? p.sigma1 : p.sigma2);
            const double2 q1 = make_double2(u0.x + hdt * w0.x, u0.y + hdt * w0.y);
            const double2 q2 = make_double2(w0.x + b * u0.x + cs * src.x, w0.y + b * u0.y + cs * src.y);
            const double2 u1 = make_double2((q1.x + hdt * q2.x) / det, (q1.y + hdt * q2.y) / det);
            const double2 w1 = make_double2((q2.x + b * q1.x) / det, (q2.y + b * q1.y) / det);
            S1[f * N + g] = u1;
            S1[(4 + f) * N + g] = w1;
            if (f == 0) phi1 = u1;
        }
        const double2 ph = make_double2(0.5 * (phi1.x + S0[g].x), 0.5 * (phi1.y + S0[g].y));
#pragma unroll
        for (int a = 0; a < 3; ++a) S1[(9 + a) * N + g] = ik(k[a], ph);
    }
}

// The CN Helmholtz solve of the central-difference operators by FFT: (I - a Delta_h) x = b, the
// wide Laplacian sum_a (f_{+2} - 2 f + f_{-2}) / (4 H_a^2) having the symbol -sum_a s2_a[m_a],
// s2_a[m] = sin^2(2 pi m / n_a) / H_a^2, so each mode is divided by 1 + a sum_a s2_a[m_a] (>= 1;
// the 1/N of the inverse transform is folded in).
__global__ void k_helm_fft_divide(MeshDims m, const double* __restrict__ s2, double a, double invN,
                                  double2* __restrict__ data, int nf) {
    const int64_t N = m.ncell;
    SPEC_LOOP(g, N) {
        const int ix = (int)(g % m.n[0]);
        const int64_t t = g / m.n[0];
        const int iy = (int)(t % m.n[1]), iz = (int)(t / m.n[1]);
        const double d = invN / (1.0 + a * (s2[ix] + s2[m.n[0] + iy] + s2[m.n[0] + m.n[1] + iz]));
        for (int f = 0; f < nf; ++f) {
            const double2 z = data[f * N + g];
            data[f * N + g] = make_double2(z.x * d, z.y * d);
        }
    }
}

// Gather table per node: A^n (3), A^{n+1} (3), D phi^{n+1/2} (3), U^{n+1/2} (3).
__global__ void k_spec_table(int64_t N, const double* __restrict__ F0, const double* __restrict__ W0,
                             const double* __restrict__ F1, const double* __restrict__ W1,
                             const double* __restrict__ gphi, double* __restrict__ table) {
    SPEC_LOOP(g, N) {
        double* t = table + 12 * g;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            t[c] = F0[(1 + c) * N + g];
            t[3 + c] = F1[(1 + c) * N + g];
            t[6 + c] = gphi[c * N + g];
            t[9 + c] = 0.5 * (W1[(1 + c) * N + g] + W0[(1 + c) * N + g]);
        }
    }
}

// e_J partial sums of the iteration (real space).
__global__ void k_spec_ej(int64_t N, const double* __restrict__ J, const double* __restrict__ Jprev,
                          double* __restrict__ partials) {
    __shared__ double sm[32];
    double num = 0.0, den = 0.0;
    SPEC_LOOP(g, 3 * N) {
        const double j = J[g];
        den += j * j;
        if (Jprev) {
            const double d = j - Jprev[g];
            num += d * d;
        }
    }
    double r = block_sum(num, sm);
    if (threadIdx.x == 0) partials[S_EJ_NUM * MAX_BLOCKS + blockIdx.x] = r;
    r = block_sum(den, sm);
    if (threadIdx.x == 0) partials[S_EJ_DEN * MAX_BLOCKS + blockIdx.x] = r;
}

// Field energy W = dV sum_g (|E|^2 / 2 sigma1 + |B|^2 / 2 sigma2) by Parseval from the
// unnormalised transforms [phi, A | psi, U]: E^ = -i k phi^ - U^, B^ = i k x A^.
__global__ void k_spec_energy(SpecParams p, const double2* __restrict__ S, double* __restrict__ partials, int slot) {
    __shared__ double sm[32];
    const int64_t N = p.m.ncell;
    double e = 0.0;
    SPEC_LOOP(g, N) {
        double k[3];
        mode_k(p, g, k);
        const double2 phi = S[g];
        const double2 A[3] = {S[N + g], S[2 * N + g], S[3 * N + g]};
        double e2 = 0.0, b2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double2 U = S[(5 + a) * N + g];
            const double2 E = make_double2(k[a] * phi.y - U.x, -k[a] * phi.x - U.y);   // -i k phi - U
            e2 += E.x * E.x + E.y * E.y;
        }
        const double2 Bx = csub(ik(k[1], A[2]), ik(k[2], A[1]));
        const double2 By = csub(ik(k[2], A[0]), ik(k[0], A[2]));
        const double2 Bz = csub(ik(k[0], A[1]), ik(k[1], A[0]));
        b2 = Bx.x * Bx.x + Bx.y * Bx.y + By.x * By.x + By.y * By.y + Bz.x * Bz.x + Bz.y * Bz.y;
        e += (e2 / (2.0 * p.sigma1) + b2 / (2.0 * p.sigma2)) * p.dV * p.invN;
    }
    const double r = block_sum(e, sm);
    if (threadIdx.x == 0) partials[slot * MAX_BLOCKS + blockIdx.x] = r;
}

// Residual transforms of the committed level n+1 (§5.1): gauge G = psi / kappa^2 + D . A,
// Gauss R = D . E - sigma1 rho, continuity C = rho^{n+1} - rho^n + dt D . J.
__global__ void k_spec_resid(SpecParams p, const double2* __restrict__ S1, const double2* __restrict__ S0,
                             const double2* __restrict__ Jh, double2* __restrict__ out) {
    const int64_t N = p.m.ncell;
    SPEC_LOOP(g, N) {
        double k[3];
        mode_k(p, g, k);
        const double2 phi = S1[g], psi = S1[4 * N + g], rho1 = S1[8 * N + g], rho0 = S0[8 * N + g];
        double2 divA = make_double2(0.0, 0.0), divE = make_double2(0.0, 0.0), divJ = make_double2(0.0, 0.0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            divA = cadd(divA, ik(k[a], S1[(1 + a) * N + g]));
            const double2 U = S1[(5 + a) * N + g];
            const double2 E = make_double2(k[a] * phi.y - U.x, -k[a] * phi.x - U.y);
            divE = cadd(divE, ik(k[a], E));
            divJ = cadd(divJ, ik(k[a], Jh[a * N + g]));
        }
        out[g] = make_double2(psi.x / p.kappa2 + divA.x, psi.y / p.kappa2 + divA.y);
        out[N + g] = make_double2(divE.x - p.sigma1 * rho1.x, divE.y - p.sigma1 * rho1.y);
        out[2 * N + g] = make_double2(rho1.x - rho0.x + p.dt * divJ.x, rho1.y - rho0.y + p.dt * divJ.y);
    }
}

// Real-space reductions of the final sweep: mesh work sum_g J . E^{n+1/2} dV with
// E^{n+1/2} = -D phi^{n+1/2} - U^{n+1/2}, and max / sum of squares of the residuals.
__global__ void k_spec_diag(SpecParams p, const double* __restrict__ J, const double* __restrict__ gphi,
                            const double* __restrict__ W0, const double* __restrict__ W1,
                            const double2* __restrict__ resid, double* __restrict__ partials) {
    __shared__ double sm[32];
    const int64_t N = p.m.ncell;
    double mwork = 0.0, gmax = 0.0, gsq = 0.0, rmax = 0.0, rsq = 0.0, cmax = 0.0;
    SPEC_LOOP(g, N) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double Eh = -gphi[a * N + g] - 0.5 * (W1[(1 + a) * N + g] + W0[(1 + a) * N + g]);
            mwork += J[a * N + g] * Eh * p.dV;
        }
        const double G = resid[g].x * p.invN, R = resid[N + g].x * p.invN, Cc = resid[2 * N + g].x * p.invN;
        gmax = fmax(gmax, fabs(G));
        gsq += G * G;
        rmax = fmax(rmax, fabs(R));
        rsq += R * R;
        cmax = fmax(cmax, fabs(Cc));
    }
    const double v[6] = {mwork, gmax, gsq, rmax, rsq, cmax};
    const int slots[6] = {S_MWORK, S_G_MAX, S_G_SQ, S_R_MAX, S_R_SQ, S_CONT_MAX};
    const bool mx[6] = {false, true, false, true, false, true};
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const double r = mx[t] ? block_max(v[t], sm) : block_sum(v[t], sm);
        if (threadIdx.x == 0) partials[slots[t] * MAX_BLOCKS + blockIdx.x] = r;
    }
}

// phi^ = sigma1 rho^ / |k|^2 away from the null modes (-Delta_h phi = sigma1 rho), 0 on them.
__global__ void k_spec_poisson(SpecParams p, double2* __restrict__ rh) {
    SPEC_LOOP(g, p.m.ncell) {
        double k[3];
        mode_k(p, g, k);
        const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        const double s = k2 > 0.0 ? p.sigma1 / k2 : 0.0;
        rh[g] = make_double2(rh[g].x * s, rh[g].y * s);
    }
}

SpecParams spec_params(const Ctx& c) {
    SpecParams p;
    p.m = c.m;
    for (int a = 0; a < 3; ++a) p.kscale[a] = 2.0 * M_PI / c.cfg.L[a];
    p.dt = c.cfg.dt;
    p.kappa2 = c.cfg.kappa * c.cfg.kappa;
    p.sigma1 = c.cfg.sigma1;
    p.sigma2 = c.cfg.sigma2;
    p.dV = c.dV;
    p.invN = 1.0 / (double)c.m.ncell;
    return p;
}

int spec_blocks(const Ctx& c, int64_t n) {
    int64_t b = (n + THREADS - 1) / THREADS;
    if (b > (int64_t)c.sms * 8) b = (int64_t)c.sms * 8;
    return (int)std::max<int64_t>(b, 1);
}

FftAxis make_axis(const Ctx& c, int a) {
    FftAxis ax;
    ax.axis = a;
    ax.n = c.m.n[a];
    ax.stride = a == 0 ? 1 : (a == 1 ? c.m.n[0] : (int64_t)c.m.n[0] * c.m.n[1]);
    ax.nst = c.fft_nst[a];
    for (int s = 0; s < FFT_MAX_STAGES; ++s) ax.radix[s] = s < ax.nst ? c.fft_radix[a][s] : 1;
    ax.tw = c.fft_tw[a];
    return ax;
}

// 3D transform of nf contiguous complex fields in place.
void fft3(Ctx& c, double2* data, int nf, bool inverse) {
    for (int a = 0; a < 3; ++a) {
        const FftAxis ax = make_axis(c, a);
        if (ax.n == 1) continue;
        const int64_t nlines = c.m.ncell / ax.n;
        // lines per block: 1 along x (contiguous); along y and z as many adjacent lines as keep
        // the two shared copies within 32 KB and divide the run of adjacent line starts (the
        // x extent for y, the x-y plane for z)
        int lb = 1;
        if (a > 0) {
            const int64_t run = a == 1 ? c.m.n[0] : (int64_t)c.m.n[0] * c.m.n[1];
            while (lb < 16 && 2 * (2 * lb) * ax.n <= 2048 && run % (2 * lb) == 0) lb *= 2;
        }
        int threads = std::min(256, std::max(32, ((lb * ax.n / 2 + 31) / 32) * 32));
        const int64_t gx = std::min<int64_t>(nlines / lb, (int64_t)c.sms * 16);
        dim3 grid((unsigned)gx, (unsigned)nf);
        k_fft_axis<<<grid, threads, 2 * lb * ax.n * sizeof(double2), c.stream>>>(data, c.m, ax, inverse ? 1 : 0, lb);
        ++c.launches;
    }
}

void r2c(Ctx& c, const double* in, double2* out, int64_t n) {
    k_r2c<<<spec_blocks(c, n), THREADS, 0, c.stream>>>(in, out, n);
    ++c.launches;
}

void c2r(Ctx& c, const double2* in, double* out, int64_t n, double scale) {
    k_c2r<<<spec_blocks(c, n), THREADS, 0, c.stream>>>(in, out, n, scale);
    ++c.launches;
}

}  // namespace

// Mesh sizes of the form 2^p 3^q up to FFT_MAX: the radices, 3s first.
bool fft_factor(int n, int* radix, int& nst) {
    nst = 0;
    if (n < 1 || n > FFT_MAX) return false;
    int r = n;
    while (r % 3 == 0) {
        radix[nst++] = 3;
        r /= 3;
    }
    while (r % 2 == 0) {
        radix[nst++] = 2;
        r /= 2;
    }
    return r == 1 && nst <= FFT_MAX_STAGES;
}

// Twiddles exp(-2 pi i t / n) of each axis, computed on the host in double precision.
void spec_twiddles(int n, std::vector<double2>& tw) {
    tw.resize((size_t)n);
    for (int t = 0; t < n; ++t) tw[t] = make_double2(std::cos(2.0 * M_PI * t / n), -std::sin(2.0 * M_PI * t / n));
}

// Start of a step: transforms of the level-n state [phi, A | psi, U | rho] into spec0.
void launch_spec_begin(Ctx& c) {
    const int64_t N = c.m.ncell;
    r2c(c, c.F0, c.spec0, 4 * N);
    r2c(c, c.W0, c.spec0 + 4 * N, 4 * N);
    r2c(c, c.rho0, c.spec0 + 8 * N, N);
    fft3(c, c.spec0, 9, false);
}

// The mesh half of an iteration with spectral operators: e_J partials, continuity and the
// exact CN update per mode, level n+1 and D phi^{n+1/2} back in real space, gather table.
void launch_spec_mesh_phase(Ctx& c, const double* Jcur, const double* Jprev) {
    const int64_t N = c.m.ncell;
    const SpecParams p = spec_params(c);
    k_spec_ej<<<mesh_blocks(c), THREADS, 0, c.stream>>>(N, Jcur, Jprev, c.partials);
    ++c.launches;
    r2c(c, Jcur, c.specJ, 3 * N);
    fft3(c, c.specJ, 3, false);
    k_spec_cn<<<spec_blocks(c, N), THREADS, 0, c.stream>>>(p, c.specJ, c.spec0, c.spec1);
    ++c.launches;
    fft3(c, c.spec1, 12, true);
    c2r(c, c.spec1, c.F1, 4 * N, p.invN);
    c2r(c, c.spec1 + 4 * N, c.W1, 4 * N, p.invN);
    c2r(c, c.spec1 + 8 * N, c.rho1, N, p.invN);
    c2r(c, c.spec1 + 9 * N, c.spec_gphi, 3 * N, p.invN);
    k_spec_table<<<mesh_blocks(c), THREADS, 0, c.stream>>>(N, c.F0, c.W0, c.F1, c.W1, c.spec_gphi, c.table);
    ++c.launches;
}

// Field energy of the state (F, W) into partial slot `slot` (spec1 is used as scratch).
void launch_spec_energy(Ctx& c, const double* F, const double* W, int slot) {
    const int64_t N = c.m.ncell;
    r2c(c, F, c.spec1, 4 * N);
    r2c(c, W, c.spec1 + 4 * N, 4 * N);
    fft3(c, c.spec1, 8, false);
    k_spec_energy<<<mesh_blocks(c), THREADS, 0, c.stream>>>(spec_params(c), c.spec1, c.partials, slot);
    ++c.launches;
}

// Diagnostics of the final sweep (after launch_spec_mesh_phase with the final current).
void launch_spec_diag(Ctx& c, const double* Jfinal) {
    const int64_t N = c.m.ncell;
    const SpecParams p = spec_params(c);
    // level n+1 in spectral form again (the mesh phase transformed spec1 back), its energy
    r2c(c, c.F1, c.spec1, 4 * N);
    r2c(c, c.W1, c.spec1 + 4 * N, 4 * N);
    r2c(c, c.rho1, c.spec1 + 8 * N, N);
    fft3(c, c.spec1, 9, false);
    k_spec_energy<<<mesh_blocks(c), THREADS, 0, c.stream>>>(p, c.spec1, c.partials, S_W);
    ++c.launches;
    k_spec_resid<<<spec_blocks(c, N), THREADS, 0, c.stream>>>(p, c.spec1, c.spec0, c.specJ, c.specR);
    ++c.launches;
    fft3(c, c.specR, 3, true);
    k_spec_diag<<<mesh_blocks(c), THREADS, 0, c.stream>>>(p, Jfinal, c.spec_gphi, c.W0, c.W1, c.specR, c.partials);
    ++c.launches;
}

// (I - a Delta_h) x = b for nf fields with the central-difference Laplacian, exactly per mode
// (c.helm_spec: nf N complex scratch; c.helm_s2: the per-axis symbols).
void launch_helmholtz_fft(Ctx& c, const double* b, double* x, int nf, double a) {
    const int64_t N = c.m.ncell;
    r2c(c, b, c.helm_spec, nf * N);
    fft3(c, c.helm_spec, nf, false);
    k_helm_fft_divide<<<spec_blocks(c, N), THREADS, 0, c.stream>>>(c.m, c.helm_s2, a, 1.0 / (double)N, c.helm_spec,
                                                                   nf);
    ++c.launches;
    fft3(c, c.helm_spec, nf, true);
    c2r(c, c.helm_spec, x, nf * N, 1.0);
}

// Initial potential: -Delta_h phi = sigma1 rho, zero on the null modes (§5.4).
void launch_spec_poisson(Ctx& c) {
    const int64_t N = c.m.ncell;
    r2c(c, c.rho0, c.specR, N);
    fft3(c, c.specR, 1, false);
    k_spec_poisson<<<spec_blocks(c, N), THREADS, 0, c.stream>>>(spec_params(c), c.specR);
    ++c.launches;
    fft3(c, c.specR, 1, true);
    c2r(c, c.specR, c.F0, N, 1.0 / (double)N);
}

}  // namespace pic
