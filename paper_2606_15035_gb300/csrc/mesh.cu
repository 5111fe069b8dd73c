// Mesh kernels of the PIC step (FP64, sm_103a): continuity, the Crank--Nicolson potential
// update solved as a Helmholtz problem by Chebyshev iteration, back-substitution, the
// particle gather table, energies and the §5.1 diagnostics.
//
// Operators (periodic, node-collocated): D_a f = (f[+1] - f[-1]) / (2 H_a) and
// Delta_h f = sum_a D_a D_a f = sum_a (f[+2] - 2 f + f[-2]) / (4 H_a^2).
//
// CN update (§3.2, Eq. (cn-field-update)).  Eliminating psi^{n+1} = 2 (phi^{n+1} - phi^n)/dt - psi^n
// gives, with a = kappa^2 dt^2 / 4,
//     (I - a Delta_h) phi^{n+1} = (I + a Delta_h) phi^n + dt psi^n + (dt^2 kappa^2 sigma1 / 2) rho^{n+1/2},
// and the same for each component of A with (U, sigma2, J^{n+1/2}).
#include <cooperative_groups.h>

#include "pic_internal.h"

namespace pic {
namespace {

struct Nb {
    int64_t g;
    int ix, iy, iz;
};

__device__ __forceinline__ Nb decompose(int64_t g, const MeshDims& m) {
    Nb r;
    r.g = g;
    r.ix = (int)(g % m.n[0]);
    int64_t t = g / m.n[0];
    r.iy = (int)(t % m.n[1]);
    r.iz = (int)(t / m.n[1]);
    return r;
}

// index of the node shifted by (dx, dy, dz), periodic
__device__ __forceinline__ int64_t shift(const Nb& b, int dx, int dy, int dz, const MeshDims& m) {
    return node_index(wrapi(b.ix + dx, m.n[0]), wrapi(b.iy + dy, m.n[1]), wrapi(b.iz + dz, m.n[2]), m);
}

__device__ __forceinline__ double dcen(const double* __restrict__ f, const Nb& b, int a, const MeshDims& m,
                                       const double* invH) {
    int64_t p = a == 0 ? shift(b, 1, 0, 0, m) : (a == 1 ? shift(b, 0, 1, 0, m) : shift(b, 0, 0, 1, m));
    int64_t q = a == 0 ? shift(b, -1, 0, 0, m) : (a == 1 ? shift(b, 0, -1, 0, m) : shift(b, 0, 0, -1, m));
    return 0.5 * invH[a] * (f[p] - f[q]);
}

// Delta_h f at node b (wide Laplacian = sum_a D_a D_a)
__device__ __forceinline__ double lap(const double* __restrict__ f, const Nb& b, const MeshDims& m, const double* invH) {
    const double c = f[b.g];
    double s = 0.25 * invH[0] * invH[0] * (f[shift(b, 2, 0, 0, m)] - 2.0 * c + f[shift(b, -2, 0, 0, m)]);
    s += 0.25 * invH[1] * invH[1] * (f[shift(b, 0, 2, 0, m)] - 2.0 * c + f[shift(b, 0, -2, 0, m)]);
    s += 0.25 * invH[2] * invH[2] * (f[shift(b, 0, 0, 2, m)] - 2.0 * c + f[shift(b, 0, 0, -2, m)]);
    return s;
}

// Position of a linear index over nfields stacked meshes in mixed radix (ix, iy, iz, field),
// advanced by a fixed grid stride with carries instead of divisions: the stencil kernels below
// would otherwise spend most of their instructions on 64-bit divisions and index wraps.
struct MeshPos {
    int ix, iy, iz, f;
    int64_t g;   // node index within its field
};

struct StrideDigits {
    int sx, sy, sz, sf;   // S = sx + n0 (sy + n1 (sz + n2 sf)), each digit below its radix
};

StrideDigits stride_digits(int64_t S, const MeshDims& m) {
    StrideDigits d;
    d.sx = (int)(S % m.n[0]);
    S /= m.n[0];
    d.sy = (int)(S % m.n[1]);
    S /= m.n[1];
    d.sz = (int)(S % m.n[2]);
    d.sf = (int)(S / m.n[2]);
    return d;
}

__device__ __forceinline__ MeshPos pos_of(int64_t idx, const MeshDims& m) {
    MeshPos q;
    q.ix = (int)(idx % m.n[0]);
    int64_t t = idx / m.n[0];
    q.iy = (int)(t % m.n[1]);
    t /= m.n[1];
    q.iz = (int)(t % m.n[2]);
    q.f = (int)(t / m.n[2]);
    q.g = (int64_t)q.ix + (int64_t)m.n[0] * ((int64_t)q.iy + (int64_t)m.n[1] * q.iz);
    return q;
}

__device__ __forceinline__ void advance(MeshPos& q, const StrideDigits& s, const MeshDims& m) {
    int c = 0;
    int ix = q.ix + s.sx;
    if (ix >= m.n[0]) ix -= m.n[0], c = 1;
    int iy = q.iy + s.sy + c;
    c = 0;
    if (iy >= m.n[1]) iy -= m.n[1], c = 1;
    int iz = q.iz + s.sz + c;
    c = 0;
    if (iz >= m.n[2]) iz -= m.n[2], c = 1;
    q.f += s.sf + c;
    q.ix = ix;
    q.iy = iy;
    q.iz = iz;
    q.g = (int64_t)ix + (int64_t)m.n[0] * ((int64_t)iy + (int64_t)m.n[1] * iz);
}

// i + k wrapped onto [0, n) for |k| <= 2 (two conditional steps also cover n = 1)
__device__ __forceinline__ int wrap2(int i, int n) {
    if (i >= n) i -= n;
    if (i >= n) i -= n;
    if (i < 0) i += n;
    if (i < 0) i += n;
    return i;
}

// Delta_h f at q: the same sums in the same order as lap(), with wrapped offsets.
__device__ __forceinline__ double lap_at(const double* __restrict__ f, const MeshPos& q, const MeshDims& m,
                                         const double* invH) {
    const int64_t g = q.g, sy = m.n[0], sz = (int64_t)m.n[0] * m.n[1];
    const int64_t xp = g + (wrap2(q.ix + 2, m.n[0]) - q.ix), xm = g + (wrap2(q.ix - 2, m.n[0]) - q.ix);
    const int64_t yp = g + sy * (wrap2(q.iy + 2, m.n[1]) - q.iy), ym = g + sy * (wrap2(q.iy - 2, m.n[1]) - q.iy);
    const int64_t zp = g + sz * (wrap2(q.iz + 2, m.n[2]) - q.iz), zm = g + sz * (wrap2(q.iz - 2, m.n[2]) - q.iz);
    const double c = f[g];
    double s = 0.25 * invH[0] * invH[0] * (f[xp] - 2.0 * c + f[xm]);
    s += 0.25 * invH[1] * invH[1] * (f[yp] - 2.0 * c + f[ym]);
    s += 0.25 * invH[2] * invH[2] * (f[zp] - 2.0 * c + f[zm]);
    return s;
}

struct MeshParams {
    MeshDims m;
    double invH[3];
    double dt, a;      // a = kappa^2 dt^2 / 4
    double c_rho;      // dt^2 kappa^2 sigma1 / 2
    double c_J;        // dt^2 kappa^2 sigma2 / 2
    double kappa2, sigma1, sigma2, dV;
};

MeshParams mesh_params(const Ctx& c) {
    MeshParams p;
    p.m = c.m;
    for (int a = 0; a < 3; ++a) p.invH[a] = c.invH[a];
    p.dt = c.cfg.dt;
    p.kappa2 = c.cfg.kappa * c.cfg.kappa;
    p.a = 0.25 * p.kappa2 * p.dt * p.dt;
    p.c_rho = 0.5 * p.dt * p.dt * p.kappa2 * c.cfg.sigma1;
    p.c_J = 0.5 * p.dt * p.dt * p.kappa2 * c.cfg.sigma2;
    p.sigma1 = c.cfg.sigma1;
    p.sigma2 = c.cfg.sigma2;
    p.dV = c.dV;
    return p;
}

#define GRID_LOOP(g, N) for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < (N); g += (int64_t)gridDim.x * blockDim.x)

__device__ __forceinline__ void put_partial(double* partials, int slot, double v, double* sm, bool is_max) {
    double r = is_max ? block_max(v, sm) : block_sum(v, sm);
    if (threadIdx.x == 0) partials[slot * MAX_BLOCKS + blockIdx.x] = r;
}

// rhs0_f = (I + a Delta_h) F0_f + dt W0_f for the four potentials f = phi, A_x, A_y, A_z.
__global__ void k_rhs0(MeshParams p, const double* __restrict__ F0, const double* __restrict__ W0,
                       double* __restrict__ rhs0) {
    const int64_t N = p.m.ncell;
    GRID_LOOP(g, N) {
        Nb b = decompose(g, p.m);
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const double* u = F0 + f * N;
            rhs0[f * N + g] = u[g] + p.a * lap(u, b, p.m, p.invH) + p.dt * W0[f * N + g];
        }
    }
}

// Continuity (Eq. (cn-continuity)) and the CN sources; e_J partial sums.
__global__ void k_source(MeshParams p, const double* __restrict__ J, const double* __restrict__ Jprev,
                         const double* __restrict__ rho0, const double* __restrict__ rhs0, double* __restrict__ rho1,
                         double* __restrict__ rhs, double* __restrict__ partials) {
    __shared__ double sm[32];
    const int64_t N = p.m.ncell;
    double num = 0.0, den = 0.0;
    GRID_LOOP(g, N) {
        Nb b = decompose(g, p.m);
        double divJ = dcen(J, b, 0, p.m, p.invH) + dcen(J + N, b, 1, p.m, p.invH) + dcen(J + 2 * N, b, 2, p.m, p.invH);
        double r0 = rho0[g];
        double r1 = r0 - p.dt * divJ;
        rho1[g] = r1;
        rhs[g] = rhs0[g] + p.c_rho * 0.5 * (r1 + r0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double j = J[c * N + g];
            rhs[(1 + c) * N + g] = rhs0[(1 + c) * N + g] + p.c_J * j;
            den += j * j;
            if (Jprev) {
                double d = j - Jprev[c * N + g];
                num += d * d;
            }
        }
    }
    put_partial(partials, S_EJ_NUM, num, sm, false);
    put_partial(partials, S_EJ_DEN, den, sm, false);
}

// The current fixed-point error of one Picard update (Algorithm 1's convergence test):
// partials of |J_new - J_old|^2 and |J_new|^2 over the 3 N mesh values, J_new being the orbit
// current of the new iterate and J_old that of the iterate it was computed from.
__global__ void k_jdiff(int64_t n3, const double* __restrict__ Jnew, const double* __restrict__ Jold,
                        double* __restrict__ partials) {
    __shared__ double sm[32];
    double num = 0.0, den = 0.0;
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n3; g += (int64_t)gridDim.x * blockDim.x) {
        const double j = Jnew[g];
        const double d = j - Jold[g];
        num += d * d;
        den += j * j;
    }
    put_partial(partials, S_EJ_NUM, num, sm, false);
    put_partial(partials, S_EJ_DEN, den, sm, false);
}

// One Chebyshev step on field blockIdx.y:  r = b - (c_id I - c_lap Delta_h) x,
// d = alpha d + beta r,  x_out = x + d   (the three-term recurrence in its
// "true residual" form, so rounding errors do not accumulate in r).
__global__ void k_cheb(MeshParams p, const double* __restrict__ x, double* __restrict__ xout, double* __restrict__ d,
                       const double* __restrict__ bvec, double c_id, double c_lap, double alpha, double beta,
                       StrideDigits sd) {
    const int64_t N = p.m.ncell;
    const int64_t off = blockIdx.y * N;
    const double* xf = x + off;
    const int64_t start = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    MeshPos q = pos_of(start, p.m);
    for (int64_t g = start; g < N; g += (int64_t)gridDim.x * blockDim.x, advance(q, sd, p.m)) {
        double Hx = c_id * xf[g] - c_lap * lap_at(xf, q, p.m, p.invH);
        double r = bvec[off + g] - Hx;
        double dn = (alpha == 0.0 ? 0.0 : alpha * d[off + g]) + beta * r;
        d[off + g] = dn;
        xout[off + g] = xf[g] + dn;
    }
}

// psi^{n+1} = 2 (phi^{n+1} - phi^n) / dt - psi^n (and U from A), then the gather table:
// A^n, A^{n+1}, grad_h phi^{n+1/2}, U^{n+1/2}.
// The Chebyshev steps of a CN mesh phase in one cooperative launch: the same element-wise
// update as k_cheb on every field, with a grid-wide barrier between steps (step k reads xa for
// even k and xb for odd k and writes the other).
//
// Step count.  The operator I - a Delta_h has spectrum in [1, lmax], so the initial error of
// field f obeys |e_0| <= |r_0| (r_0 = b - A x_0, the warm start's residual) and after K steps
// |e_K| <= 2 rho^K |r_0|, rho = (sqrt(lmax) - 1) / (sqrt(lmax) + 1); the solution obeys
// |x| >= |b| / lmax.  Step 0 measures |r_0,f| and |b_f| (a grid reduction in a fixed order,
// so every block takes the same decision) and the solve stops after the smallest K with
// 2 rho^K |r_0,f| lmax <= tol |b_f| for every field, rounded up to the parity of the full
// schedule (so the result lands in the same buffer) and at most `iters`.  A warm start that is
// already close, as in the later Picard iterations, needs far fewer steps than the schedule.
__global__ void __launch_bounds__(THREADS) k_cheb_all(MeshParams p, double* xa, double* xb, double* __restrict__ d,
                                                      const double* __restrict__ bvec, double c_id, double c_lap,
                                                      int nfields, int iters, const double* __restrict__ alpha,
                                                      const double* __restrict__ beta, double* __restrict__ red,
                                                      double lmax, double rate, double tol, StrideDigits sd) {
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    __shared__ double sm[32];
    __shared__ int sK;
    const int64_t N = p.m.ncell, total = (int64_t)nfields * N;
    double r2[4] = {0.0, 0.0, 0.0, 0.0}, b2[4] = {0.0, 0.0, 0.0, 0.0};
    int K = iters;
    for (int k = 0; k < K; ++k) {
        const double* x = (k & 1) ? xb : xa;
        double* xo = (k & 1) ? xa : xb;
        const double al = alpha[k], be = beta[k];
        const int64_t start = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        MeshPos q = pos_of(start, p.m);
        for (int64_t idx = start; idx < total; idx += (int64_t)gridDim.x * blockDim.x, advance(q, sd, p.m)) {
            const int f = q.f;
            const int64_t g = q.g, off = (int64_t)f * N;
            const double* xf = x + off;
            double Hx = c_id * xf[g] - c_lap * lap_at(xf, q, p.m, p.invH);
            const double bv = bvec[off + g];
            double r = bv - Hx;
            if (k == 0) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    r2[q] += q == f ? r * r : 0.0;
                    b2[q] += q == f ? bv * bv : 0.0;
                }
            }
            double dn = (al == 0.0 ? 0.0 : al * d[off + g]) + be * r;
            d[off + g] = dn;
            xo[off + g] = xf[g] + dn;
        }
        if (k == 0 && rate > 0.0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const double sr = block_sum(r2[q], sm);
                const double sb = block_sum(b2[q], sm);
                if (threadIdx.x == 0) {
                    red[blockIdx.x * 8 + q] = sr;
                    red[blockIdx.x * 8 + 4 + q] = sb;
                }
            }
        }
        grid.sync();
        if (k == 0 && rate > 0.0) {
            // every block sums the per-block partials the same way: thread t takes blocks
            // t, t + blockDim, ..., then a fixed-order block sum
            double tot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                double v = 0.0;
                for (unsigned blk = threadIdx.x; blk < gridDim.x; blk += blockDim.x) v += red[blk * 8 + q];
                tot[q] = block_sum(v, sm);
            }
            if (threadIdx.x == 0) {
                int need = 1;
                for (int q = 0; q < nfields; ++q) {
                    const double sr = tot[q], sb = tot[4 + q];
                    int kq;
                    if (sr == 0.0) kq = 1;
                    else if (sb == 0.0) kq = iters;
                    else {
                        const double ratio = 2.0 * sqrt(sr) * lmax / (tol * sqrt(sb));
                        kq = ratio <= 1.0 ? 1 : (int)ceil(log(ratio) * rate);
                    }
                    need = max(need, kq);
                }
                need = min(need, iters);
                if ((need & 1) != (iters & 1)) need = min(need + 1, iters);
                sK = need;
            }
            __syncthreads();
            K = sK;
        }
    }
}

__global__ void k_backsub_table(MeshParams p, const double* __restrict__ F0, const double* __restrict__ W0,
                                const double* __restrict__ F1, double* __restrict__ W1, double* __restrict__ table) {
    const int64_t N = p.m.ncell;
    GRID_LOOP(g, N) {
        Nb b = decompose(g, p.m);
        double w1[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            w1[f] = 2.0 * (F1[f * N + g] - F0[f * N + g]) / p.dt - W0[f * N + g];
            W1[f * N + g] = w1[f];
        }
        double* t = table + 12 * g;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            t[c] = F0[(1 + c) * N + g];
            t[3 + c] = F1[(1 + c) * N + g];
            t[9 + c] = 0.5 * (w1[1 + c] + W0[(1 + c) * N + g]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) t[6 + a] = 0.5 * (dcen(F1, b, a, p.m, p.invH) + dcen(F0, b, a, p.m, p.invH));
    }
}

// Field energy W = sum_g (|E|^2 / (2 sigma1) + |B|^2 / (2 sigma2)) dV, E = -grad phi - U, B = curl A.
__device__ __forceinline__ double node_energy(const MeshParams& p, const double* F, const double* W, const Nb& b) {
    const int64_t N = p.m.ncell;
    const double* phi = F;
    const double* Ax = F + N;
    const double* Ay = F + 2 * N;
    const double* Az = F + 3 * N;
    double E[3], B[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) E[a] = -dcen(phi, b, a, p.m, p.invH) - W[(1 + a) * N + b.g];
    B[0] = dcen(Az, b, 1, p.m, p.invH) - dcen(Ay, b, 2, p.m, p.invH);
    B[1] = dcen(Ax, b, 2, p.m, p.invH) - dcen(Az, b, 0, p.m, p.invH);
    B[2] = dcen(Ay, b, 0, p.m, p.invH) - dcen(Ax, b, 1, p.m, p.invH);
    return ((E[0] * E[0] + E[1] * E[1] + E[2] * E[2]) / (2.0 * p.sigma1) +
            (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]) / (2.0 * p.sigma2)) * p.dV;
}

__global__ void k_mesh_energy(MeshParams p, const double* __restrict__ F, const double* __restrict__ W,
                              double* __restrict__ partials, int slot) {
    __shared__ double sm[32];
    double e = 0.0;
    GRID_LOOP(g, p.m.ncell) e += node_energy(p, F, W, decompose(g, p.m));
    put_partial(partials, slot, e, sm, false);
}

// §5.1-§5.3 mesh diagnostics of the accepted step.
__global__ void k_mesh_diag(MeshParams p, const double* __restrict__ F0, const double* __restrict__ W0,
                            const double* __restrict__ rho0, const double* __restrict__ F1,
                            const double* __restrict__ W1, const double* __restrict__ rho1,
                            const double* __restrict__ J, double* __restrict__ partials) {
    __shared__ double sm[32];
    const int64_t N = p.m.ncell;
    double w1 = 0.0, mwork = 0.0, gmax = 0.0, gsq = 0.0, rmax = 0.0, rsq = 0.0, cmax = 0.0;
    GRID_LOOP(g, N) {
        Nb b = decompose(g, p.m);
        w1 += node_energy(p, F1, W1, b);
        // J . E^{n+1/2} dV
        double divJ = 0.0, divA = 0.0, divU = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double Eh = -0.5 * (dcen(F1, b, a, p.m, p.invH) + dcen(F0, b, a, p.m, p.invH)) -
                        0.5 * (W1[(1 + a) * N + g] + W0[(1 + a) * N + g]);
            mwork += J[a * N + g] * Eh * p.dV;
            divJ += dcen(J + a * N, b, a, p.m, p.invH);
            divA += dcen(F1 + (1 + a) * N, b, a, p.m, p.invH);
            divU += dcen(W1 + (1 + a) * N, b, a, p.m, p.invH);
        }
        double G = W1[g] / p.kappa2 + divA;                              // Eq. (gauge-diagnostic)
        double R = -lap(F1, b, p.m, p.invH) - divU - p.sigma1 * rho1[g]; // Eq. (gauss-diagnostic)
        double C = rho1[g] - rho0[g] + p.dt * divJ;
        gmax = fmax(gmax, fabs(G));
        gsq += G * G;
        rmax = fmax(rmax, fabs(R));
        rsq += R * R;
        cmax = fmax(cmax, fabs(C));
    }
    put_partial(partials, S_W, w1, sm, false);
    put_partial(partials, S_MWORK, mwork, sm, false);
    put_partial(partials, S_G_MAX, gmax, sm, true);
    put_partial(partials, S_G_SQ, gsq, sm, false);
    put_partial(partials, S_R_MAX, rmax, sm, true);
    put_partial(partials, S_R_SQ, rsq, sm, false);
    put_partial(partials, S_CONT_MAX, cmax, sm, true);
}

// Projections of f on the 8 patterns (-1)^(a . i), a in {0,1}^3.
__global__ void k_null_dots(MeshParams p, const double* __restrict__ f, double* __restrict__ partials) {
    __shared__ double sm[32];
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    GRID_LOOP(g, p.m.ncell) {
        Nb b = decompose(g, p.m);
        double v = f[g];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            int par = ((k & 1) ? b.ix : 0) + ((k & 2) ? b.iy : 0) + ((k & 4) ? b.iz : 0);
            acc[k] += (par & 1) ? -v : v;
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) put_partial(partials, S_PROJ0 + k, acc[k], sm, false);
}

// f -= sum over null patterns of (f . pattern / N) pattern, then f += add_const (added before
// projecting would be removed again, so the constant is only used with projection skipped).
__global__ void k_null_subtract(MeshParams p, double* __restrict__ f, const double* __restrict__ results) {
    const int64_t N = p.m.ncell;
    GRID_LOOP(g, N) {
        Nb b = decompose(g, p.m);
        double v = f[g];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            bool null_mode = (!(k & 1) || (p.m.n[0] % 2 == 0)) && (!(k & 2) || (p.m.n[1] % 2 == 0)) &&
                             (!(k & 4) || (p.m.n[2] % 2 == 0));
            if (!null_mode) continue;
            int par = ((k & 1) ? b.ix : 0) + ((k & 2) ? b.iy : 0) + ((k & 4) ? b.iz : 0);
            double coef = results[S_PROJ0 + k] / (double)N;
            v -= (par & 1) ? -coef : coef;
        }
        f[g] = v;
    }
}

__global__ void k_add_const(double* __restrict__ f, int64_t n, double c) {
    GRID_LOOP(i, n) f[i] += c;
}

// Fold nblocks partials of each slot, in a fixed order, into results[slot].
__global__ void k_finalize(const double* __restrict__ partials, double* __restrict__ results, int slot0, int nblocks,
                           int is_max) {
    __shared__ double sm[32];
    const int slot = slot0 + blockIdx.x;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        double x = partials[slot * MAX_BLOCKS + b];
        v = is_max ? fmax(v, x) : v + x;
    }
    double r = is_max ? block_max(v, sm) : block_sum(v, sm);
    if (threadIdx.x == 0) results[slot] = r;
}

__global__ void k_fill(double* __restrict__ p, int64_t n, double v) {
    GRID_LOOP(i, n) p[i] = v;
}

__global__ void k_scale_copy(double* __restrict__ dst, const double* __restrict__ src, int64_t n, double s) {
    GRID_LOOP(i, n) dst[i] = s * src[i];
}

__global__ void k_add_to(double* __restrict__ dst, const double* __restrict__ src, int64_t n) {
    GRID_LOOP(i, n) dst[i] += src[i];
}

}  // namespace

int mesh_blocks(const Ctx& c) {
    int64_t b = (c.m.ncell + THREADS - 1) / THREADS;
    int64_t cap = (int64_t)c.sms * 8;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

void launch_rhs0(Ctx& c) {
    k_rhs0<<<mesh_blocks(c), THREADS, 0, c.stream>>>(mesh_params(c), c.F0, c.W0, c.rhs0);
    ++c.launches;
}

void launch_source(Ctx& c, const double* Jcur, const double* Jprev) {
    k_source<<<mesh_blocks(c), THREADS, 0, c.stream>>>(mesh_params(c), Jcur, Jprev, c.rho0, c.rhs0, c.rho1, c.rhs,
                                                       c.partials);
    ++c.launches;
}

void launch_jdiff(Ctx& c, const double* Jnew, const double* Jold) {
    k_jdiff<<<mesh_blocks(c), THREADS, 0, c.stream>>>(3 * c.m.ncell, Jnew, Jold, c.partials);
    ++c.launches;
}

void launch_helmholtz(Ctx& c, const double* b, double c_id, double c_lap, int nfields, int iters, const double* alpha,
                      const double* beta, double** x_io, double** x_spare) {
    MeshParams p = mesh_params(c);
    dim3 grid(mesh_blocks(c), nfields);
    const StrideDigits sd = stride_digits((int64_t)grid.x * THREADS, c.m);
    for (int k = 0; k < iters; ++k) {
        k_cheb<<<grid, THREADS, 0, c.stream>>>(p, *x_io, *x_spare, c.cheb_d, b, c_id, c_lap, alpha[k], beta[k], sd);
        ++c.launches;
        std::swap(*x_io, *x_spare);
    }
}

// The CN Helmholtz solve of a mesh phase by FFT (c.helm_fft), exact per mode up to the
// transforms' rounding (~1e-14 of the solution), then one step of iterative refinement: the
// residual r = b - (I - a Delta_h) x from the stencil (a k_cheb step with alpha = 0, beta = 1
// leaves r in c.cheb_d), its FFT solve, x += that.  The refined solution is accurate to the
// rounding of the residual, like the Chebyshev solve at helmholtz_tol; psi and U, which take
// 2 / dt times the change of phi and A, need that.
void launch_helmholtz_fft_refined(Ctx& c, double* x) {
    const double a = 0.25 * c.cfg.kappa * c.cfg.kappa * c.cfg.dt * c.cfg.dt;
    const int64_t N = c.m.ncell;
    launch_helmholtz_fft(c, c.rhs, x, 4, a);
    MeshParams p = mesh_params(c);
    dim3 grid(mesh_blocks(c), 4);
    const StrideDigits sd = stride_digits((int64_t)grid.x * THREADS, c.m);
    k_cheb<<<grid, THREADS, 0, c.stream>>>(p, x, c.F1b, c.cheb_d, c.rhs, 1.0, a, 0.0, 1.0, sd);
    ++c.launches;
    launch_helmholtz_fft(c, c.cheb_d, c.F1b, 4, a);
    k_add_to<<<mesh_blocks(c), THREADS, 0, c.stream>>>(x, c.F1b, 4 * N);
    ++c.launches;
}

// The CN Helmholtz solve of a mesh phase: one cooperative launch when the device allows
// it (the step coefficients are in device memory), which stops at the first step whose error
// bound is below tol times the solution's norm; else one launch per step of the full schedule.
void launch_helmholtz_cn(Ctx& c, double** x_io, double** x_spare, double tol) {
    const double a = 0.25 * c.cfg.kappa * c.cfg.kappa * c.cfg.dt * c.cfg.dt;
    if (c.cheb_coop_blocks <= 0 || !c.cheb_coef_dev) {
        launch_helmholtz(c, c.rhs, 1.0, a, 4, c.cheb_iters, c.cheb_alpha, c.cheb_beta, x_io, x_spare);
        return;
    }
    MeshParams p = mesh_params(c);
    double* xa = *x_io;
    double* xb = *x_spare;
    const double* bvec = c.rhs;
    double c_id = 1.0, c_lap = a;
    int nf = 4, iters = c.cheb_iters;
    const double* al = c.cheb_coef_dev;
    const double* be = c.cheb_coef_dev + 1024;
    double lmax = c.cheb_lmax, rate = c.cheb_rate;
    const int64_t want = (4 * c.m.ncell + THREADS - 1) / THREADS;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, c.cheb_coop_blocks));
    StrideDigits sd = stride_digits((int64_t)grid * THREADS, c.m);
    void* args[] = {&p, &xa, &xb, &c.cheb_d, &bvec, &c_id, &c_lap, &nf, &iters, &al, &be, &c.cheb_red, &lmax, &rate,
                    &tol, &sd};
    cudaLaunchCooperativeKernel((const void*)k_cheb_all, dim3(grid), dim3(THREADS), args, 0, c.stream);
    ++c.launches;
    if (iters & 1) std::swap(*x_io, *x_spare);
}

// Co-resident blocks of k_cheb_all on the device (0: no cooperative launch).
int cheb_coop_capacity(const Ctx& c) {
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cheb_all, THREADS, 0) != cudaSuccess) return 0;
    return per_sm * c.sms;
}

void launch_backsub_table(Ctx& c, bool) {
    k_backsub_table<<<mesh_blocks(c), THREADS, 0, c.stream>>>(mesh_params(c), c.F0, c.W0, c.F1, c.W1, c.table);
    ++c.launches;
}

void launch_null_project(Ctx& c, double* f, double add_const) {
    MeshParams p = mesh_params(c);
    int nb = mesh_blocks(c);
    if (add_const != 0.0) {
        k_add_const<<<nb, THREADS, 0, c.stream>>>(f, c.m.ncell, add_const);
        ++c.launches;
    }
    k_null_dots<<<nb, THREADS, 0, c.stream>>>(p, f, c.partials);
    ++c.launches;
    launch_finalize(c, S_PROJ0, 8, nb, false);
    k_null_subtract<<<nb, THREADS, 0, c.stream>>>(p, f, c.results);
    ++c.launches;
}

void launch_mesh_energy(Ctx& c, const double* F, const double* W, int slot) {
    k_mesh_energy<<<mesh_blocks(c), THREADS, 0, c.stream>>>(mesh_params(c), F, W, c.partials, slot);
    ++c.launches;
}

void launch_mesh_diag(Ctx& c, const double* Jfinal) {
    k_mesh_diag<<<mesh_blocks(c), THREADS, 0, c.stream>>>(mesh_params(c), c.F0, c.W0, c.rho0, c.F1, c.W1, c.rho1,
                                                          Jfinal, c.partials);
    ++c.launches;
}

void launch_finalize(Ctx& c, int slot0, int nslots, int nblocks, bool is_max) {
    k_finalize<<<nslots, THREADS, 0, c.stream>>>(c.partials, c.results, slot0, nblocks, is_max ? 1 : 0);
    ++c.launches;
}

void launch_fill(Ctx& c, double* p, int64_t n, double value) {
    k_fill<<<mesh_blocks(c), THREADS, 0, c.stream>>>(p, n, value);
    ++c.launches;
}

void launch_scale_copy(Ctx& c, double* dst, const double* src, int64_t n, double s) {
    k_scale_copy<<<std::max(mesh_blocks(c), particle_blocks(c)), THREADS, 0, c.stream>>>(dst, src, n, s);
    ++c.launches;
}

}  // namespace pic
