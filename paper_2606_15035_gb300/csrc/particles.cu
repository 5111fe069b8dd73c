// Particle kernels of the orbit-averaged PIC step (FP64, sm_103a).
//
// One particle per thread, grid-stride loops, particles in structure-of-arrays layout
// (component c of particle i at c * np + i) and cell-sorted so that neighbouring
// threads gather the same mesh nodes.  Mesh data for the gather come from a per-node
// table of 12 doubles: A^n (3), A^{n+1,p} (3), grad_h phi^{n+1/2,p} (3), U^{n+1/2,p} (3).
#include <algorithm>
#include <cmath>

#include "pic_internal.h"
#include "particle_common.cuh"

namespace pic {

__constant__ double c_gauss_t[16];
__constant__ double c_gauss_w[16];

// Gauss-Legendre nodes on [0, 1] by Newton's method on the Legendre polynomial P_nq
// (three-term recurrence), weights 1 / ((1 - x^2) P'(x)^2) mapped from [-1, 1].
void set_gauss_rule(int nq) {
    double t[16] = {0}, w[16] = {0};
    for (int k = 0; k < nq; ++k) {
        double x = std::cos(M_PI * (k + 0.75) / (nq + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= nq; ++j) {
                double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pn = nq == 0 ? 1.0 : (nq == 1 ? x : p1);
            double pm = nq == 1 ? 1.0 : p0;
            dp = nq * (x * pn - pm) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-17) break;
        }
        t[k] = 0.5 * (1.0 - x);
        w[k] = 1.0 / ((1.0 - x * x) * dp * dp);  // = 0.5 * 2 / ((1 - x^2) P'^2)
    }
    cudaMemcpyToSymbol(c_gauss_t, t, sizeof(t));
    cudaMemcpyToSymbol(c_gauss_w, w, sizeof(w));
}

namespace {


// ---- orbit current scatter (Eq. (orbit-current)) -------------------------------------

// J_c[g] += w_c * Sbar contribution of every piece (closed form, Appendix A).
__device__ __forceinline__ int scatter_closed(const StepParams& p, const double x0[3], const double beta[3],
                                              const double w[3], double* __restrict__ J) {
    const int64_t N = p.m.ncell;
    return for_each_segment(x0, beta, true, [&](const Segment<double>& sg) {
        double I[8];
        int64_t g[8];
        weights_from_ints(piece_integrals(sg, beta, false), I);
        segment_nodes8(sg, p.m, g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (p.det) {
                exact_add(p.acc, g[k], w[0] * I[k]);
                exact_add(p.acc, N + g[k], w[1] * I[k]);
                exact_add(p.acc, 2 * N + g[k], w[2] * I[k]);
            } else {
                atomicAdd(J + g[k], w[0] * I[k]);
                atomicAdd(J + N + g[k], w[1] * I[k]);
                atomicAdd(J + 2 * N + g[k], w[2] * I[k]);
            }
        }
    });
}

// Same with an n_q-point Gauss rule on each piece (split) or on the whole path (unsplit).
__device__ __forceinline__ int scatter_gauss(const StepParams& p, const double x0[3], const double beta[3],
                                             const double w[3], double* __restrict__ J) {
    const int64_t N = p.m.ncell;
    return for_each_segment(x0, beta, p.split != 0, [&](const Segment<double>& sg) {
        for (int qd = 0; qd < p.nq; ++qd) {
            double s = sg.s0 + sg.h * c_gauss_t[qd];
            double wq = sg.h * c_gauss_w[qd];
            double xq[3] = {x0[0] + s * beta[0], x0[1] + s * beta[1], x0[2] + s * beta[2]};
            int64_t g[8];
            double S[8];
            point_weights8(xq, p.m, g, S);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                double f = wq * S[k];
                if (p.det) {
                    exact_add(p.acc, g[k], w[0] * f);
                    exact_add(p.acc, N + g[k], w[1] * f);
                    exact_add(p.acc, 2 * N + g[k], w[2] * f);
                } else {
                    atomicAdd(J + g[k], w[0] * f);
                    atomicAdd(J + N + g[k], w[1] * f);
                    atomicAdd(J + 2 * N + g[k], w[2] * f);
                }
            }
        }
    });
}

// ---- shapes of degree R = 2, 3 (§4.7) ---------------------------------------------------
//
// One axis of the tensor-product B-spline of degree R at x (cell units): the R + 1 non-zero
// values, their x-derivatives and the first node.  The nodes sit at the integers, the knots
// at the integers (odd R) or the half-integers (even R); on the knot interval holding x, in
// its local coordinate t in [0, 1), the centred cardinal B-spline's pieces are
//   R = 2:  (1 - t)^2 / 2,  1/2 + t (1 - t),  t^2 / 2;
//   R = 3:  (1 - t)^3 / 6,  (3 t^3 - 6 t^2 + 4) / 6,  (-3 t^3 + 3 t^2 + 3 t + 1) / 6,  t^3 / 6.
template <int R>
struct Basis1 {
    double w[R + 1], dw[R + 1];
    int first;
};

template <int R>
__device__ __forceinline__ void basis1(double x, double invH, Basis1<R>& b) {
    const double xs = (R % 2 == 0) ? x - 0.5 : x;
    const double f = floor(xs), t = xs - f, u = 1.0 - t;
    b.first = (int)f - (R - 1) / 2;
    if constexpr (R == 2) {
        b.w[0] = 0.5 * u * u;
        b.w[1] = 0.5 + t * u;
        b.w[2] = 0.5 * t * t;
        b.dw[0] = -u * invH;
        b.dw[1] = (u - t) * invH;
        b.dw[2] = t * invH;
    } else {
        const double t2 = t * t, t3 = t2 * t;
        b.w[0] = u * u * u * (1.0 / 6.0);
        b.w[1] = (3.0 * t3 - 6.0 * t2 + 4.0) * (1.0 / 6.0);
        b.w[2] = (-3.0 * t3 + 3.0 * t2 + 3.0 * t + 1.0) * (1.0 / 6.0);
        b.w[3] = t3 * (1.0 / 6.0);
        b.dw[0] = -0.5 * u * u * invH;
        b.dw[1] = (1.5 * t2 - 2.0 * t) * invH;
        b.dw[2] = (-1.5 * t2 + t + 0.5) * invH;
        b.dw[3] = 0.5 * t2 * invH;
    }
}

template <int R>
__device__ __forceinline__ void basis3(const StepParams& p, const double x[3], Basis1<R> b[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) basis1<R>(x[a], p.invH[a], b[a]);
}

// Visit the (R + 1)^3 nodes of the shape at a point: f(node row, S_g, grad S_g).
template <int R, typename F>
__device__ __forceinline__ void for_each_node(const StepParams& p, const Basis1<R> b[3], F&& f) {
    for (int iz = 0; iz <= R; ++iz) {
        const int gz = wrapi(b[2].first + iz, p.m.n[2]);
        for (int iy = 0; iy <= R; ++iy) {
            const int gy = wrapi(b[1].first + iy, p.m.n[1]);
            const double wyz = b[1].w[iy] * b[2].w[iz];
            const double dy = b[1].dw[iy] * b[2].w[iz], dz = b[1].w[iy] * b[2].dw[iz];
#pragma unroll
            for (int ix = 0; ix <= R; ++ix) {
                const int gx = wrapi(b[0].first + ix, p.m.n[0]);
                const double wx = b[0].w[ix];
                const double dS[3] = {b[0].dw[ix] * wyz, wx * dy, wx * dz};
                f(node_index(gx, gy, gz, p.m), wx * wyz, dS);
            }
        }
    }
}

// The orbit current with an n_q-point Gauss rule on each piece between the knots of the
// degree-R shape (split) or on the whole path (unsplit).
template <int R>
__device__ __forceinline__ int scatter_gauss_r(const StepParams& p, const double x0[3], const double beta[3],
                                               const double w[3], double* __restrict__ J) {
    const int64_t N = p.m.ncell;
    const double xs[3] = {x0[0] - p.koff, x0[1] - p.koff, x0[2] - p.koff};
    return for_each_segment(xs, beta, p.split != 0, [&](const Segment<double>& sg) {
        for (int qd = 0; qd < p.nq; ++qd) {
            const double s = sg.s0 + sg.h * c_gauss_t[qd];
            const double wq = sg.h * c_gauss_w[qd];
            const double xq[3] = {x0[0] + s * beta[0], x0[1] + s * beta[1], x0[2] + s * beta[2]};
            Basis1<R> b[3];
            basis3<R>(p, xq, b);
            for_each_node<R>(p, b, [&](int64_t g, double S, const double*) {
                const double f = wq * S;
                if (p.det) {
                    exact_add(p.acc, g, w[0] * f);
                    exact_add(p.acc, N + g, w[1] * f);
                    exact_add(p.acc, 2 * N + g, w[2] * f);
                } else {
                    atomicAdd(J + g, w[0] * f);
                    atomicAdd(J + N + g, w[1] * f);
                    atomicAdd(J + 2 * N + g, w[2] * f);
                }
            });
        }
    });
}

template <int QUAD>
__device__ __forceinline__ int scatter_orbit(const StepParams& p, const double x0[3], const double beta[3],
                                             const double w[3], double* J) {
    if constexpr (QUAD == 0) return scatter_closed(p, x0, beta, w, J);
    else {
        if (p.order == 2) return scatter_gauss_r<2>(p, x0, beta, w, J);
        if (p.order == 3) return scatter_gauss_r<3>(p, x0, beta, w, J);
        return scatter_gauss(p, x0, beta, w, J);
    }
}

// ---- push (Eq. (orbit-push)) -------------------------------------------------------

struct PushAcc {
    double gphi[3];   // orbit gather of grad_h phi^{n+1/2} (Eq. (gphibar-definition))
    double F[3];      // (D_i A)^T vbar (Eq. (DA-def), Appendix B)
    double Ubar[3];   // orbit gather of U^{n+1/2} (Eq. (Ubar-def)), diagnostics only
    double DAv[3];    // (D_i A) vbar, diagnostics only
    double pu;        // sum_g Sbar_ig, diagnostics only
};

template <bool DIAG>
__device__ __forceinline__ void push_piece_closed(const StepParams& p, const Segment<double>& sg, const double beta[3],
                                                  const double vb[3], const double* __restrict__ table, PushAcc& acc) {
    double I[8];
    int64_t g[8];
    segment_weights8(sg, beta, I);
    segment_nodes8(sg, p.m, g);
    const double s = sg.s0, h = sg.h;
    double am[8], cc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double* t = table + 12 * g[k];
        double an = t[0] * vb[0] + t[1] * vb[1] + t[2] * vb[2];   // A^n_g . vbar
        double a1 = t[3] * vb[0] + t[4] * vb[1] + t[5] * vb[2];   // A^{n+1}_g . vbar
        am[k] = (1.0 - s) * an + s * a1;                          // A^{(m)}_nu . vbar
        cc[k] = a1 - an;                                          // C^{(m)}_nu . vbar
        acc.gphi[0] += I[k] * t[6];
        acc.gphi[1] += I[k] * t[7];
        acc.gphi[2] += I[k] * t[8];
        if constexpr (DIAG) {
            acc.Ubar[0] += I[k] * t[9];
            acc.Ubar[1] += I[k] * t[10];
            acc.Ubar[2] += I[k] * t[11];
            acc.pu += I[k];
        }
    }
    AxisPoly<double> px = axis_poly(sg.r[0], beta[0]);
    AxisPoly<double> py = axis_poly(sg.r[1], beta[1]);
    AxisPoly<double> pz = axis_poly(sg.r[2], beta[2]);
    // transverse integrals T0, T1 per derivative direction j and transverse offsets
    double t0x[4], t1x[4], t0y[4], t1y[4], t0z[4], t1z[4];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            transverse_integrals(quad_product(py.L[a], py.M[a], pz.L[b], pz.M[b]), h, t0x[a + 2 * b], t1x[a + 2 * b]);
            transverse_integrals(quad_product(px.L[a], px.M[a], pz.L[b], pz.M[b]), h, t0y[a + 2 * b], t1y[a + 2 * b]);
            transverse_integrals(quad_product(px.L[a], px.M[a], py.L[b], py.M[b]), h, t0z[a + 2 * b], t1z[a + 2 * b]);
        }
    // [(D A)^T vbar]_j = sum_nu (sigma_{nu_j} / H_j) (A^{(m)}_nu.vbar T0 + C_nu.vbar T1)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            int k;
            k = 2 * a + 4 * b;  // nu = (0, a, b) vs (1, a, b)
            acc.F[0] += p.invH[0] * (t0x[a + 2 * b] * (am[k + 1] - am[k]) + t1x[a + 2 * b] * (cc[k + 1] - cc[k]));
            k = a + 4 * b;      // nu = (a, 0, b) vs (a, 1, b)
            acc.F[1] += p.invH[1] * (t0y[a + 2 * b] * (am[k + 2] - am[k]) + t1y[a + 2 * b] * (cc[k + 2] - cc[k]));
            k = a + 2 * b;      // nu = (a, b, 0) vs (a, b, 1)
            acc.F[2] += p.invH[2] * (t0z[a + 2 * b] * (am[k + 4] - am[k]) + t1z[a + 2 * b] * (cc[k + 4] - cc[k]));
        }
    if constexpr (DIAG) {
        // [(D A) vbar]_l = sum_nu (A^{(m)}_{l nu} G0_nu + C_{l nu} G1_nu),
        // G_nu = sum_j sigma_{nu_j} vbar_j / H_j * T_j(transverse of nu)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int nx = k & 1, ny = (k >> 1) & 1, nz = (k >> 2) & 1;
            const double sx = nx ? 1.0 : -1.0, sy = ny ? 1.0 : -1.0, sz = nz ? 1.0 : -1.0;
            double G0 = sx * p.invH[0] * vb[0] * t0x[ny + 2 * nz] + sy * p.invH[1] * vb[1] * t0y[nx + 2 * nz] +
                        sz * p.invH[2] * vb[2] * t0z[nx + 2 * ny];
            double G1 = sx * p.invH[0] * vb[0] * t1x[ny + 2 * nz] + sy * p.invH[1] * vb[1] * t1y[nx + 2 * nz] +
                        sz * p.invH[2] * vb[2] * t1z[nx + 2 * ny];
            const double* t = table + 12 * g[k];
#pragma unroll
            for (int l = 0; l < 3; ++l) {
                double Am = (1.0 - s) * t[l] + s * t[3 + l];
                acc.DAv[l] += Am * G0 + (t[3 + l] - t[l]) * G1;
            }
        }
    }
}

// The same piece contribution from the base integrals (no diagnostics).  For derivative
// direction j with transverse axes (p, q), sum over the four transverse offsets (a, b) of
// T0(a, b) D_ab with T0 = int w_{p,a} w_{q,b} and D_ab the difference across j of the nodes'
// A^{(m)}.vbar, is D00 h + (D10 - D00) Sp + (D01 - D00) Sq + (D11 - D10 - D01 + D00) Spq;
// the T1 (eta-weighted, C^{(m)}.vbar) sum has the same form with h^2/2, Ep, Eq, Epq.
__device__ __forceinline__ void push_piece_fast(const StepParams& p, const Segment<double>& sg, const double beta[3],
                                                const double vb[3], const double* __restrict__ table, PushAcc& acc) {
    const PieceInts<double> I = piece_integrals(sg, beta, true);
    double W[8];
    weights_from_ints(I, W);
    int64_t g[8];
    segment_nodes8(sg, p.m, g);
    const double s = sg.s0, oms = 1.0 - s, h = sg.h, hh2 = 0.5 * h * h;
    double am[8], cc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double* t = table + 12 * g[k];
        const double an = t[0] * vb[0] + t[1] * vb[1] + t[2] * vb[2];   // A^n_g . vbar
        const double a1 = t[3] * vb[0] + t[4] * vb[1] + t[5] * vb[2];   // A^{n+1}_g . vbar
        am[k] = oms * an + s * a1;                                       // A^{(m)}_nu . vbar
        cc[k] = a1 - an;                                                 // C^{(m)}_nu . vbar
        acc.gphi[0] += W[k] * t[6];
        acc.gphi[1] += W[k] * t[7];
        acc.gphi[2] += W[k] * t[8];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int pa = j == 0 ? 1 : 0, qa = j == 2 ? 1 : 2;              // transverse axes
        const int sp = j == 0 ? 2 : 1, sq = j == 2 ? 2 : 4;              // their index strides
        const int sj = j == 0 ? 1 : (j == 1 ? 2 : 4);                    // stride of axis j
        const double D00 = am[sj] - am[0], D10 = am[sp + sj] - am[sp];
        const double D01 = am[sq + sj] - am[sq], D11 = am[sp + sq + sj] - am[sp + sq];
        const double C00 = cc[sj] - cc[0], C10 = cc[sp + sj] - cc[sp];
        const double C01 = cc[sq + sj] - cc[sq], C11 = cc[sp + sq + sj] - cc[sp + sq];
        const double t0 = D00 * h + (D10 - D00) * I.S1[pa] + (D01 - D00) * I.S1[qa] +
                          (D11 - D10 - D01 + D00) * I.S2[j];
        const double t1 = C00 * hh2 + (C10 - C00) * I.E1[pa] + (C01 - C00) * I.E1[qa] +
                          (C11 - C10 - C01 + C00) * I.E2[j];
        acc.F[j] += p.invH[j] * (t0 + t1);
    }
}

template <bool DIAG>
__device__ __forceinline__ void push_piece_gauss(const StepParams& p, const Segment<double>& sg, const double x0[3],
                                                 const double beta[3], const double vb[3],
                                                 const double* __restrict__ table, PushAcc& acc) {
    for (int qd = 0; qd < p.nq; ++qd) {
        const double s = sg.s0 + sg.h * c_gauss_t[qd];
        const double wq = sg.h * c_gauss_w[qd];
        double xq[3] = {x0[0] + s * beta[0], x0[1] + s * beta[1], x0[2] + s * beta[2]};
        int c[3];
        double r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double f = floor(xq[a]);
            c[a] = (int)f;
            r[a] = xq[a] - f;
        }
        Segment<double> cs;
        cs.cell[0] = c[0];
        cs.cell[1] = c[1];
        cs.cell[2] = c[2];
        int64_t g[8];
        segment_nodes8(cs, p.m, g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int nx = k & 1, ny = (k >> 1) & 1, nz = (k >> 2) & 1;
            const double wx = nx ? r[0] : 1.0 - r[0], wy = ny ? r[1] : 1.0 - r[1], wz = nz ? r[2] : 1.0 - r[2];
            const double W = wq * wx * wy * wz;
            const double dW[3] = {wq * (nx ? p.invH[0] : -p.invH[0]) * wy * wz,
                                  wq * (ny ? p.invH[1] : -p.invH[1]) * wx * wz,
                                  wq * (nz ? p.invH[2] : -p.invH[2]) * wx * wy};
            const double* t = table + 12 * g[k];
            const double an = t[0] * vb[0] + t[1] * vb[1] + t[2] * vb[2];
            const double a1 = t[3] * vb[0] + t[4] * vb[1] + t[5] * vb[2];
            const double as = (1.0 - s) * an + s * a1;           // A_g(s) . vbar
            acc.gphi[0] += W * t[6];
            acc.gphi[1] += W * t[7];
            acc.gphi[2] += W * t[8];
            acc.F[0] += as * dW[0];
            acc.F[1] += as * dW[1];
            acc.F[2] += as * dW[2];
            if constexpr (DIAG) {
                acc.Ubar[0] += W * t[9];
                acc.Ubar[1] += W * t[10];
                acc.Ubar[2] += W * t[11];
                acc.pu += W;
                const double vdW = vb[0] * dW[0] + vb[1] * dW[1] + vb[2] * dW[2];
#pragma unroll
                for (int l = 0; l < 3; ++l) acc.DAv[l] += ((1.0 - s) * t[l] + s * t[3 + l]) * vdW;
            }
        }
    }
}

// The Gauss-rule piece of push_piece_gauss for the degree-R shape.
template <int R, bool DIAG>
__device__ __forceinline__ void push_piece_gauss_r(const StepParams& p, const Segment<double>& sg, const double x0[3],
                                                   const double beta[3], const double vb[3],
                                                   const double* __restrict__ table, PushAcc& acc) {
    for (int qd = 0; qd < p.nq; ++qd) {
        const double s = sg.s0 + sg.h * c_gauss_t[qd];
        const double wq = sg.h * c_gauss_w[qd];
        const double xq[3] = {x0[0] + s * beta[0], x0[1] + s * beta[1], x0[2] + s * beta[2]};
        Basis1<R> b[3];
        basis3<R>(p, xq, b);
        for_each_node<R>(p, b, [&](int64_t g, double S, const double* dS) {
            const double W = wq * S;
            const double dW[3] = {wq * dS[0], wq * dS[1], wq * dS[2]};
            const double* t = table + 12 * g;
            const double an = t[0] * vb[0] + t[1] * vb[1] + t[2] * vb[2];
            const double a1 = t[3] * vb[0] + t[4] * vb[1] + t[5] * vb[2];
            const double as = (1.0 - s) * an + s * a1;           // A_g(s) . vbar
            acc.gphi[0] += W * t[6];
            acc.gphi[1] += W * t[7];
            acc.gphi[2] += W * t[8];
            acc.F[0] += as * dW[0];
            acc.F[1] += as * dW[1];
            acc.F[2] += as * dW[2];
            if constexpr (DIAG) {
                acc.Ubar[0] += W * t[9];
                acc.Ubar[1] += W * t[10];
                acc.Ubar[2] += W * t[11];
                acc.pu += W;
                const double vdW = vb[0] * dW[0] + vb[1] * dW[1] + vb[2] * dW[2];
#pragma unroll
                for (int l = 0; l < 3; ++l) acc.DAv[l] += ((1.0 - s) * t[l] + s * t[3 + l]) * vdW;
            }
        });
    }
}

// Point interpolant of columns [col, col+3) of the table at a wrapped position.
__device__ __forceinline__ void point_gather3(const StepParams& p, const double xq[3], const double* __restrict__ table,
                                              int col, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    auto add = [&](int64_t g, double S, const double*) {
        const double* t = table + 12 * g + col;
        out[0] += S * t[0];
        out[1] += S * t[1];
        out[2] += S * t[2];
    };
    if (p.order == 2) {
        Basis1<2> b[3];
        basis3<2>(p, xq, b);
        for_each_node<2>(p, b, add);
        return;
    }
    if (p.order == 3) {
        Basis1<3> b[3];
        basis3<3>(p, xq, b);
        for_each_node<3>(p, b, add);
        return;
    }
    int64_t g[8];
    double w[8];
    point_weights8(xq, p.m, g, w);
#pragma unroll
    for (int k = 0; k < 8; ++k) add(g[k], w[k], nullptr);
}

// ---- kernels ----------------------------------------------------------------------

__global__ void k_init_positions(StepParams p, const double* __restrict__ x, double* __restrict__ xi,
                                 int64_t* __restrict__ id) {
    const int64_t np = p.np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) xi[a * np + i] = wrap_pos_any(x[a * np + i] * p.invH[a], (double)p.m.n[a]);
        id[i] = i;
    }
}

// Cell-unit positions in caller order -> device order, wrapped to [0, n_a) (the identity on
// values already in range).
__global__ void k_set_positions(StepParams p, const int64_t* __restrict__ id, const double* __restrict__ src,
                                double* __restrict__ xi) {
    const int64_t np = p.np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) xi[a * np + i] = wrap_pos_any(src[a * np + id[i]], (double)p.m.n[a]);
    }
}

__global__ void k_point_deposit(StepParams p, const double* __restrict__ xi, double* __restrict__ rho) {
    const int64_t np = p.np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        double x[3] = {xi[i], xi[np + i], xi[2 * np + i]};
        auto dep = [&](int64_t g, double S, const double*) {
            if (p.det) exact_add(p.acc, g, p.q_dV * S);
            else atomicAdd(rho + g, p.q_dV * S);
        };
        if (p.order == 2) {
            Basis1<2> b[3];
            basis3<2>(p, x, b);
            for_each_node<2>(p, b, dep);
        } else if (p.order == 3) {
            Basis1<3> b[3];
            basis3<3>(p, x, b);
            for_each_node<3>(p, b, dep);
        } else {
            int64_t g[8];
            double w[8];
            point_weights8(x, p.m, g, w);
#pragma unroll
            for (int k = 0; k < 8; ++k) dep(g[k], w[k], nullptr);
        }
    }
}

// v^{n+1,0} = 2 v^n - v^{n-1} (Algorithm 1, extrapolated start) unless an iterate is given;
// then the orbit current of that iterate, and sum_i |v^n_i| for the e_J floor.
template <int QUAD>
__global__ void k_first_scatter(StepParams p, const double* __restrict__ xi, const double* __restrict__ v,
                                const double* __restrict__ vprev, const double* __restrict__ vgiven,
                                double* __restrict__ vit, double* __restrict__ J, double* __restrict__ partials,
                                int* __restrict__ status) {
    __shared__ double sm[32];
    __shared__ int order[THREADS];
    __shared__ int wcount[THREADS / 32][PIECE_CLASSES];
    const int64_t np = p.np, nchunks = (np + THREADS - 1) / THREADS;
    double jsc = 0.0;
    // chunks of THREADS particles handed to the threads by orbit-piece count (as in k_push)
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t base = ch * THREADS;
        double x0[3], vn[3], vi[3], beta[3], w[3];
        int cls = PIECE_CLASSES - 1;
        if (base + threadIdx.x < np) {
            const int64_t j = base + threadIdx.x;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = xi[a * np + j];
                vn[a] = v[a * np + j];
                vi[a] = vgiven ? vgiven[a * np + j] : 2.0 * vn[a] - vprev[a * np + j];
                vit[a * np + j] = vi[a];
                beta[a] = p.dt * 0.5 * (vi[a] + vn[a]) * p.invH[a];
            }
            jsc += sqrt(vn[0] * vn[0] + vn[1] * vn[1] + vn[2] * vn[2]);
            cls = piece_class_of(p, x0, beta);
        }
        order[stable_class_rank(cls, wcount)] = threadIdx.x;
        __syncthreads();
        const int64_t i = base + order[threadIdx.x];
        if (i < np) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = xi[a * np + i];
                vn[a] = v[a * np + i];
                vi[a] = vgiven ? vgiven[a * np + i] : 2.0 * vn[a] - vprev[a * np + i];
                const double vb = 0.5 * (vi[a] + vn[a]);
                beta[a] = p.dt * vb * p.invH[a];
                w[a] = p.q_dV * vb;
            }
            if (scatter_orbit<QUAD>(p, x0, beta, w, J) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
        }
        __syncthreads();   // order[] is rewritten by the next chunk
    }
    write_partial<double>(partials, S_JSCALE, jsc, sm, false);
}

// Constants of the particle-local solve for "creeping" particles (see k_local); the
// classifier is_creeping and its BETA_CREEP / D_KNOT live in pic_device.cuh.
constexpr int LOCAL_STEPS = 32;      // push evaluations per creeping particle
constexpr double LOCAL_TOL = 1e-15;  // relative to the particle's speed
constexpr double OMEGA_MAX = 8.0;    // bound on the secant step factor
constexpr double SLIDE_PROBE = 1e-12; // cells: the sliding test probes SLIDE_PROBE short of the knot
constexpr double SLIDE_FAR = 64.0;    // ... and max(SLIDE_PROBE, SLIDE_FAR |d|) past it
constexpr double D_FALLBACK = 1e-6;   // cells: a failed solve slides the components that start
                                      // this near a knot
constexpr double FAIL_RES = 1e-10;    // failed: best residual above FAIL_RES x the speed
constexpr double BETA_TRIAL = 1.0;    // cells: trial orbits stay within this beyond the iterate's
                                      // own orbit, per axis

struct PushOut {
    double Pw[3], xe[3], Ae[3], vw[3];
    int nseg;
};

// G(u): the Algorithm 1 push of one particle for the end-of-step iterate u with the
// current mesh table: orbit vbar = (u + v^n)/2, P^{n+1} (Eq. (orbit-P-update)),
// x^{n+1} (Eq. (orbit-x-update)) and v^{n+1} = (P^{n+1} - q A_h^{n+1}(x^{n+1})) / m.
template <int QUAD, bool DIAG>
__device__ __forceinline__ void push_eval(const StepParams& p, const double x0[3], const double vn[3],
                                          const double Pn[3], const double u[3], const double* __restrict__ table,
                                          PushAcc& acc, PushOut& o) {
    double vb[3], beta[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vb[a] = 0.5 * (u[a] + vn[a]);
        beta[a] = p.dt * vb[a] * p.invH[a];
    }
    acc = PushAcc{};
    if constexpr (QUAD == 0) {
        o.nseg = for_each_segment(x0, beta, true, [&](const Segment<double>& sg) {
            if constexpr (DIAG) push_piece_closed<true>(p, sg, beta, vb, table, acc);
            else push_piece_fast(p, sg, beta, vb, table, acc);
        });
    } else {
        // pieces between the knots of the shape's degree (shifted by 1/2 for even degrees)
        const double xs[3] = {x0[0] - p.koff, x0[1] - p.koff, x0[2] - p.koff};
        o.nseg = for_each_segment(xs, beta, p.split != 0, [&](const Segment<double>& sg) {
            if (p.order == 2) push_piece_gauss_r<2, DIAG>(p, sg, x0, beta, vb, table, acc);
            else if (p.order == 3) push_piece_gauss_r<3, DIAG>(p, sg, x0, beta, vb, table, acc);
            else push_piece_gauss<DIAG>(p, sg, x0, beta, vb, table, acc);
        });
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        o.Pw[a] = Pn[a] + p.dt * (-p.q * acc.gphi[a] + p.q * acc.F[a]);
        o.xe[a] = wrap_pos(x0[a] + beta[a], (double)p.m.n[a]);
    }
    point_gather3(p, o.xe, table, 3, o.Ae);
#pragma unroll
    for (int a = 0; a < 3; ++a) o.vw[a] = (o.Pw[a] - p.q * o.Ae[a]) * p.inv_mass;
}

// The Algorithm 1 push for iterate vit, then either
//   (iterate)  the next iterate and its orbit current into Jnext, plus the e_v partial sums.
//              The next iterate is G(v^p); with p.accel, creeping particles are instead
//              appended to a list and solved locally by k_local (which also scatters them);
//   (commit)   x^{n+1}, P^{n+1}, v^{n+1} and (optionally) the particle diagnostics.
// Two resident blocks per SM (at most 128 registers, a few spills) hide more of the FP64
// pipe's latency than one block at 178 registers (measured: 5% less push time at 32^3); the
// diagnostics variant keeps one block, its larger state would spill far more.
template <int QUAD, bool COMMIT, bool DIAG>
__global__ void __launch_bounds__(THREADS, DIAG ? 1 : 2) k_push(StepParams p, const double* __restrict__ xi,
                                                  const double* __restrict__ v, const double* __restrict__ P,
                                                  const double* __restrict__ vit, const double* __restrict__ table,
                                                  double* __restrict__ vnew, double* __restrict__ Jnext,
                                                  double* __restrict__ xi_out, double* __restrict__ P_out,
                                                  int32_t* __restrict__ creep_list, int* __restrict__ creep_count,
                                                  uint8_t* __restrict__ creep_flag,
                                                  const uint8_t* __restrict__ slide, double* __restrict__ partials,
                                                  int* __restrict__ status) {
    __shared__ double sm[32];
    const int64_t np = p.np;
    double ev_num = 0.0, ev_den = 0.0, pieces_push = 0.0, pieces_scatter = 0.0;
    double k1 = 0.0, pwork = 0.0, ra_sq = 0.0, ra_max = 0.0, pu_max = 0.0;
    __shared__ int order[THREADS];
    __shared__ int wcount[THREADS / 32][PIECE_CLASSES];
    const int64_t nchunks = (np + THREADS - 1) / THREADS;
    // Chunks of THREADS consecutive particles; inside a chunk the particles are handed to the
    // threads in order of their (estimated) number of orbit pieces, so that the lanes of a
    // warp run the same number of piece iterations (a stable ordering: deterministic).
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t base = ch * THREADS;
        {
            const int64_t j = base + threadIdx.x;
            const int cls = j < np ? piece_class(p, xi, v, vit, j) : PIECE_CLASSES - 1;
            order[stable_class_rank(cls, wcount)] = threadIdx.x;
        }
        __syncthreads();
        const int64_t i = base + order[threadIdx.x];
        if (i < np) {
            double x0[3], vn[3], vi[3], Pn[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = xi[a * np + i];
                vn[a] = v[a * np + i];
                vi[a] = vit[a * np + i];
                Pn[a] = P[a * np + i];
            }
            PushAcc acc;
            PushOut o;
            push_eval<QUAD, DIAG>(p, x0, vn, Pn, vi, table, acc, o);
            if (o.nseg < 0) atomicOr(status, DEV_ERR_SEGMENTS);
            pieces_push += (double)o.nseg;
            if (!(isfinite(o.vw[0]) && isfinite(o.vw[1]) && isfinite(o.vw[2]))) atomicOr(status, DEV_ERR_NONFINITE);
            if constexpr (COMMIT) {
#pragma unroll
                for (int a = 0; a < 3; ++a) vnew[a * np + i] = o.vw[a];
            }
            if constexpr (!COMMIT) {
                double beta_it[3];
#pragma unroll
                for (int a = 0; a < 3; ++a) beta_it[a] = p.dt * 0.5 * (vi[a] + vn[a]) * p.invH[a];
                const double xk[3] = {x0[0] - p.koff, x0[1] - p.koff, x0[2] - p.koff};   // knot lattice
                // a particle solved locally earlier in this step keeps the local solve, so that
                // none alternates between it and the plain update
                // So does one whose change did not shrink below SLOW_RATIO of the previous one: its
                // own feedback is too strong for the outer iteration (orbits crossing a knot just
                // past the creeping range, once the force jumps at knots grow).  A contracting
                // outer loop shrinks field-driven changes far faster, so it flags almost none.
                bool slow = false;
                if (p.hist) {
                    double dn = 0.0, dold = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        dn = fmax(dn, fabs(o.vw[a] - vi[a]));
                        dold = fmax(dold, fabs(vi[a] - vnew[a * np + i]));   // v^p - v^{p-1}
                    }
                    const double spd = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
                    slow = dn > SLOW_RATIO * dold && dn > p.slow_floor * spd;
                }
                const bool creep = p.accel && (is_creeping(xk, beta_it) || (slide[i] & SLIDE_CREPT) || slow);
                if (creep_flag) creep_flag[i] = creep ? 1 : 0;   // deterministic mode: k_local walks the flags
                if (creep) {
#pragma unroll
                    for (int a = 0; a < 3; ++a) vnew[a * np + i] = o.vw[a];   // G(v^p): the local solve starts there
                    if (!creep_flag) {
                        int k = atomicAdd(creep_count, 1);   // k_local solves it and adds its e_v terms
                        creep_list[k] = (int32_t)i;
                    }
                } else {
                    double wv[3], bet2[3], dnum = 0.0, dden = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vnew[a * np + i] = o.vw[a];
                        const double d = o.vw[a] - vi[a];   // change of the iterate, v^{p+1} - v^p
                        dnum += d * d;
                        dden += o.vw[a] * o.vw[a];
                        const double vb2 = 0.5 * (o.vw[a] + vn[a]);
                        bet2[a] = p.dt * vb2 * p.invH[a];
                        wv[a] = p.q_dV * vb2;
                    }
                    ev_num += dnum;
                    ev_den += dden;
                    int ns = scatter_orbit<QUAD>(p, x0, bet2, wv, Jnext);
                    if (ns < 0) atomicOr(status, DEV_ERR_SEGMENTS);
                    pieces_scatter += (double)ns;
                }
            } else {
                // components sliding onto a knot (set by k_local): the orbit lands on the knot,
                // v^{n+1}_a is the iterate itself and P_a follows from v = (P - q A_h(x)) / m
                const uint8_t sb = slide ? slide[i] : 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    if (sb & (1u << a)) {
                        o.vw[a] = vi[a];
                        o.Pw[a] = p.mass * o.vw[a] + p.q * o.Ae[a];
                        vnew[a * np + i] = o.vw[a];
                    }
                    xi_out[a * np + i] = o.xe[a];
                    P_out[a * np + i] = o.Pw[a];
                    // the residual of the accepted iterate itself, ||G(v*) - v*||
                    const double d = o.vw[a] - vi[a];
                    ev_num += d * d;
                    ev_den += o.vw[a] * o.vw[a];
                }
                if constexpr (DIAG) {
                    double As[3], vb[3];
                    point_gather3(p, x0, table, 0, As);                       // A_h^n(x^n)
                    double ra2 = 0.0;
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        vb[a] = 0.5 * (vi[a] + vn[a]);
                        double ra = o.Ae[a] - As[a] - p.dt * (acc.Ubar[a] + acc.DAv[a]);   // Eq. (RA-test)
                        ra2 += ra * ra;
                        ra_max = fmax(ra_max, fabs(ra));
                        pwork += p.q * vb[a] * (-acc.gphi[a] - acc.Ubar[a]);                // q vbar . Ebar
                        k1 += 0.5 * p.mass * o.vw[a] * o.vw[a];
                    }
                    ra_sq += ra2;
                    pu_max = fmax(pu_max, fabs(acc.pu - 1.0));
                }
            }
        }
        __syncthreads();   // order[] is rewritten by the next chunk
    }
    write_partial<double>(partials, S_EV_NUM, ev_num, sm, false);
    write_partial<double>(partials, S_EV_DEN, ev_den, sm, false);
    if constexpr (!COMMIT) {
        write_partial<double>(partials, S_PIECES_PUSH, pieces_push, sm, false);
        write_partial<double>(partials, S_PIECES_SCATTER, pieces_scatter, sm, false);
    } else if constexpr (DIAG) {
        write_partial<double>(partials, S_K1, k1, sm, false);
        write_partial<double>(partials, S_PWORK, pwork, sm, false);
        write_partial<double>(partials, S_RA_SQ, ra_sq, sm, false);
        write_partial<double>(partials, S_RA_MAX, ra_max, sm, true);
        write_partial<double>(partials, S_PU_MAX, pu_max, sm, true);
    }
}

// Particle-local solve of v = G_i(v) with the iteration's fields fixed, for the creeping
// particles listed by k_push (§4.8 allows any converged solver).  Per component of
// g(u) = G_i(u) - u, starting from (v^p, G(v^p)): clamped secant steps while each one at
// least halves |g| (a nearby root is found first); otherwise steps u + f g with f = 2, 4,
// 8, ... (g is continuous and G bounded, so g changes sign that way: a particle that barely
// crosses a knot can have no root near its iterate).  Inside a bracket the new point replaces
// the end of its sign:
//  - a bracket holding the velocity that lands the orbit exactly on a knot is first split
//    there: the force weight of the path beyond a knot makes G steep just past it, so g is
//    smooth only between landings;
//  - inside one knot-free piece past a crossing (landing beta_L), G in cells is close to
//    A + B beta_L / beta; the step solves beta = A + B beta_L / beta exactly for the line
//    through the two ends (a quadratic), elsewhere it is the regula falsi point;
//  - the components share each evaluation, so another component's move can leave a bracket
//    stale, and regula falsi can stagnate: a bracket whose same end is replaced twice running
//    is released for a secant step.
// At most LOCAL_STEPS push evaluations, stopping once one evaluation has every component's
// residual below LOCAL_TOL times the particle's speed; the evaluation with the smallest
// largest-component residual is kept whole (the components are coupled).  A particle solved
// here keeps the local solve for the rest of the step (SLIDE_CREPT), so that none alternates
// between it and the plain update.  Sliding (sticky for the rest of the step once detected,
// so that the outer iteration cannot cycle between pinned and free): a component starting
// within D_KNOT of a knot (signed distance d) whose two sides, probed SLIDE_PROBE short of
// the landing and max(SLIDE_PROBE, SLIDE_FAR |d|) past it, both push onto the knot has no
// root that double precision resolves; it lands exactly on the knot (the Filippov solution)
// and the commit push sets v^{n+1}_a to it with P_a from the canonical relation.  The energy
// identities hold to the size of vbar_a = d H / dt < D_KNOT H / dt.  The plain image G(v^p)
// is saved in gsave (diagnostics), then the orbit current of the result is scattered.
template <int QUAD>
__global__ void __launch_bounds__(THREADS) k_local(StepParams p, const double* __restrict__ xi,
                                                   const double* __restrict__ v, const double* __restrict__ P,
                                                   const double* __restrict__ vit, const double* __restrict__ table,
                                                   double* __restrict__ vnew, double* __restrict__ gsave,
                                                   double* __restrict__ Jnext, const int32_t* __restrict__ creep_list,
                                                   const int* __restrict__ creep_count,
                                                   const uint8_t* __restrict__ creep_flag, uint8_t* __restrict__ slide,
                                                   int* __restrict__ queue_head, double* __restrict__ partials,
                                                   int* __restrict__ status) {
    __shared__ double sm[32];
    const int64_t np = p.np;
    // The creeping particles: a list in arrival order, taken from a shared queue by whichever
    // lane is free; or (deterministic mode) flags in index order, each thread walking its own
    // fixed stride, so that the assignment (and every partial sum) is reproducible.
    const int64_t count = creep_flag ? np : (int64_t)*creep_count;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    int64_t next_static = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double ev_num = 0.0, ev_den = 0.0;
    // One particle's solve is a sequence of push evaluations: sliding probes (phase 0: just
    // short of the knot, phase 1: just past it, per probed axis), the first evaluation
    // (phase 2), then up to LOCAL_STEPS - 1 iteration steps (phase 3).  Every round, each lane
    // with a particle makes its next evaluation together with the others, and a lane whose
    // particle is done takes a new one: the warp's evaluations stay full even when particles
    // need very different numbers of them.
    bool active = false, exhausted = false;
    int64_t i = 0;
    int phase = 0, paxis = 0, nstep = 0;
    double x0[3], vn[3], Pn[3], u0[3], r0[3], u1[3], r1[3], bu[3];
    double ua[3], ga[3], ub[3], gb[3], side[3], fac[3], uland[3], dk[3], ue[3], blim[3];
    bool brk[3], secok[3], sl[3], probe[3];
    int nrep[3];
    double tol = 0.0, spd = 0.0, gm = 0.0, brs = 0.0;
    double nsolve = 0.0, neval = 0.0, nfail = 0.0, nfail_free = 0.0;
    while (true) {
        if (!active && !exhausted) {
            int64_t k = -1;
            if (creep_flag) {
                while (next_static < count && !creep_flag[next_static]) next_static += T;
                if (next_static < count) {
                    k = next_static;
                    next_static += T;
                }
            } else {
                const int q = atomicAdd(queue_head, 1);
                k = q < count ? q : -1;
            }
            if (k < 0) {
                exhausted = true;
            } else {
                i = creep_flag ? k : (int64_t)creep_list[k];
                double nrm = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    x0[a] = xi[a * np + i];
                    vn[a] = v[a * np + i];
                    Pn[a] = P[a * np + i];
                    u0[a] = vit[a * np + i];
                    u1[a] = vnew[a * np + i];          // G(v^p) from k_push
                    gsave[a * np + i] = u1[a];
                    r0[a] = u1[a] - u0[a];
                    nrm += u0[a] * u0[a];
                    blim[a] = fabs(p.dt * 0.5 / p.H[a] * (u0[a] + vn[a])) + BETA_TRIAL;   // trial-orbit bound
                    dk[a] = rint(x0[a] - p.koff) - (x0[a] - p.koff);   // signed distance to the nearest knot
                    uland[a] = 2.0 * dk[a] * p.H[a] / p.dt - vn[a];
                    sl[a] = (slide[i] >> a) & 1u;       // pinned earlier in this step: stays pinned
                    probe[a] = !sl[a] && fabs(dk[a]) < D_KNOT;
                }
                spd = fmax(sqrt(nrm), 1e-300);
                tol = LOCAL_TOL * spd;
                paxis = 0;
                while (paxis < 3 && !probe[paxis]) ++paxis;
                phase = paxis < 3 ? 0 : 2;
                if (phase == 2) {
#pragma unroll
                    for (int a = 0; a < 3; ++a)
                        if (sl[a]) u1[a] = uland[a];
                }
                nstep = 0;
                active = true;
            }
        }
        if (!__any_sync(0xffffffffu, active)) break;
        // the evaluation point of this round
        if (active) {
            if (phase <= 1) {
                // Sliding probes: a component starting within D_KNOT of a knot (signed distance
                // d) is tested SLIDE_PROBE short of landing on it and max(SLIDE_PROBE,
                // SLIDE_FAR |d|) past it, where the path beyond the knot carries most of the
                // orbit average; if both sides push onto the knot, the root lies within that
                // hair, unresolved in double precision, and the component lands on the knot.
#pragma unroll
                for (int a = 0; a < 3; ++a) ue[a] = u1[a];
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (a == paxis) {
                        const double d = dk[a], far = fmax(SLIDE_PROBE, SLIDE_FAR * fabs(d));
                        ue[a] = phase == 0 ? 2.0 * (d - (d > 0.0 ? SLIDE_PROBE : far)) * p.H[a] / p.dt - vn[a]
                                           : 2.0 * (d + (d > 0.0 ? far : SLIDE_PROBE)) * p.H[a] / p.dt - vn[a];
                    }
            } else if (phase == 2) {
#pragma unroll
                for (int a = 0; a < 3; ++a) ue[a] = u1[a];
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double c = p.dt * 0.5 / p.H[a];   // beta = c (u + v^n), in cells
                    const double xk = x0[a] - p.koff;        // start on the knot lattice
                    double fp = ub[a] - gb[a] * (ub[a] - ua[a]) / (gb[a] - ga[a]);
                    {
                        // Both ends past the same last knot (landing beta_L): on that knot-free
                        // piece the image G in cells is close to A + B w, w = beta_L / beta, steep
                        // near the knot and flat far past it; solve beta = A + B w exactly for the
                        // line through the two ends (D beta^2 - c1 beta - e = 0, root in bracket).
                        const double ba = c * (ua[a] + vn[a]), bb = c * (ub[a] + vn[a]);
                        const double la = ba > 0.0 ? floor(xk + ba) - xk : ceil(xk + ba) - xk;
                        const double lb = bb > 0.0 ? floor(xk + bb) - xk : ceil(xk + bb) - xk;
                        const double Ga = c * ga[a] + ba, Gb = c * gb[a] + bb;
                        const double wa = la / ba, wb = la / bb;
                        const double D = wb - wa;
                        const double c1 = Ga * D - (Gb - Ga) * wa;
                        const double e = (Gb - Ga) * la;
                        const double disc = c1 * c1 + 4.0 * D * e;
                        const double qq = 0.5 * (c1 + copysign(sqrt(fmax(disc, 0.0)), c1));
                        const double x1 = qq / D, x2 = -e / qq;
                        const double bl = fmin(ba, bb), bh = fmax(ba, bb);
                        const bool in1 = x1 > bl && x1 < bh, in2 = x2 > bl && x2 < bh;
                        const double fpm = 2.0 * (in1 ? x1 : x2) * p.H[a] / p.dt - vn[a];
                        if (la == lb && la != 0.0 && la * ba > 0.0 && la * bb > 0.0 && disc >= 0.0 && (in1 || in2) &&
                            isfinite(fpm))
                            fp = fpm;
                    }
                    double sec = -(u1[a] - u0[a]) / (r1[a] - r0[a]);
                    sec = isfinite(sec) ? fmin(fmax(sec, -OMEGA_MAX), OMEGA_MAX) : 1.0;
                    // the knot landing strictly inside the bracket (the highest one, if several)
                    const double lo = fmin(ua[a], ub[a]), hi = fmax(ua[a], ub[a]);
                    const double blo = c * (lo + vn[a]), bhi = c * (hi + vn[a]);
                    const double bland = (ceil(xk + bhi) - 1.0) - xk;
                    const double usplit = 2.0 * bland * p.H[a] / p.dt - vn[a];
                    if (sl[a]) {
                        ue[a] = uland[a];                    // pinned: lands on the knot
                    } else if (brk[a] && bland > blo && usplit > lo && usplit < hi) {
                        ue[a] = usplit;                      // split the bracket where G kinks
                    } else if (brk[a] && isfinite(fp)) {
                        ue[a] = fp;                          // bracketed step
                    } else if (!brk[a] && !secok[a]) {
                        ue[a] = u1[a] + fac[a] * r1[a];      // grow along g until g changes sign
                        fac[a] *= 2.0;
                    } else {
                        ue[a] = u1[a] + sec * r1[a];         // secant while it converges
                    }
                    // trial orbits stay within BETA_TRIAL cells beyond the iterate's own orbit, per
                    // axis (the growing steps along g would otherwise run past any neighbourhood
                    // of the root)
                    ue[a] = fmin(fmax(ue[a], -blim[a] / c - vn[a]), blim[a] / c - vn[a]);
                }
            }
        }
        PushAcc acc;
        PushOut o;
        if (active) {
            push_eval<QUAD, false>(p, x0, vn, Pn, ue, table, acc, o);
            if (phase >= 2 && o.nseg < 0) atomicOr(status, DEV_ERR_SEGMENTS);
            neval += 1.0;
        }
        if (!active) continue;
        bool done = false;
        if (phase == 0) {
            gm = o.vw[paxis] - ue[paxis];
            phase = 1;
        } else if (phase == 1) {
            const double gp = o.vw[paxis] - ue[paxis];
            sl[paxis] = gm > 0.0 && gp < 0.0;
            ++paxis;
            while (paxis < 3 && !probe[paxis]) ++paxis;
            if (paxis < 3) {
                phase = 0;
            } else {
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    if (sl[a]) u1[a] = uland[a];
                phase = 2;
            }
        } else if (phase == 2) {
            double m0 = 0.0, m1 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                r1[a] = sl[a] ? 0.0 : o.vw[a] - u1[a];
                if (sl[a]) r0[a] = 0.0;
                m0 = fmax(m0, fabs(r0[a]));
                m1 = fmax(m1, fabs(r1[a]));
                brk[a] = !sl[a] && r0[a] * r1[a] < 0.0;
                ua[a] = u0[a];
                ga[a] = r0[a];
                ub[a] = u1[a];
                gb[a] = r1[a];
                side[a] = 0.0;
                secok[a] = fabs(r1[a]) <= 0.5 * fabs(r0[a]);
                fac[a] = 2.0;
                nrep[a] = 0;
            }
            // the best evaluation so far, whole (the components are coupled): the smallest
            // largest-component |g|; pinned components land on their knot
            const bool take1 = m1 < m0;
#pragma unroll
            for (int a = 0; a < 3; ++a) bu[a] = sl[a] ? uland[a] : (take1 ? u1[a] : u0[a]);
            brs = fmin(m0, m1);
            phase = 3;
            done = nstep >= LOCAL_STEPS - 1 || brs <= tol;
        } else {
            double r2v[3], m2 = 0.0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                r2v[a] = sl[a] ? 0.0 : o.vw[a] - ue[a];
                m2 = fmax(m2, fabs(r2v[a]));
            }
            if (m2 < brs) {
                brs = m2;
#pragma unroll
                for (int a = 0; a < 3; ++a) bu[a] = ue[a];
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double r2 = r2v[a];
                secok[a] = secok[a] && fabs(r2) <= 0.5 * fabs(r1[a]);
                if (brk[a]) {
                    if (r2 * gb[a] > 0.0) {            // replaces the b end
                        nrep[a] = side[a] > 0.0 ? nrep[a] + 1 : 1;
                        ub[a] = ue[a];
                        gb[a] = r2;
                        side[a] = 1.0;
                    } else {                           // replaces the a end
                        nrep[a] = side[a] < 0.0 ? nrep[a] + 1 : 1;
                        ua[a] = ue[a];
                        ga[a] = r2;
                        side[a] = -1.0;
                    }
                    // the same end replaced twice running: the kept end is stale (its g was
                    // taken before the other components moved) or regula falsi stagnates;
                    // released, the next step is a secant one from two fresh points
                    if (nrep[a] >= 2) {
                        brk[a] = false;
                        secok[a] = true;
                        nrep[a] = 0;
                        side[a] = 0.0;
                    }
                } else if (!sl[a] && r2 * r1[a] < 0.0) {
                    brk[a] = true;
                    ua[a] = u1[a];
                    ga[a] = r1[a];
                    ub[a] = ue[a];
                    gb[a] = r2;
                }
                u0[a] = u1[a];
                r0[a] = r1[a];
                u1[a] = ue[a];
                r1[a] = r2;
            }
            ++nstep;
            done = nstep >= LOCAL_STEPS - 1 || brs <= tol;
        }
        if (!done) continue;
        // the particle's solve is over: its best iterate, sliding marks, e_v terms and current.
        // A solve that ends above the tolerance on the landing of its nearest knot, or that
        // fails (best residual above FAIL_RES of the speed) with a component starting within
        // D_FALLBACK of a knot: that root lies in the hair past the knot that double precision
        // (or the steps) did not resolve, and the component slides onto the knot.  Its energy
        // defect is then bounded by vbar_a = d H / dt times its residual, where it would
        // otherwise be the whole velocity times that residual; below FAIL_RES the residual
        // itself costs less.
        {
            const bool failed = brs > FAIL_RES * spd;
            bool pinned = false;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if ((brs > tol && bu[a] == uland[a]) || (failed && fabs(dk[a]) < D_FALLBACK)) sl[a] = true;
                pinned = pinned || (failed && fabs(dk[a]) < D_FALLBACK);
            }
            nfail += failed ? 1.0 : 0.0;
            nfail_free += (failed && !pinned) ? 1.0 : 0.0;
        }
        uint8_t sb = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (sl[a]) {
                bu[a] = uland[a];
                sb |= (uint8_t)(1u << a);
            }
        slide[i] = sb | SLIDE_CREPT;
        double wv[3], bet2[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (!isfinite(bu[a])) atomicOr(status, DEV_ERR_NONFINITE);
            const double d = bu[a] - vit[a * np + i];
            ev_num += d * d;
            ev_den += bu[a] * bu[a];
            vnew[a * np + i] = bu[a];
            const double vb2 = 0.5 * (bu[a] + vn[a]);
            bet2[a] = p.dt * vb2 * p.invH[a];
            wv[a] = p.q_dV * vb2;
        }
        if (scatter_orbit<QUAD>(p, x0, bet2, wv, Jnext) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
        nsolve += 1.0;
        active = false;
    }
    write_partial<double>(partials, S_EVL_NUM, ev_num, sm, false);
    write_partial<double>(partials, S_EVL_DEN, ev_den, sm, false);
    write_partial<double>(partials, S_LOCAL_SOLVES, nsolve, sm, false);
    write_partial<double>(partials, S_LOCAL_EVALS, neval, sm, false);
    write_partial<double>(partials, S_LOCAL_FAILED, nfail, sm, false);
    write_partial<double>(partials, S_LOCAL_FAILED_FREE, nfail_free, sm, false);
}

__global__ void k_kinetic(StepParams p, const double* __restrict__ v, double* __restrict__ partials) {
    __shared__ double sm[32];
    const int64_t np = p.np;
    double k = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        double a = v[i], b = v[np + i], c = v[2 * np + i];
        k += 0.5 * p.mass * (a * a + b * b + c * c);
    }
    write_partial<double>(partials, S_K, k, sm, false);
}

// ---- counting sort by cell of x^n -------------------------------------------------------

__global__ void k_sort_keys(StepParams p, const double* __restrict__ xi, int32_t* __restrict__ key,
                            int32_t* __restrict__ count) {
    const int64_t np = p.np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int c0 = min(max((int)floor(xi[i]), 0), p.m.n[0] - 1);
        int c1 = min(max((int)floor(xi[np + i]), 0), p.m.n[1] - 1);
        int c2 = min(max((int)floor(xi[2 * np + i]), 0), p.m.n[2] - 1);
        int32_t k = (int32_t)node_index(c0, c1, c2, p.m);
        key[i] = k;
        atomicAdd(count + k, 1);
    }
}

// Exclusive scan of n ints in blocks of 1024 (phase 1: local scan and block totals).
__global__ void k_scan_local(const int32_t* __restrict__ in, int32_t* __restrict__ out, int32_t* __restrict__ totals,
                             int64_t n) {
    __shared__ int32_t s[1024];
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    int32_t v = i < n ? in[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        int32_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += t;
        __syncthreads();
    }
    if (i < n) out[i] = s[threadIdx.x] - v;
    if (threadIdx.x == 1023) totals[blockIdx.x] = s[1023];
}

// Phase 2: one block scans the block totals sequentially in chunks of 1024.
__global__ void k_scan_totals(int32_t* __restrict__ totals, int nb) {
    __shared__ int32_t s[1024];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        int32_t v = i < nb ? totals[i] : 0;
        s[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            int32_t t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
            __syncthreads();
            s[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < nb) totals[i] = carry + s[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += s[1023];
        __syncthreads();
    }
}

__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ totals, int64_t n) {
    int64_t i = blockIdx.x * 1024LL + threadIdx.x;
    if (i < n) out[i] += totals[blockIdx.x];
}

// Place particle i at offset[key] + (arrival order within its cell) in the destination arrays.
__global__ void k_sort_scatter(StepParams p, const int32_t* __restrict__ key, const int32_t* __restrict__ offset,
                               int32_t* __restrict__ cursor, const double* __restrict__ xi, const double* __restrict__ v,
                               const double* __restrict__ P, const double* __restrict__ vprev,
                               const int64_t* __restrict__ id, double* __restrict__ xi_d, double* __restrict__ v_d,
                               double* __restrict__ P_d, double* __restrict__ vprev_d, int64_t* __restrict__ id_d) {
    const int64_t np = p.np;
    const int lane = threadIdx.x & 31;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = key[i];
        // the lanes of a warp with the same cell take consecutive places with one atomic (the
        // particles are nearly sorted already, so a warp holds one or two cells)
        const unsigned act = __activemask();
        const unsigned peers = __match_any_sync(act, k);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (lane == leader) first = atomicAdd(cursor + k, __popc(peers));
        first = __shfl_sync(peers, first, leader);
        const int64_t pos = (int64_t)offset[k] + first + __popc(peers & ((1u << lane) - 1u));
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi_d[a * np + pos] = xi[a * np + i];
            v_d[a * np + pos] = v[a * np + i];
            P_d[a * np + pos] = P[a * np + i];
            vprev_d[a * np + pos] = vprev[a * np + i];
        }
        id_d[pos] = id[i];
    }
}

// ---- stable LSD radix sort of the cell keys (deterministic mode) ---------------------------
//
// 8-bit digits; each pass counts the digits of every tile of RS_TILE keys, scans the counts
// in digit-major order (so tile b's keys of digit d go after those of every earlier tile),
// and scatters each tile in index order, ranking equal digits within a warp by
// __match_any_sync.  Every pass is stable, so the result is ordered by key and, among equal
// keys, by the previous order: a deterministic permutation.

constexpr int RS_RADIX = 256, RS_ITEMS = 8, RS_TILE = THREADS * RS_ITEMS;
static_assert(THREADS == RS_RADIX, "one thread per digit in the scatter's bookkeeping");

__global__ void k_rs_hist(const int32_t* __restrict__ key, int64_t n, int shift, int ntiles,
                          int32_t* __restrict__ hist) {
    __shared__ int32_t cnt[RS_RADIX];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[(key[i] >> shift) & (RS_RADIX - 1)], 1);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rs_scatter(const int32_t* __restrict__ key_in, const int32_t* __restrict__ val_in, int64_t n,
                             int shift, int ntiles, const int32_t* __restrict__ offs, int32_t* __restrict__ key_out,
                             int32_t* __restrict__ val_out) {
    __shared__ int32_t run[RS_RADIX];
    __shared__ int32_t wc[THREADS / 32][RS_RADIX];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    run[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
#pragma unroll
    for (int v = 0; v < THREADS / 32; ++v) wc[v][tid] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int r = 0; r < RS_ITEMS; ++r) {
        const int64_t i = base + r * THREADS + tid;
        const bool valid = i < n;
        const int32_t k = valid ? key_in[i] : 0;
        const int d = valid ? (k >> shift) & (RS_RADIX - 1) : RS_RADIX + lane;   // invalid lanes: own groups
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wc[w][d] = __popc(peers);
        __syncthreads();
        int pos = 0;
        if (valid) {
            pos = run[d] + rank;
            for (int v = 0; v < w; ++v) pos += wc[v][d];
        }
        __syncthreads();
        int add = 0;
#pragma unroll
        for (int v = 0; v < THREADS / 32; ++v) {
            add += wc[v][tid];
            wc[v][tid] = 0;
        }
        run[tid] += add;
        __syncthreads();
        if (valid) {
            key_out[pos] = k;
            val_out[pos] = val_in[i];
        }
    }
}

__global__ void k_iota(int64_t n, int32_t* __restrict__ a) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

// Destination j takes particle perm[j].
__global__ void k_sort_gather(StepParams p, const int32_t* __restrict__ perm, const double* __restrict__ xi,
                              const double* __restrict__ v, const double* __restrict__ P,
                              const double* __restrict__ vprev, const int64_t* __restrict__ id,
                              double* __restrict__ xi_d, double* __restrict__ v_d, double* __restrict__ P_d,
                              double* __restrict__ vprev_d, int64_t* __restrict__ id_d) {
    const int64_t np = p.np;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < np; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = perm[j];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xi_d[a * np + j] = xi[a * np + i];
            v_d[a * np + j] = v[a * np + i];
            P_d[a * np + j] = P[a * np + i];
            vprev_d[a * np + j] = vprev[a * np + i];
        }
        id_d[j] = id[i];
    }
}

// dst[c, id[i]] = scale_c * src[c, i]  (device order -> caller order)
__global__ void k_unpermute(int64_t np, const int64_t* __restrict__ id, const double* __restrict__ src,
                            double* __restrict__ dst, double s0, double s1, double s2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = id[i];
        dst[j] = s0 * src[i];
        dst[np + j] = s1 * src[np + i];
        dst[2 * np + j] = s2 * src[2 * np + i];
    }
}

// dst[c, i] = scale_c * src[c, id[i]]  (caller order -> device order)
__global__ void k_permute_in(int64_t np, const int64_t* __restrict__ id, const double* __restrict__ src,
                             double* __restrict__ dst, double s0, double s1, double s2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int64_t j = id[i];
        dst[i] = s0 * src[j];
        dst[np + i] = s1 * src[np + j];
        dst[2 * np + i] = s2 * src[2 * np + j];
    }
}

}  // namespace

StepParams make_params(const Ctx& c) {
    StepParams p;
    p.m = c.m;
    for (int a = 0; a < 3; ++a) {
        p.H[a] = c.H[a];
        p.invH[a] = c.invH[a];
    }
    p.dt = c.cfg.dt;
    p.q = c.q;
    p.mass = c.mass;
    p.inv_mass = 1.0 / c.mass;
    p.q_dV = c.q / c.dV;
    p.np = c.np;
    p.split = c.cfg.split_orbit_at_knots;
    p.nq = c.cfg.nq;
    p.accel = c.cfg.picard_accel;
    p.hist = 0;
    p.slow_floor = c.run.after32 ? SLOW_FLOOR_AFTER32 : SLOW_FLOOR;
    p.order = c.cfg.shape_order;
    p.koff = (c.cfg.shape_order % 2 == 0) ? 0.5 : 0.0;
    p.det = c.cfg.deterministic;
    p.acc = ExactAcc{c.acc_hi, c.acc_lo, c.inv_u_J, c.dev_status};
    return p;
}

int local_blocks(const Ctx& c) { return std::max(1, std::min(particle_blocks(c), c.sms * 2)); }

int particle_blocks(const Ctx& c) {
    int64_t b = (c.np + THREADS - 1) / THREADS;
    int64_t cap = (int64_t)c.sms * c.push_bps;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

void launch_init_positions(Ctx& c, const double* x_dev) {
    StepParams p = make_params(c);
    k_init_positions<<<particle_blocks(c), THREADS, 0, c.stream>>>(p, x_dev, c.xi, c.id);
    ++c.launches;
}

void launch_set_positions(Ctx& c, const double* src_dev) {
    k_set_positions<<<particle_blocks(c), THREADS, 0, c.stream>>>(make_params(c), c.id, src_dev, c.xi);
    ++c.launches;
}

void launch_point_deposit(Ctx& c) {
    StepParams p = make_params(c);
    p.acc.inv_u = c.inv_u_rho;
    k_point_deposit<<<particle_blocks(c), THREADS, 0, c.stream>>>(p, c.xi, c.rho0);
    ++c.launches;
    if (c.cfg.deterministic) launch_exact_finish(c, c.rho0, c.m.ncell, c.inv_u_rho);
}

void launch_first_scatter(Ctx& c, double* J, const double* v_iter_or_null) {
    StepParams p = make_params(c);
    int nb = particle_blocks(c);
    if (c.cfg.quadrature == PIC_QUAD_CLOSED)
        k_first_scatter<0><<<nb, THREADS, 0, c.stream>>>(p, c.xi, c.v, c.vprev, v_iter_or_null, c.vit, J, c.partials,
                                                         c.dev_status);
    else
        k_first_scatter<1><<<nb, THREADS, 0, c.stream>>>(p, c.xi, c.v, c.vprev, v_iter_or_null, c.vit, J, c.partials,
                                                         c.dev_status);
    ++c.launches;
    if (c.cfg.deterministic) launch_exact_finish(c, J, 3 * c.m.ncell, c.inv_u_J);
}

void launch_push(Ctx& c, const double* vit, double* vnew, double* Jnext, bool commit, bool diag) {
    StepParams p = make_params(c);
    p.hist = !commit && c.cfg.picard_accel && c.run.hist;
    int nb = particle_blocks(c);
    const bool det = c.cfg.deterministic && !commit;
    const bool closed = c.cfg.quadrature == PIC_QUAD_CLOSED;
    if (!commit) cudaMemsetAsync(c.creep_count, 0, 2 * sizeof(int), c.stream);   // count, k_local queue head
#define PIC_PUSH(Q, C, D)                                                                                        \
    k_push<Q, C, D><<<nb, THREADS, 0, c.stream>>>(p, c.xi, c.v, c.P, vit, c.table, vnew, Jnext, c.xi_new, c.P_new, \
                                                  c.creep_list, c.creep_count, det ? c.creep_flag : nullptr,  \
                                                  c.slide,                                                    \
                                                  c.partials, c.dev_status)
    if (!commit) {
        if (closed) PIC_PUSH(0, false, false);
        else PIC_PUSH(1, false, false);
    } else if (!diag) {
        if (closed) PIC_PUSH(0, true, false);
        else PIC_PUSH(1, true, false);
    } else {
        if (closed) PIC_PUSH(0, true, true);
        else PIC_PUSH(1, true, true);
    }
#undef PIC_PUSH
    ++c.launches;
    // in deterministic mode the exact current is rounded once all of its deposits are in
    if (det && Jnext && !c.cfg.picard_accel) launch_exact_finish(c, Jnext, 3 * c.m.ncell, c.inv_u_J);
}

void launch_local(Ctx& c, const double* vit, double* vnew, double* Jnext) {
    StepParams p = make_params(c);
    const bool det = c.cfg.deterministic != 0;
    const int lb = local_blocks(c);
    if (c.cfg.quadrature == PIC_QUAD_CLOSED)
        k_local<0><<<lb, THREADS, 0, c.stream>>>(p, c.xi, c.v, c.P, vit, c.table, vnew, c.gsave, Jnext, c.creep_list,
                                                 c.creep_count, det ? c.creep_flag : nullptr, c.slide,
                                                 c.creep_count + 1, c.partials, c.dev_status);
    else
        k_local<1><<<lb, THREADS, 0, c.stream>>>(p, c.xi, c.v, c.P, vit, c.table, vnew, c.gsave, Jnext, c.creep_list,
                                                 c.creep_count, det ? c.creep_flag : nullptr, c.slide,
                                                 c.creep_count + 1, c.partials, c.dev_status);
    ++c.launches;
    if (det && Jnext) launch_exact_finish(c, Jnext, 3 * c.m.ncell, c.inv_u_J);
}

void launch_kinetic(Ctx& c) {
    StepParams p = make_params(c);
    k_kinetic<<<particle_blocks(c), THREADS, 0, c.stream>>>(p, c.v, c.partials);
    ++c.launches;
}

// out[i] = (hi[i] 2^40 + lo[i]) u, then hi[i] = lo[i] = 0 for the next deposit (the
// deterministic mode's exact accumulators; see ExactAcc).
__global__ void k_exact_finish(int64_t n, long long* __restrict__ hi, long long* __restrict__ lo, double u,
                               double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = ((double)hi[i] * 0x1p40 + (double)lo[i]) * u;
        hi[i] = 0;
        lo[i] = 0;
    }
}

void launch_exact_finish(Ctx& c, double* out, int64_t n, double inv_u) {
    int64_t nb = (n + THREADS - 1) / THREADS;
    if (nb > (int64_t)c.sms * 8) nb = (int64_t)c.sms * 8;
    if (nb < 1) nb = 1;
    k_exact_finish<<<(int)nb, THREADS, 0, c.stream>>>(n, c.acc_hi, c.acc_lo, 1.0 / inv_u, out);
    ++c.launches;
}

int radix_tiles(int64_t np) { return (int)std::max<int64_t>(1, (np + RS_TILE - 1) / RS_TILE); }

// Stable radix sort of the cell keys; the particle arrays are then gathered in that order.
void launch_sort_stable(Ctx& c) {
    StepParams p = make_params(c);
    const int64_t N = c.m.ncell, np = c.np;
    const int nb = particle_blocks(c);
    cudaMemsetAsync(c.count, 0, sizeof(int32_t) * N, c.stream);
    k_sort_keys<<<nb, THREADS, 0, c.stream>>>(p, c.xi, c.rs_key[0], c.count);
    k_iota<<<nb, THREADS, 0, c.stream>>>(np, c.rs_val[0]);
    c.launches += 2;
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < N) ++bits;
    const int passes = std::max(1, (bits + 7) / 8);
    const int ntiles = radix_tiles(np);
    const int64_t nh = (int64_t)RS_RADIX * ntiles;
    const int nsb = (int)((nh + 1023) / 1024);
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = 8 * pass;
        k_rs_hist<<<ntiles, THREADS, 0, c.stream>>>(c.rs_key[cur], np, shift, ntiles, c.rs_hist);
        k_scan_local<<<nsb, 1024, 0, c.stream>>>(c.rs_hist, c.rs_offs, c.rs_scan_tmp, nh);
        k_scan_totals<<<1, 1024, 0, c.stream>>>(c.rs_scan_tmp, nsb);
        k_scan_add<<<nsb, 1024, 0, c.stream>>>(c.rs_offs, c.rs_scan_tmp, nh);
        k_rs_scatter<<<ntiles, THREADS, 0, c.stream>>>(c.rs_key[cur], c.rs_val[cur], np, shift, ntiles, c.rs_offs,
                                                        c.rs_key[cur ^ 1], c.rs_val[cur ^ 1]);
        c.launches += 5;
        cur ^= 1;
    }
    k_sort_gather<<<nb, THREADS, 0, c.stream>>>(p, c.rs_val[cur], c.xi, c.v, c.P, c.vprev, c.id, c.xi_new, c.vnew,
                                                c.P_new, c.vit, c.id_tmp);
    ++c.launches;
    std::swap(c.xi, c.xi_new);
    std::swap(c.v, c.vnew);
    std::swap(c.P, c.P_new);
    std::swap(c.vprev, c.vit);
    std::swap(c.id, c.id_tmp);
}

void launch_sort(Ctx& c) {
    if (c.cfg.deterministic) {
        launch_sort_stable(c);
        return;
    }
    StepParams p = make_params(c);
    const int64_t N = c.m.ncell;
    int nb = particle_blocks(c);
    cudaMemsetAsync(c.count, 0, sizeof(int32_t) * N, c.stream);
    cudaMemsetAsync(c.cursor, 0, sizeof(int32_t) * N, c.stream);
    k_sort_keys<<<nb, THREADS, 0, c.stream>>>(p, c.xi, c.key, c.count);
    ++c.launches;
    int nsb = (int)((N + 1023) / 1024);
    k_scan_local<<<nsb, 1024, 0, c.stream>>>(c.count, c.offset, c.scan_tmp, N);
    ++c.launches;
    k_scan_totals<<<1, 1024, 0, c.stream>>>(c.scan_tmp, nsb);
    ++c.launches;
    k_scan_add<<<nsb, 1024, 0, c.stream>>>(c.offset, c.scan_tmp, N);
    ++c.launches;
    // destinations: the free iterate/commit buffers of the step
    k_sort_scatter<<<nb, THREADS, 0, c.stream>>>(p, c.key, c.offset, c.cursor, c.xi, c.v, c.P, c.vprev, c.id,
                                                 c.xi_new, c.vnew, c.P_new, c.vit, c.id_tmp);
    ++c.launches;
    std::swap(c.xi, c.xi_new);
    std::swap(c.v, c.vnew);
    std::swap(c.P, c.P_new);
    std::swap(c.vprev, c.vit);
    std::swap(c.id, c.id_tmp);
}

// g[c, list[k]] = gsave[c, list[k]] for the particles solved locally in the last iteration.
__global__ void k_patch_local(int64_t np, const int32_t* __restrict__ list, const int* __restrict__ count,
                              const double* __restrict__ gsave, double* __restrict__ g) {
    const int n = *count;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const int64_t i = list[k];
        g[i] = gsave[i];
        g[np + i] = gsave[np + i];
        g[2 * np + i] = gsave[2 * np + i];
    }
}

void launch_patch_local(Ctx& c, double* g) {
    k_patch_local<<<std::max(1, c.sms), THREADS, 0, c.stream>>>(c.np, c.creep_list, c.creep_count, c.gsave, g);
    ++c.launches;
}

// dst[id[i]] = the sliding bits (components 0..2) of particle i (device order -> caller order).
__global__ void k_slide_out(int64_t np, const int64_t* __restrict__ id, const uint8_t* __restrict__ slide,
                            uint8_t* __restrict__ dst) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x)
        dst[id[i]] = slide[i] & 7u;
}

void launch_slide_out(Ctx& c, uint8_t* dst) {
    k_slide_out<<<particle_blocks(c), THREADS, 0, c.stream>>>(c.np, c.id, c.slide, dst);
    ++c.launches;
}

void launch_unpermute(Ctx& c, const double* src, double* dst, double s0, double s1, double s2) {
    k_unpermute<<<particle_blocks(c), THREADS, 0, c.stream>>>(c.np, c.id, src, dst, s0, s1, s2);
    ++c.launches;
}

void launch_permute_in(Ctx& c, const double* src, double* dst, double s0, double s1, double s2) {
    k_permute_in<<<particle_blocks(c), THREADS, 0, c.stream>>>(c.np, c.id, src, dst, s0, s1, s2);
    ++c.launches;
}

}  // namespace pic
