// Adjoint (reverse mode) of the implicit step and of the initial data (sm_103a, FP64).
//
// One step maps the level-n state s = (x, v, P, phi, psi, A, U, rho) to level n+1 through the
// accepted iterate v*, a fixed point of Algorithm 1's map, v* = G(v*; s), and the final sweep
// s' = F(v*, s) (§5.4), whose velocity output is G itself.  For a scalar L(s') with adjoint
// lambda' = dL/ds', the implicit-function theorem gives dL/ds = F_s^T (lambda' + mu e_v) with
// mu (the adjoint of v*) the solution of the transposed fixed point
//     mu = F_v*^T (lambda' + mu e_v),
// e_v placing mu on the velocity output.  Each application of F^T (a "sweep") is:
//   1. the particles' value pass: lambda_P' + lambda_v / m becomes the adjoint of the impulse,
//      which scatters onto the mesh adjoints of the gather table (grad phi^{n+1/2}, and A^n,
//      A^{n+1} through the transposed contraction of D_i A with vbar) and of A^{n+1} at the end
//      point (the point interpolant's transpose);
//   2. the mesh phase transposed: grad^T = -div, the Crank--Nicolson Helmholtz operator
//      I - a Delta_h is symmetric (one Chebyshev solve of the same schedule), continuity's
//      div^T = -grad; this gives the adjoints of phi^n, psi^n, A^n, U^n, rho^n and of J;
//   3. the particles' derivative pass: each particle's scalar
//         Phi = lam_gphibar . gphibar + lam_F . (D A)^T vbar + lam_Aend . A_h^{n+1}(x + beta)
//             + lam_x' . (x + beta) + sum_g lam_J[g] . J_g(particle)
//      is differentiated with respect to its start position and displacement beta by
//      forward-mode dual numbers through the same closed-form orbit integrals (dual.cuh), six
//      directions, with the mesh adjoints and fields held fixed.  beta = dt (v* + v^n) / (2 H)
//      gives the adjoints of v* and v^n.
// The transposed fixed point (I - K) mu = b0, g(mu) = K mu + b0 being step 3's adjoint of v*,
// is solved by restarted GMRES with right preconditioning.  The preconditioner is the transpose
// of the forward iteration's own splitting: a particle that the step solved locally (its
// slide byte's SLIDE_CREPT bit) gets its 3 x 3 block (I - B^T)^{-1}, B = dG_i / dv*_i with the
// fields fixed (from the same dual passes); every other particle gets the identity, as the plain
// Picard update treats it.  The stationary iteration with this splitting is the transposed
// linearisation of the forward solve, so its spectral radius is that of the forward iteration
// at the accepted step (below one, since the step converged), and the preconditioned operator's
// spectrum lies in a disc around 1 of that radius.  Within a restart cycle GMRES's residual is
// never above the stationary iteration's, and it is far below it where the forward iteration
// itself converged slowly.
//
// Sliding components (the step committed them by the sliding equations, §9 of the notes on the
// local solve): their iterate is the explicit landing velocity v*_a = 2 d_a H_a / dt - v^n_a,
// d_a the start's signed distance to its knot, their velocity output is v*_a itself and their
// momentum m v*_a + q A_h,a(x^{n+1}).  So they have no fixed-point equation (mu_a = 0, their
// rows and columns of B are dropped), their push impulse is unused (the adjoint of P^n_a is
// zero), the adjoint of their momentum reaches A_h at the end point and m v*_a, and the total
// adjoint nu_a of v*_a (direct, plus the orbit's g_a) goes to the start through d_a
// (d v*_a / d xi_a = -2 H_a / dt) and to v^n_a (-1).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "pic_internal.h"
#include "particle_common.cuh"
#include "dual.cuh"

namespace pic {
namespace {

struct AdjParams {
    StepParams p;
    double a, c_rho, c_J;     // CN constants: a = kappa^2 dt^2 / 4, dt^2 kappa^2 sigma_i / 2
    double sigma1, sigma2;
};

AdjParams adj_params(const Ctx& c) {
    AdjParams ap;
    ap.p = make_params(c);
    const double k2 = c.cfg.kappa * c.cfg.kappa, dt = c.cfg.dt;
    ap.a = 0.25 * k2 * dt * dt;
    ap.c_rho = 0.5 * dt * dt * k2 * c.cfg.sigma1;
    ap.c_J = 0.5 * dt * dt * k2 * c.cfg.sigma2;
    ap.sigma1 = c.cfg.sigma1;
    ap.sigma2 = c.cfg.sigma2;
    return ap;
}

__device__ __forceinline__ int64_t nshift(int64_t g, int dx, int dy, int dz, const MeshDims& m) {
    const int ix = (int)(g % m.n[0]);
    const int64_t t = g / m.n[0];
    const int iy = (int)(t % m.n[1]), iz = (int)(t / m.n[1]);
    return node_index(wrapi(ix + dx, m.n[0]), wrapi(iy + dy, m.n[1]), wrapi(iz + dz, m.n[2]), m);
}

// D_a f at node g (stride: distance between a field's consecutive node values in memory)
__device__ __forceinline__ double dcen_s(const double* __restrict__ f, int64_t stride, int64_t g, int a,
                                         const MeshDims& m, const double* invH) {
    const int64_t p = a == 0 ? nshift(g, 1, 0, 0, m) : (a == 1 ? nshift(g, 0, 1, 0, m) : nshift(g, 0, 0, 1, m));
    const int64_t q = a == 0 ? nshift(g, -1, 0, 0, m) : (a == 1 ? nshift(g, 0, -1, 0, m) : nshift(g, 0, 0, -1, m));
    return 0.5 * invH[a] * (f[stride * p] - f[stride * q]);
}

__device__ __forceinline__ double lap_s(const double* __restrict__ f, int64_t g, const MeshDims& m, const double* invH) {
    const double c = f[g];
    double s = 0.25 * invH[0] * invH[0] * (f[nshift(g, 2, 0, 0, m)] - 2.0 * c + f[nshift(g, -2, 0, 0, m)]);
    s += 0.25 * invH[1] * invH[1] * (f[nshift(g, 0, 2, 0, m)] - 2.0 * c + f[nshift(g, 0, -2, 0, m)]);
    s += 0.25 * invH[2] * invH[2] * (f[nshift(g, 0, 0, 2, m)] - 2.0 * c + f[nshift(g, 0, 0, -2, m)]);
    return s;
}

#define ADJ_LOOP(i, n) for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// ---- the particles' push, templated on the scalar type (double, or Dual for derivatives) -----
//
// The same formulas as the FP64 push (push_piece_fast, push_eval and scatter_closed): the
// orbit gather of grad phi, (D_i A)^T vbar contracted with vbar first, the end point's
// A_h^{n+1}, and the orbit weights of the current.  Positions are in cell units.

template <typename T>
__device__ __forceinline__ void push_piece_t(const StepParams& p, const Segment<T>& sg, const T beta[3], const T vb[3],
                                             const double* __restrict__ table, T gphi[3], T F[3]) {
    const PieceInts<T> I = piece_integrals(sg, beta, true);
    T W[8];
    weights_from_ints(I, W);
    int64_t g[8];
    Segment<double> sd;
    sd.cell[0] = sg.cell[0];
    sd.cell[1] = sg.cell[1];
    sd.cell[2] = sg.cell[2];
    segment_nodes8(sd, p.m, g);
    const T s = sg.s0, oms = T(1) - sg.s0, h = sg.h, hh2 = T(0.5) * sg.h * sg.h;
    T am[8], cc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const double* t = table + 12 * g[k];
        const T an = vb[0] * t[0] + vb[1] * t[1] + vb[2] * t[2];
        const T a1 = vb[0] * t[3] + vb[1] * t[4] + vb[2] * t[5];
        am[k] = oms * an + s * a1;
        cc[k] = a1 - an;
        gphi[0] += W[k] * t[6];
        gphi[1] += W[k] * t[7];
        gphi[2] += W[k] * t[8];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int pa = j == 0 ? 1 : 0, qa = j == 2 ? 1 : 2;
        const int sp = j == 0 ? 2 : 1, sq = j == 2 ? 2 : 4;
        const int sj = j == 0 ? 1 : (j == 1 ? 2 : 4);
        const T D00 = am[sj] - am[0], D10 = am[sp + sj] - am[sp];
        const T D01 = am[sq + sj] - am[sq], D11 = am[sp + sq + sj] - am[sp + sq];
        const T C00 = cc[sj] - cc[0], C10 = cc[sp + sj] - cc[sp];
        const T C01 = cc[sq + sj] - cc[sq], C11 = cc[sp + sq + sj] - cc[sp + sq];
        const T t0 = D00 * h + (D10 - D00) * I.S1[pa] + (D01 - D00) * I.S1[qa] + (D11 - D10 - D01 + D00) * I.S2[j];
        const T t1 = C00 * hh2 + (C10 - C00) * I.E1[pa] + (C01 - C00) * I.E1[qa] + (C11 - C10 - C01 + C00) * I.E2[j];
        F[j] += T(p.invH[j]) * (t0 + t1);
    }
}

// Wrap onto [0, n) as the forward push does (derivative 1).
template <typename T>
__device__ __forceinline__ T wrap_t(T x, double n) {
    T w = x < T(0) ? x + T(n) : (x >= T(n) ? x - T(n) : x);
    return w >= T(n) ? w - T(n) : w;
}

// A_h^{n+1} at a wrapped position (8 linear B-splines), table column block 3..5.
template <typename T>
__device__ __forceinline__ void point_A1_t(const StepParams& p, const T xq[3], const double* __restrict__ table, T out[3]) {
    int c[3];
    T r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const T f = floor(xq[a]);
        c[a] = (int)f;
        r[a] = xq[a] - f;
    }
    Segment<double> sd;
    sd.cell[0] = c[0];
    sd.cell[1] = c[1];
    sd.cell[2] = c[2];
    int64_t g[8];
    segment_nodes8(sd, p.m, g);
    out[0] = out[1] = out[2] = T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const T wx = (k & 1) ? r[0] : T(1) - r[0];
        const T wy = (k & 2) ? r[1] : T(1) - r[1];
        const T wz = (k & 4) ? r[2] : T(1) - r[2];
        const T w = wx * wy * wz;
        const double* t = table + 12 * g[k] + 3;
        out[0] += w * t[0];
        out[1] += w * t[1];
        out[2] += w * t[2];
    }
}

// ---- step 1: the particles' value pass (mesh adjoints of the gather table) ---------------------

// lam_tab per node: [A^n (3) | A^{n+1} (3) | grad phi^{n+1/2} (3)], 9 doubles, accumulated.
// The output adjoints of one particle component: lP1 (of P^{n+1}), lAe (of A_h^{n+1} at the end
// point), lg and lF (of the orbit gathers grad phi-bar and (D A)^T vbar).
__device__ __forceinline__ void out_adjoints(const StepParams& p, bool sl, double lv, double lP, double mu_c,
                                             double& lP1, double& lAe, double& lg, double& lF) {
    if (sl) {             // v1 = v*, P1 = m v* + q A_end: no impulse
        lP1 = lP;
        lAe = p.q * lP;
        lg = lF = 0.0;
    } else {              // v1 = (P1 - q A_end) / m, P1 = P + dt q (-gphibar + F)
        const double lv1 = lv + mu_c;
        lP1 = lP + lv1 * p.inv_mass;
        lAe = -p.q * p.inv_mass * lv1;
        lg = -p.dt * p.q * lP1;
        lF = p.dt * p.q * lP1;
    }
}

__global__ void k_adj_scatter(AdjParams ap, const double* __restrict__ xi, const double* __restrict__ v,
                              const double* __restrict__ vstar, const double* __restrict__ table,
                              const double* __restrict__ lam_P, const double* __restrict__ lam_v,
                              const double* __restrict__ mu, const uint8_t* __restrict__ slide,
                              double* __restrict__ lam_tab) {
    const StepParams& p = ap.p;
    const int64_t np = p.np;
    ADJ_LOOP(i, np) {
        double x0[3], beta[3], vb[3], lP1[3], lAe[3], lg[3], lF[3];
        const uint8_t sb = slide[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x0[a] = xi[a * np + i];
            vb[a] = 0.5 * (vstar[a * np + i] + v[a * np + i]);
            beta[a] = p.dt * vb[a] * p.invH[a];
            out_adjoints(p, (sb >> a) & 1u, lam_v[a * np + i], lam_P[a * np + i], mu[a * np + i], lP1[a], lAe[a], lg[a],
                         lF[a]);
        }
        // the end point's interpolant of A^{n+1}, transposed
        double xe[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) xe[a] = wrap_pos(x0[a] + beta[a], (double)p.m.n[a]);
        {
            int64_t g[8];
            double w[8];
            point_weights8(xe, p.m, g, w);
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) atomicAdd(lam_tab + 9 * g[k] + 3 + a, w[k] * lAe[a]);
        }
        // the orbit gather and D_i A, transposed piece by piece
        for_each_segment(x0, beta, true, [&](const Segment<double>& sg) {
            const PieceInts<double> I = piece_integrals(sg, beta, true);
            double W[8];
            weights_from_ints(I, W);
            int64_t g[8];
            segment_nodes8(sg, p.m, g);
            const double s = sg.s0, h = sg.h, hh2 = 0.5 * h * h;
            double lam_am[8] = {0, 0, 0, 0, 0, 0, 0, 0}, lam_cc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int pa = j == 0 ? 1 : 0, qa = j == 2 ? 1 : 2;
                const int sp = j == 0 ? 2 : 1, sq = j == 2 ? 2 : 4;
                const int sj = j == 0 ? 1 : (j == 1 ? 2 : 4);
                const double f = p.invH[j] * lF[j];
                // t0 = sum over transverse corners (a, b) of k0_ab (am[k_ab + sj] - am[k_ab])
                const double k0[4] = {h - I.S1[pa] - I.S1[qa] + I.S2[j], I.S1[pa] - I.S2[j], I.S1[qa] - I.S2[j], I.S2[j]};
                const double k1[4] = {hh2 - I.E1[pa] - I.E1[qa] + I.E2[j], I.E1[pa] - I.E2[j], I.E1[qa] - I.E2[j],
                                      I.E2[j]};
                const int kb[4] = {0, sp, sq, sp + sq};
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    lam_am[kb[c] + sj] += f * k0[c];
                    lam_am[kb[c]] -= f * k0[c];
                    lam_cc[kb[c] + sj] += f * k1[c];
                    lam_cc[kb[c]] -= f * k1[c];
                }
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const double lan = (1.0 - s) * lam_am[k] - lam_cc[k];   // am = (1-s) an + s a1, cc = a1 - an
                const double la1 = s * lam_am[k] + lam_cc[k];
                double* t = lam_tab + 9 * g[k];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    atomicAdd(t + a, vb[a] * lan);                  // an = A^n . vbar
                    atomicAdd(t + 3 + a, vb[a] * la1);              // a1 = A^{n+1} . vbar
                    atomicAdd(t + 6 + a, W[k] * lg[a]);             // gphibar = sum W grad phi
                }
            }
        });
    }
}

// ---- step 2: the mesh phase transposed -----------------------------------------------------------
//
// Inputs: lam_tab, and the level-(n+1) adjoints lF1 = [phi | A] (4 N), lW1 = [psi | U] (4 N),
// lrho1 (N).  t_f = lF1_f + (particles' adjoint of F^{n+1}_f) + (2/dt) lW1_f is the right-hand
// side of the adjoint Helmholtz solve (psi^{n+1} = 2 (phi^{n+1} - phi^n)/dt - psi^n);
// pn_f collects the particles' adjoint of F^n_f.  grad phi^{n+1/2} = grad (phi^n + phi^{n+1})/2
// gives -div(lam_gphi)/2 to both levels of phi.
__global__ void k_adj_mesh_rhs(AdjParams ap, const double* __restrict__ lam_tab, const double* __restrict__ lF1,
                               const double* __restrict__ lW1, double* __restrict__ t, double* __restrict__ pn) {
    const StepParams& p = ap.p;
    const int64_t N = p.m.ncell;
    ADJ_LOOP(g, N) {
        double ldiv = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) ldiv += dcen_s(lam_tab + 6 + a, 9, g, a, p.m, p.invH);
        const double lphi_half = -0.5 * ldiv;
        t[g] = lF1[g] + lphi_half + 2.0 / p.dt * lW1[g];
        pn[g] = lphi_half;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int64_t o = (1 + c) * N + g;
            t[o] = lF1[o] + lam_tab[9 * g + 3 + c] + 2.0 / p.dt * lW1[o];
            pn[o] = lam_tab[9 * g + c];
        }
    }
}

// After y = (I - a Delta_h)^{-1} t: the level-n adjoints and the adjoint of J.
__global__ void k_adj_mesh_out(AdjParams ap, const double* __restrict__ y, const double* __restrict__ pn,
                               const double* __restrict__ lW1, const double* __restrict__ lrho1,
                               double* __restrict__ lF0, double* __restrict__ lW0, double* __restrict__ lrho0,
                               double* __restrict__ lJ) {
    const StepParams& p = ap.p;
    const int64_t N = p.m.ncell;
    ADJ_LOOP(g, N) {
#pragma unroll
        for (int f = 0; f < 4; ++f) {
            const double* yf = y + f * N;
            lF0[f * N + g] = yf[g] + ap.a * lap_s(yf, g, p.m, p.invH) - 2.0 / p.dt * lW1[f * N + g] + pn[f * N + g];
            lW0[f * N + g] = p.dt * yf[g] - lW1[f * N + g];
        }
        // rho^{n+1/2} = (rho^n + rho^{n+1}) / 2 feeds phi's source with c_rho; rho^{n+1} = rho^n - dt div J
        lrho0[g] = lrho1[g] + ap.c_rho * y[g];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // lam_rho^{n+1} (total) = lrho1 + c_rho y_phi / 2 at the neighbours, then J's dt grad
            const int64_t pp = c == 0 ? nshift(g, 1, 0, 0, p.m) : (c == 1 ? nshift(g, 0, 1, 0, p.m) : nshift(g, 0, 0, 1, p.m));
            const int64_t qq = c == 0 ? nshift(g, -1, 0, 0, p.m) : (c == 1 ? nshift(g, 0, -1, 0, p.m) : nshift(g, 0, 0, -1, p.m));
            const double lr_p = lrho1[pp] + 0.5 * ap.c_rho * y[pp], lr_q = lrho1[qq] + 0.5 * ap.c_rho * y[qq];
            lJ[c * N + g] = ap.c_J * y[(1 + c) * N + g] + p.dt * 0.5 * p.invH[c] * (lr_p - lr_q);
        }
    }
}

// ---- step 3: the particles' derivative pass --------------------------------------------------------

// Phi of one particle for start x0 and displacement beta (cell units), with the scalar type T.
template <typename T>
__device__ __forceinline__ T particle_phi(const AdjParams& ap, const T x0[3], const T beta[3], const double lg[3],
                                          const double lF[3], const double lAe[3], const double lxe[3],
                                          const double* __restrict__ table, const double* __restrict__ lJ, T gphi[3],
                                          T F[3], T Ae[3]) {
    const StepParams& p = ap.p;
    const int64_t N = p.m.ncell;
    T vb[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vb[a] = beta[a] * T(p.H[a] / p.dt);
        gphi[a] = T(0);
        F[a] = T(0);
    }
    T phi = T(0);
    for_each_segment(x0, beta, true, [&](const Segment<T>& sg) {
        push_piece_t(p, sg, beta, vb, table, gphi, F);
        // this particle's orbit current q vbar Sbar / dV against the adjoint of J
        T I[8];
        weights_from_ints(piece_integrals(sg, beta, false), I);
        Segment<double> sd;
        sd.cell[0] = sg.cell[0];
        sd.cell[1] = sg.cell[1];
        sd.cell[2] = sg.cell[2];
        int64_t g[8];
        segment_nodes8(sd, p.m, g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const T s = vb[0] * lJ[g[k]] + vb[1] * lJ[N + g[k]] + vb[2] * lJ[2 * N + g[k]];
            phi += T(p.q_dV) * I[k] * s;
        }
    });
    T xe[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) xe[a] = wrap_t(x0[a] + beta[a], (double)p.m.n[a]);
    point_A1_t(p, xe, table, Ae);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        phi += T(lg[a]) * gphi[a] + T(lF[a]) * F[a] + T(lAe[a]) * Ae[a];
        phi += T(lxe[a]) * (x0[a] + beta[a]);
    }
    return phi;
}

// Per particle: the adjoints of the start position (lam_xi) and of v* (g = dt/(2H) dPhi/dbeta,
// which is also the adjoint of v^n), and the block B = dG_i/dv*_i (9, row-major) of the
// transposed solve's preconditioner (zero outside the particles the step solved locally).
// lam_xe: adjoint of the end position x^{n+1} in cell units.
__global__ void __launch_bounds__(THREADS) k_adj_derivs(AdjParams ap, const double* __restrict__ xi,
                                                        const double* __restrict__ v, const double* __restrict__ vstar,
                                                        const double* __restrict__ table, const double* __restrict__ lJ,
                                                        const double* __restrict__ lam_P, const double* __restrict__ lam_v,
                                                        const double* __restrict__ lam_xe, const double* __restrict__ mu,
                                                        const uint8_t* __restrict__ slide, double* __restrict__ lam_xi,
                                                        double* __restrict__ gout, double* __restrict__ lvn,
                                                        double* __restrict__ lPn, double* __restrict__ Bout,
                                                        int* __restrict__ status) {
    const StepParams& p = ap.p;
    const int64_t np = p.np;
    ADJ_LOOP(i, np) {
        double x0[3], beta[3], lg[3], lF[3], lAe[3], lxe[3], lP1[3];
        const uint8_t sb = slide[i];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x0[a] = xi[a * np + i];
            beta[a] = p.dt * 0.5 * (vstar[a * np + i] + v[a * np + i]) * p.invH[a];
            out_adjoints(p, (sb >> a) & 1u, lam_v[a * np + i], lam_P[a * np + i], mu[a * np + i], lP1[a], lAe[a], lg[a],
                         lF[a]);
            lxe[a] = lam_xe[a * np + i];
        }
        double dB[3][3];
        bool ok = true;
        for (int dir = 0; dir < 6; ++dir) {
            Dual xd[3], bd[3], gphi[3], F[3], Ae[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xd[a] = Dual(x0[a], dir == a ? 1.0 : 0.0);
                bd[a] = Dual(beta[a], dir == 3 + a ? 1.0 : 0.0);
            }
            const Dual phi = particle_phi(ap, xd, bd, lg, lF, lAe, lxe, table, lJ, gphi, F, Ae);
            ok = ok && isfinite(phi.d);
            if (dir < 3) {
                lam_xi[dir * np + i] = phi.d;
            } else {
                const int d = dir - 3;
                const double c = p.dt * 0.5 * p.invH[d];   // d beta_d / d v*_d
                gout[d * np + i] = c * phi.d;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    // v1 = (P + dt q (-gphibar + F) - q A_end) / m
                    const double dv1 = (p.dt * p.q * (F[a].d - gphi[a].d) - p.q * Ae[a].d) * p.inv_mass;
                    dB[a][d] = c * dv1;
                }
            }
        }
        if (!ok) atomicOr(status, DEV_ERR_NONFINITE);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const bool sl = (sb >> a) & 1u;
            const double g = gout[a * np + i];          // the orbit's adjoint of v*_a (also of v^n_a)
            if (sl) {
                // nu_a: the direct adjoint of v*_a (its velocity and momentum outputs) plus the
                // orbit's; v*_a = 2 d_a H_a / dt - v^n_a with d_a = knot - xi_a
                const double nu = lam_v[a * np + i] + p.mass * lam_P[a * np + i] + g;
                lam_xi[a * np + i] -= nu * 2.0 * p.H[a] / p.dt;
                lvn[a * np + i] = g - nu;
                lPn[a * np + i] = 0.0;
                gout[a * np + i] = 0.0;                  // no fixed-point equation: mu_a = 0
            } else {
                lvn[a * np + i] = g;
                lPn[a * np + i] = lP1[a];
            }
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const bool drop = sl || ((sb >> d) & 1u) || !(sb & SLIDE_CREPT);
                Bout[(3 * a + d) * np + i] = drop ? 0.0 : dB[a][d];
            }
        }
    }
}

// x = (I - B^T)^{-1} r for particle i's 3 x 3 block (Cramer's rule); false if singular.
__device__ __forceinline__ bool solve_block(const double* __restrict__ B, int64_t np, int64_t i, const double r[3],
                                            double x[3]) {
    double M[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int d = 0; d < 3; ++d) M[a][d] = (a == d ? 1.0 : 0.0) - B[(3 * d + a) * np + i];   // (B^T)[a][d] = B[d][a]
    const double det = M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) -
                       M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
                       M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0]);
    if (!(fabs(det) > 1e-300)) {
        x[0] = x[1] = x[2] = 0.0;
        return false;
    }
#pragma unroll
    for (int col = 0; col < 3; ++col) {
        double Mc[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int d = 0; d < 3; ++d) Mc[a][d] = d == col ? r[a] : M[a][d];
        const double dc = Mc[0][0] * (Mc[1][1] * Mc[2][2] - Mc[1][2] * Mc[2][1]) -
                          Mc[0][1] * (Mc[1][0] * Mc[2][2] - Mc[1][2] * Mc[2][0]) +
                          Mc[0][2] * (Mc[1][0] * Mc[2][1] - Mc[1][1] * Mc[2][0]);
        x[col] = dc / det;
    }
    return true;
}

// The preconditioner of the transposed solve, z = P r: per particle (I - B^T)^{-1} r, with B
// zero outside the particles the step solved locally (there P = I).
__global__ void k_adj_precond(int64_t np, const double* __restrict__ B, const double* __restrict__ r,
                              double* __restrict__ z, int* __restrict__ status) {
    ADJ_LOOP(i, np) {
        double ri[3], x[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ri[a] = r[a * np + i];
        if (!solve_block(B, np, i, ri, x)) atomicOr(status, DEV_ERR_NONFINITE);
#pragma unroll
        for (int a = 0; a < 3; ++a) z[a * np + i] = x[a];
    }
}

// w = z - (g - b0): the transposed fixed point's operator (I - K) applied to z, g = K z + b0
// being the sweep's output at mu = z.
__global__ void k_adj_apply(int64_t n, const double* __restrict__ z, const double* __restrict__ g,
                            const double* __restrict__ b0, double* __restrict__ w) {
    ADJ_LOOP(i, n) w[i] = z[i] - g[i] + b0[i];
}

// part[k * gridDim.x + b] = block b's share of w . V_k, k < nv (V_k at V + k ldv).
__global__ void k_adj_mdot(int64_t n, const double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int nv,
                           double* __restrict__ part) {
    __shared__ double sm[32];
    for (int k = 0; k < nv; ++k) {
        double s = 0.0;
        const double* vk = V + k * ldv;
        ADJ_LOOP(i, n) s += w[i] * vk[i];
        s = block_sum(s, sm);
        if (threadIdx.x == 0) part[k * gridDim.x + blockIdx.x] = s;
    }
}

// out[k] = sum over the nb block shares of dot k, in a fixed order (one block per dot).
__global__ void k_adj_mdot_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
    __shared__ double sm[32];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[blockIdx.x * nb + b];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w += sign * sum_k h[k] V_k, k < nv (h on the device).
__global__ void k_adj_combine(int64_t n, double* __restrict__ w, const double* __restrict__ V, int64_t ldv, int nv,
                              const double* __restrict__ h, double sign) {
    ADJ_LOOP(i, n) {
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s += h[k] * V[k * ldv + i];
        w[i] += sign * s;
    }
}

// Elementwise helpers.
__global__ void k_adj_axpy(int64_t n, double* __restrict__ y, const double* __restrict__ x, double s) {
    ADJ_LOOP(i, n) y[i] += s * x[i];
}

// ---- the initial data: rho^0 = sum q S(x)/dV, phi^0 from Poisson, P^0 = m v^0 ------------------
//
// lam_xi_i += (q/dV) sum_g dS_g/dxi (x_i) lam_dep[g] (the point deposit transposed).
__global__ void k_adj_deposit(AdjParams ap, const double* __restrict__ xi, const double* __restrict__ lam_dep,
                              double* __restrict__ lam_xi) {
    const StepParams& p = ap.p;
    const int64_t np = p.np;
    ADJ_LOOP(i, np) {
        double x[3], r[3];
        int c[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x[a] = xi[a * np + i];
            const double f = ::floor(x[a]);
            c[a] = (int)f;
            r[a] = x[a] - f;
        }
        Segment<double> sd;
        sd.cell[0] = c[0];
        sd.cell[1] = c[1];
        sd.cell[2] = c[2];
        int64_t g[8];
        segment_nodes8(sd, p.m, g);
        double out[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const double wx = (k & 1) ? r[0] : 1.0 - r[0], sx = (k & 1) ? 1.0 : -1.0;
            const double wy = (k & 2) ? r[1] : 1.0 - r[1], sy = (k & 2) ? 1.0 : -1.0;
            const double wz = (k & 4) ? r[2] : 1.0 - r[2], sz = (k & 4) ? 1.0 : -1.0;
            const double l = p.q_dV * lam_dep[g[k]];
            out[0] += sx * wy * wz * l;
            out[1] += wx * sy * wz * l;
            out[2] += wx * wy * sz * l;
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) lam_xi[a * np + i] += out[a];
    }
}

// The adjoint of W (field energy) with respect to phi, U and A of the current state:
// W = sum (|E|^2 / (2 sigma1) + |B|^2 / (2 sigma2)) dV with E = -grad phi - U, B = curl A.
__global__ void k_energy_grad(AdjParams ap, const double* __restrict__ F, const double* __restrict__ Wf,
                              double* __restrict__ lF, double* __restrict__ lW) {
    const StepParams& p = ap.p;
    const int64_t N = p.m.ncell;
    const double dV = p.H[0] * p.H[1] * p.H[2];
    ADJ_LOOP(g, N) {
        // E at a node and B at a node, as in the energy sum
        auto E = [&](int64_t n, int a) { return -dcen_s(F, 1, n, a, p.m, p.invH) - Wf[(1 + a) * N + n]; };
        auto Bc = [&](int64_t n, int c) {
            const double* Ax = F + N;
            const double* Ay = F + 2 * N;
            const double* Az = F + 3 * N;
            if (c == 0) return dcen_s(Az, 1, n, 1, p.m, p.invH) - dcen_s(Ay, 1, n, 2, p.m, p.invH);
            if (c == 1) return dcen_s(Ax, 1, n, 2, p.m, p.invH) - dcen_s(Az, 1, n, 0, p.m, p.invH);
            return dcen_s(Ay, 1, n, 0, p.m, p.invH) - dcen_s(Ax, 1, n, 1, p.m, p.invH);
        };
        // dW/dphi = -(D^T E) dV / sigma1 = (div E) dV / sigma1 (D_a^T = -D_a), dW/dU = -E dV / sigma1
        double divE = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const int64_t pp = a == 0 ? nshift(g, 1, 0, 0, p.m) : (a == 1 ? nshift(g, 0, 1, 0, p.m) : nshift(g, 0, 0, 1, p.m));
            const int64_t qq = a == 0 ? nshift(g, -1, 0, 0, p.m) : (a == 1 ? nshift(g, 0, -1, 0, p.m) : nshift(g, 0, 0, -1, p.m));
            divE += 0.5 * p.invH[a] * (E(pp, a) - E(qq, a));
            lW[(1 + a) * N + g] = -E(g, a) * dV / ap.sigma1;
        }
        lF[g] = divE * dV / ap.sigma1;
        lW[g] = 0.0;
        // dW/dA = curl^T (B) dV / sigma2 = curl(B) dV / sigma2 (curl is symmetric for skew D)
        auto dB = [&](int c, int a) {
            const int64_t pp = a == 0 ? nshift(g, 1, 0, 0, p.m) : (a == 1 ? nshift(g, 0, 1, 0, p.m) : nshift(g, 0, 0, 1, p.m));
            const int64_t qq = a == 0 ? nshift(g, -1, 0, 0, p.m) : (a == 1 ? nshift(g, 0, -1, 0, p.m) : nshift(g, 0, 0, -1, p.m));
            return 0.5 * p.invH[a] * (Bc(pp, c) - Bc(qq, c));
        };
        lF[N + g] = (dB(2, 1) - dB(1, 2)) * dV / ap.sigma2;
        lF[2 * N + g] = (dB(0, 2) - dB(2, 0)) * dV / ap.sigma2;
        lF[3 * N + g] = (dB(1, 0) - dB(0, 1)) * dV / ap.sigma2;
    }
}

}  // namespace

// ---- launchers ---------------------------------------------------------------------------------

int adj_blocks(const Ctx& c, int64_t n) {
    int64_t b = (n + THREADS - 1) / THREADS;
    b = std::min<int64_t>(std::max<int64_t>(b, 1), (int64_t)c.sms * 8);
    return (int)std::min<int64_t>(b, MAX_BLOCKS);
}

void launch_adj_scatter(Ctx& c, const double* xi, const double* v, const double* vstar, const double* lam_P,
                        const double* lam_v, const double* mu, double* lam_tab) {
    k_adj_scatter<<<adj_blocks(c, c.np), THREADS, 0, c.stream>>>(adj_params(c), xi, v, vstar, c.table, lam_P, lam_v,
                                                                  mu, c.slide, lam_tab);
    ++c.launches;
}

void launch_adj_mesh_rhs(Ctx& c, const double* lam_tab, const double* lF1, const double* lW1, double* t, double* pn) {
    k_adj_mesh_rhs<<<adj_blocks(c, c.m.ncell), THREADS, 0, c.stream>>>(adj_params(c), lam_tab, lF1, lW1, t, pn);
    ++c.launches;
}

void launch_adj_mesh_out(Ctx& c, const double* y, const double* pn, const double* lW1, const double* lrho1,
                         double* lF0, double* lW0, double* lrho0, double* lJ) {
    k_adj_mesh_out<<<adj_blocks(c, c.m.ncell), THREADS, 0, c.stream>>>(adj_params(c), y, pn, lW1, lrho1, lF0, lW0,
                                                                        lrho0, lJ);
    ++c.launches;
}

void launch_adj_derivs(Ctx& c, const double* xi, const double* v, const double* vstar, const double* lJ,
                       const double* lam_P, const double* lam_v, const double* lam_xe, const double* mu,
                       double* lam_xi, double* g, double* lvn, double* lPn, double* B) {
    k_adj_derivs<<<adj_blocks(c, c.np), THREADS, 0, c.stream>>>(adj_params(c), xi, v, vstar, c.table, lJ, lam_P,
                                                                 lam_v, lam_xe, mu, c.slide, lam_xi, g, lvn, lPn, B,
                                                                 c.dev_status);
    ++c.launches;
}

void launch_adj_precond(Ctx& c, const double* B, const double* r, double* z) {
    k_adj_precond<<<adj_blocks(c, c.np), THREADS, 0, c.stream>>>(c.np, B, r, z, c.dev_status);
    ++c.launches;
}

void launch_adj_apply(Ctx& c, int64_t n, const double* z, const double* g, const double* b0, double* w) {
    k_adj_apply<<<adj_blocks(c, n), THREADS, 0, c.stream>>>(n, z, g, b0, w);
    ++c.launches;
}

void launch_adj_mdot(Ctx& c, int64_t n, const double* w, const double* V, int64_t ldv, int nv, double* part,
                     double* out) {
    const int nb = adj_blocks(c, n);
    k_adj_mdot<<<nb, THREADS, 0, c.stream>>>(n, w, V, ldv, nv, part);
    k_adj_mdot_final<<<nv, THREADS, 0, c.stream>>>(part, nb, out);
    c.launches += 2;
}

void launch_adj_combine(Ctx& c, int64_t n, double* w, const double* V, int64_t ldv, int nv, const double* h,
                        double sign) {
    k_adj_combine<<<adj_blocks(c, n), THREADS, 0, c.stream>>>(n, w, V, ldv, nv, h, sign);
    ++c.launches;
}

void launch_adj_axpy(Ctx& c, int64_t n, double* y, const double* x, double s) {
    k_adj_axpy<<<adj_blocks(c, n), THREADS, 0, c.stream>>>(n, y, x, s);
    ++c.launches;
}

void launch_adj_deposit(Ctx& c, const double* xi, const double* lam_dep, double* lam_xi) {
    k_adj_deposit<<<adj_blocks(c, c.np), THREADS, 0, c.stream>>>(adj_params(c), xi, lam_dep, lam_xi);
    ++c.launches;
}

void launch_energy_grad(Ctx& c, double* lF, double* lW) {
    k_energy_grad<<<adj_blocks(c, c.m.ncell), THREADS, 0, c.stream>>>(adj_params(c), c.F0, c.W0, lF, lW);
    ++c.launches;
}

}  // namespace pic
