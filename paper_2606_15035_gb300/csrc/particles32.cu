// FP32 particle kernels of the mixed-precision Picard iterations (sm_103a).
//
// The mixed path runs the first Picard iterations of Algorithm 1 in single precision: the
// orbit breakpoints, the Appendix A/B orbit integrals, the gather, the canonical-momentum
// push and the orbit current are computed in FP32 from an FP32 working set, while the mesh
// solve (continuity, Crank--Nicolson), the reductions and the accumulation of J stay FP64.
// The FP64 kernels then refine the iterate to the FP64 tolerance and run the final sweep, so
// the accepted step is a solution of the FP64 discrete equations.
//
// FP32 working set (device order, structure of arrays):
//   cell[i]   packed cell index cx | cy << 10 | cz << 20 of the particle's start position;
//   off[c,i]  offset of the start position inside that cell, in [0, 1) (cell units);
//   v, P      v^n and P^n rounded to FP32;  vit, vnew: the Picard iterates.
// Positions relative to the cell keep ~1e-7-cell resolution for the knot tests at any mesh size.
#include <cmath>

#include "pic_internal.h"

namespace pic {
namespace {

constexpr int CELL_BITS = 10;
constexpr int CELL_MASK = (1 << CELL_BITS) - 1;

__device__ __forceinline__ void unpack_cell(int32_t c, int cc[3]) {
    cc[0] = c & CELL_MASK;
    cc[1] = (c >> CELL_BITS) & CELL_MASK;
    cc[2] = (c >> (2 * CELL_BITS)) & CELL_MASK;
}

struct Params32 {
    MeshDims m;
    float invH[3];
    float dt, q, inv_mass, q_dV;
    int64_t np;
};

template <typename T>
__device__ __forceinline__ void write_partial32(double* partials, int slot, double v, double* sm) {
    double r = block_sum(v, sm);
    if (threadIdx.x == 0) partials[slot * MAX_BLOCKS + blockIdx.x] = r;
}

// Orbit current of one FP32 orbit (closed form, Appendix A) into the FP64 J.
__device__ __forceinline__ int scatter32(const Params32& p, const int cb[3], const float x0[3], const float beta[3],
                                         const float w[3], double* __restrict__ J) {
    const int64_t N = p.m.ncell;
    return for_each_segment(x0, beta, true, [&](const Segment<float>& sg0) {
        Segment<float> sg = sg0;
        float I[8];
        weights_from_ints(piece_integrals(sg, beta, false), I);
        sg.cell[0] += cb[0];
        sg.cell[1] += cb[1];
        sg.cell[2] += cb[2];
        int64_t g[8];
        segment_nodes8(sg, p.m, g);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            atomicAdd(J + g[k], (double)(w[0] * I[k]));
            atomicAdd(J + N + g[k], (double)(w[1] * I[k]));
            atomicAdd(J + 2 * N + g[k], (double)(w[2] * I[k]));
        }
    });
}

// G(u) in FP32: the orbit push of Algorithm 1 with the FP32 gather table
// (per node: A^n (3), A^{n+1} (3), grad_h phi^{n+1/2} (3), 3 unused).
__device__ __forceinline__ int push32(const Params32& p, const int cb[3], const float x0[3], const float vn[3],
                                      const float Pn[3], const float u[3], const float* __restrict__ table,
                                      float vw[3]) {
    float vb[3], beta[3], gphi[3] = {0.f, 0.f, 0.f}, F[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        vb[a] = 0.5f * (u[a] + vn[a]);
        beta[a] = p.dt * vb[a] * p.invH[a];
    }
    const int nseg = for_each_segment(x0, beta, true, [&](const Segment<float>& sg0) {
        Segment<float> sg = sg0;
        const PieceInts<float> I = piece_integrals(sg, beta, true);
        float W[8];
        weights_from_ints(I, W);
        sg.cell[0] += cb[0];
        sg.cell[1] += cb[1];
        sg.cell[2] += cb[2];
        int64_t g[8];
        segment_nodes8(sg, p.m, g);
        const float s = sg.s0, oms = 1.f - s, h = sg.h, hh2 = 0.5f * h * h;
        float am[8], cc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4* t4 = reinterpret_cast<const float4*>(table + 12 * g[k]);
            const float4 a = t4[0], b = t4[1], c = t4[2];
            const float an = a.x * vb[0] + a.y * vb[1] + a.z * vb[2];
            const float a1 = a.w * vb[0] + b.x * vb[1] + b.y * vb[2];
            am[k] = oms * an + s * a1;
            cc[k] = a1 - an;
            gphi[0] += W[k] * b.z;
            gphi[1] += W[k] * b.w;
            gphi[2] += W[k] * c.x;
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int pa = j == 0 ? 1 : 0, qa = j == 2 ? 1 : 2;
            const int sp = j == 0 ? 2 : 1, sq = j == 2 ? 2 : 4;
            const int sj = j == 0 ? 1 : (j == 1 ? 2 : 4);
            const float D00 = am[sj] - am[0], D10 = am[sp + sj] - am[sp];
            const float D01 = am[sq + sj] - am[sq], D11 = am[sp + sq + sj] - am[sp + sq];
            const float C00 = cc[sj] - cc[0], C10 = cc[sp + sj] - cc[sp];
            const float C01 = cc[sq + sj] - cc[sq], C11 = cc[sp + sq + sj] - cc[sp + sq];
            const float t0 = D00 * h + (D10 - D00) * I.S1[pa] + (D01 - D00) * I.S1[qa] +
                             (D11 - D10 - D01 + D00) * I.S2[j];
            const float t1 = C00 * hh2 + (C10 - C00) * I.E1[pa] + (C01 - C00) * I.E1[qa] +
                             (C11 - C10 - C01 + C00) * I.E2[j];
            F[j] += p.invH[j] * (t0 + t1);
        }
    });
    // end point, in the particle's frame, then the point interpolant of A^{n+1}
    int cc[3];
    float r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xe = x0[a] + beta[a];
        const float f = floorf(xe);
        cc[a] = cb[a] + (int)f;
        r[a] = xe - f;
    }
    Segment<float> cs;
    cs.cell[0] = cc[0];
    cs.cell[1] = cc[1];
    cs.cell[2] = cc[2];
    int64_t g[8];
    segment_nodes8(cs, p.m, g);
    float Ae[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float wx = (k & 1) ? r[0] : 1.f - r[0], wy = (k & 2) ? r[1] : 1.f - r[1], wz = (k & 4) ? r[2] : 1.f - r[2];
        const float w = wx * wy * wz;
        const float4* t4 = reinterpret_cast<const float4*>(table + 12 * g[k]);
        const float4 a = t4[0], b = t4[1];
        Ae[0] += w * a.w;
        Ae[1] += w * b.x;
        Ae[2] += w * b.y;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float Pw = Pn[a] + p.dt * (p.q * (F[a] - gphi[a]));
        vw[a] = (Pw - p.q * Ae[a]) * p.inv_mass;
    }
    return nseg;
}

// FP64 masters -> FP32 working set; v^{n+1,0} = 2 v^n - v^{n-1}.
__global__ void k_to32(Params32 p, const double* __restrict__ xi, const double* __restrict__ v,
                       const double* __restrict__ P, const double* __restrict__ vprev, int32_t* __restrict__ cell,
                       float* __restrict__ off, float* __restrict__ v32, float* __restrict__ P32,
                       float* __restrict__ vit32, double* __restrict__ partials) {
    __shared__ double sm[32];
    const int64_t np = p.np;
    double jsc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t packed = 0;
        const double va = v[i], vb = v[np + i], vc = v[2 * np + i];
        jsc += sqrt(va * va + vb * vb + vc * vc);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double x = xi[a * np + i];
            double c = floor(x);
            if (c < 0.0) c = 0.0;
            if (c > (double)(p.m.n[a] - 1)) c = (double)(p.m.n[a] - 1);
            off[a * np + i] = (float)(x - c);
            packed |= ((int32_t)c & CELL_MASK) << (a * CELL_BITS);
            const double vv = v[a * np + i];
            v32[a * np + i] = (float)vv;
            P32[a * np + i] = (float)P[a * np + i];
            vit32[a * np + i] = (float)(2.0 * vv - vprev[a * np + i]);
        }
        cell[i] = packed;
    }
    write_partial32<double>(partials, S_JSCALE, jsc, sm);
}

// Orbit current of the FP32 iterate (first iteration of the step).
__global__ void k_scatter32(Params32 p, const int32_t* __restrict__ cell, const float* __restrict__ off,
                            const float* __restrict__ v32, const float* __restrict__ vit32, double* __restrict__ J,
                            int* __restrict__ status) {
    const int64_t np = p.np;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int cb[3];
        unpack_cell(cell[i], cb);
        float x0[3], beta[3], w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x0[a] = off[a * np + i];
            const float vb = 0.5f * (vit32[a * np + i] + v32[a * np + i]);
            beta[a] = p.dt * vb * p.invH[a];
            w[a] = p.q_dV * vb;
        }
        if (scatter32(p, cb, x0, beta, w, J) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
    }
}

// One FP32 Picard iteration: G(v^p), the e_v partial sums, and the orbit current of
// v^{p+1} = G(v^p) into Jnext.
__global__ void __launch_bounds__(THREADS) k_push32(Params32 p, const int32_t* __restrict__ cell,
                                                    const float* __restrict__ off, const float* __restrict__ v32,
                                                    const float* __restrict__ P32, const float* __restrict__ vit32,
                                                    const float* __restrict__ table, float* __restrict__ vnew32,
                                                    double* __restrict__ Jnext, double* __restrict__ partials,
                                                    int* __restrict__ status) {
    __shared__ double sm[32];
    const int64_t np = p.np;
    double ev_num = 0.0, ev_den = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int cb[3];
        unpack_cell(cell[i], cb);
        float x0[3], vn[3], Pn[3], u[3], vw[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            x0[a] = off[a * np + i];
            vn[a] = v32[a * np + i];
            Pn[a] = P32[a * np + i];
            u[a] = vit32[a * np + i];
        }
        if (push32(p, cb, x0, vn, Pn, u, table, vw) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
        if (!(isfinite(vw[0]) && isfinite(vw[1]) && isfinite(vw[2]))) atomicOr(status, DEV_ERR_NONFINITE);
        float beta[3], w[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const double d = (double)vw[a] - (double)u[a];
            ev_num += d * d;
            ev_den += (double)vw[a] * (double)vw[a];
            vnew32[a * np + i] = vw[a];
            const float vb = 0.5f * (vw[a] + vn[a]);
            beta[a] = p.dt * vb * p.invH[a];
            w[a] = p.q_dV * vb;
        }
        if (scatter32(p, cb, x0, beta, w, Jnext) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
    }
    write_partial32<double>(partials, S_EV_NUM, ev_num, sm);
    write_partial32<double>(partials, S_EV_DEN, ev_den, sm);
}

// FP64 gather table -> FP32 table (A^n, A^{n+1}, grad phi; 3 unused).
__global__ void k_table32(int64_t N, const double* __restrict__ t64, float* __restrict__ t32) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 9; ++k) t32[12 * g + k] = (float)t64[12 * g + k];
        t32[12 * g + 9] = t32[12 * g + 10] = t32[12 * g + 11] = 0.f;
    }
}

__global__ void k_from32(int64_t n3, const float* __restrict__ a, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n3; i += (int64_t)gridDim.x * blockDim.x)
        b[i] = (double)a[i];
}

Params32 make_params32(const Ctx& c) {
    Params32 p;
    p.m = c.m;
    for (int a = 0; a < 3; ++a) p.invH[a] = (float)c.invH[a];
    p.dt = (float)c.cfg.dt;
    p.q = (float)c.q;
    p.inv_mass = (float)(1.0 / c.mass);
    p.q_dV = (float)(c.q / c.dV);
    p.np = c.np;
    return p;
}

}  // namespace

void launch_to32(Ctx& c) {
    k_to32<<<particle_blocks(c), THREADS, 0, c.stream>>>(make_params32(c), c.xi, c.v, c.P, c.vprev, c.cell32,
                                                         c.off32, c.v32, c.P32, c.vit32, c.partials);
    ++c.launches;
}

void launch_scatter32(Ctx& c, double* J) {
    k_scatter32<<<particle_blocks(c), THREADS, 0, c.stream>>>(make_params32(c), c.cell32, c.off32, c.v32, c.vit32, J,
                                                              c.dev_status);
    ++c.launches;
}

void launch_push32(Ctx& c, double* Jnext) {
    k_push32<<<particle_blocks(c), THREADS, 0, c.stream>>>(make_params32(c), c.cell32, c.off32, c.v32, c.P32, c.vit32,
                                                           c.table32, c.vnew32, Jnext, c.partials, c.dev_status);
    ++c.launches;
}

void launch_table32(Ctx& c) {
    k_table32<<<mesh_blocks(c), THREADS, 0, c.stream>>>(c.m.ncell, c.table, c.table32);
    ++c.launches;
}

void launch_from32(Ctx& c, const float* a, double* b) {
    k_from32<<<particle_blocks(c), THREADS, 0, c.stream>>>(3 * c.np, a, b);
    ++c.launches;
}

}  // namespace pic
