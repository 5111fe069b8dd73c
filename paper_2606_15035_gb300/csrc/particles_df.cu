// FP32-pair refinement push of the mixed-precision path (sm_103a).
//
// After the FP32 Picard iterations have brought the iterate to the FP32 floor (~1e-9), the
// mixed path refines it with Algorithm 1 iterations whose particle half (orbit breakpoints,
// Appendix A/B orbit integrals, gather, canonical-momentum push, point interpolant, next-orbit
// current) runs in FP32-pair arithmetic (dfloat.cuh: 48-bit significands on the FP32 pipes)
// instead of FP64.  The iterates stay FP64 arrays, so the FP64 particle-local solves, the
// residual sums and the FP64 iterations that close the step use them unchanged.  The pair
// map differs from the FP64 map G by ~1e-15 of the velocity (positions are carried as the
// cell index plus a pair offset in the cell, so their resolution is 2^-48 cells at any mesh
// size), so its fixed point is the FP64 fixed point to that level.  What checks the iterate
// is FP64: the FP64 final sweep, which measures ||G(v*) - v*|| of the pair iterate itself
// before committing it (the mixed path's default with mixed_tol64 > 0), or the FP64
// iterations that follow.  Compiled for four resident blocks per SM (64 registers, with
// spills): the pair arithmetic's dependent chains need the warps more than the registers.
//
// Per chunk of THREADS cell-sorted particles the next-orbit current goes into a shared-memory
// tile of 64-bit fixed-point sums (exact, order independent, 2^-52 of the chunk's largest
// weight per unit), added to the FP64 J once per node; a chunk whose orbits' node box does not
// fit the tile adds its contributions to J directly.
#include <algorithm>
#include <climits>
#include <cmath>

#include "pic_internal.h"
#include "particle_common.cuh"
#include "dfloat.cuh"

namespace pic {
namespace {

constexpr int DF_TILE_CAP = 320;   // nodes of a chunk's current tile
constexpr int DF_NODE4 = 5;        // float4 per node of the pair table: A^n, A^{n+1}, grad phi (9 pairs)

struct ParamsDF {
    StepParams p;       // the FP64 parameters (creeping tests, residual sums, iterate I/O)
    DF dth[3];          // dt / (2 H_a): beta_a = dth_a (u_a + v^n_a)
    DF dt_invH[3];      // dt / H_a
    DF invH[3];         // 1 / H_a
    DF dt_q;            // dt q
    DF q;
    DF q_dV;            // q / dV
};

DF pair_of(double d) {
    const float h = (float)d;
    return DF(h, (float)(d - (double)h));
}

// The 9 pairs of node g: A^n (3), A^{n+1} (3), grad_h phi^{n+1/2} (3).
struct NodeDF {
    DF An[3], A1[3], g[3];
};

__device__ __forceinline__ NodeDF load_node(const float4* __restrict__ t, int64_t g) {
    const float4* q = t + DF_NODE4 * g;
    const float4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3), e = __ldg(q + 4);
    NodeDF n;
    n.An[0] = DF(a.x, a.y);
    n.An[1] = DF(a.z, a.w);
    n.An[2] = DF(b.x, b.y);
    n.A1[0] = DF(b.z, b.w);
    n.A1[1] = DF(c.x, c.y);
    n.A1[2] = DF(c.z, c.w);
    n.g[0] = DF(d.x, d.y);
    n.g[1] = DF(d.z, d.w);
    n.g[2] = DF(e.x, e.y);
    return n;
}

__device__ __forceinline__ void cell_nodes(const int c[3], const MeshDims& m, int64_t g[8]) {
    Segment<float> s;
    s.cell[0] = c[0];
    s.cell[1] = c[1];
    s.cell[2] = c[2];
    segment_nodes8(s, m, g);
}

// One knot-free piece of the push (Appendices A and B), as push_piece_fast in FP64: the
// orbit gather of grad phi and (D_i A)^T vbar, contracted with vbar first.  Piece cells are
// relative to the particle's start cell c0.
__device__ __forceinline__ void push_piece_df(const ParamsDF& pd, const Segment<DF>& sg, const int c0[3],
                                              const DF beta[3], const DF vb[3], const float4* __restrict__ table,
                                              DF gphi[3], DF F[3]) {
    const PieceInts<DF> I = piece_integrals(sg, beta, true);
    DF W[8];
    weights_from_ints(I, W);
    const int c[3] = {c0[0] + sg.cell[0], c0[1] + sg.cell[1], c0[2] + sg.cell[2]};
    int64_t g[8];
    cell_nodes(c, pd.p.m, g);
    const DF s = sg.s0, oms = DF(1) - sg.s0, h = sg.h, hh2 = DF(0.5f) * (sg.h * sg.h);
    DF am[8], cc[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const NodeDF n = load_node(table, g[k]);
        const DF an = n.An[0] * vb[0] + n.An[1] * vb[1] + n.An[2] * vb[2];   // A^n_g . vbar
        const DF a1 = n.A1[0] * vb[0] + n.A1[1] * vb[1] + n.A1[2] * vb[2];   // A^{n+1}_g . vbar
        am[k] = oms * an + s * a1;                                           // A^{(m)}_nu . vbar
        cc[k] = a1 - an;                                                     // C^{(m)}_nu . vbar
        gphi[0] += W[k] * n.g[0];
        gphi[1] += W[k] * n.g[1];
        gphi[2] += W[k] * n.g[2];
    }
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int pa = j == 0 ? 1 : 0, qa = j == 2 ? 1 : 2;
        const int sp = j == 0 ? 2 : 1, sq = j == 2 ? 2 : 4;
        const int sj = j == 0 ? 1 : (j == 1 ? 2 : 4);
        const DF D00 = am[sj] - am[0], D10 = am[sp + sj] - am[sp];
        const DF D01 = am[sq + sj] - am[sq], D11 = am[sp + sq + sj] - am[sp + sq];
        const DF C00 = cc[sj] - cc[0], C10 = cc[sp + sj] - cc[sp];
        const DF C01 = cc[sq + sj] - cc[sq], C11 = cc[sp + sq + sj] - cc[sp + sq];
        const DF t0 = D00 * h + (D10 - D00) * I.S1[pa] + (D01 - D00) * I.S1[qa] + (D11 - D10 - D01 + D00) * I.S2[j];
        const DF t1 = C00 * hh2 + (C10 - C00) * I.E1[pa] + (C01 - C00) * I.E1[qa] + (C11 - C10 - C01 + C00) * I.E2[j];
        F[j] += pd.invH[j] * (t0 + t1);
    }
}

// Minimal-image offset of cell c from cell ref on a periodic axis of n cells.
__device__ __forceinline__ int rel_cell_df(int c, int ref, int n) {
    int d = c - ref;
    if (2 * d > n) d -= n;
    else if (2 * d < -n) d += n;
    return d;
}

// Block-wide box of node ranges [lo, hi] and maxima of amax (non-negative floats, reduced
// through their bit patterns); sm holds 9 * 32 + 9 ints.  Every thread gets the result.
__device__ __forceinline__ void block_box_df(int lo[3], int hi[3], float amax[3], int* sm) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int v[9];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        v[a] = __reduce_min_sync(0xffffffffu, lo[a]);
        v[3 + a] = __reduce_max_sync(0xffffffffu, hi[a]);
        v[6 + a] = __reduce_max_sync(0xffffffffu, __float_as_int(amax[a]));
    }
    if (lane == 0) {
#pragma unroll
        for (int t = 0; t < 9; ++t) sm[t * 32 + wid] = v[t];
    }
    __syncthreads();
    if (threadIdx.x < 9) {
        const int t = threadIdx.x;
        int r = sm[t * 32];
        for (int w = 1; w < nw; ++w) r = t < 3 ? min(r, sm[t * 32 + w]) : max(r, sm[t * 32 + w]);
        sm[288 + t] = r;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        lo[a] = sm[288 + a];
        hi[a] = sm[291 + a];
        amax[a] = __int_as_float(sm[294 + a]);
    }
    __syncthreads();   // sm is reused by the next reduction
}

// The chunk's current tile: node (lx, ly, lz) of the box at lx + ex (ly + ey lz), one 64-bit
// fixed-point sum per component in units of 1 / scale[a].
struct TileDF {
    long long* jt;
    int lo[3], ext[3];
    int vol;
    float scale[3];
};

__device__ __forceinline__ long long fixed64(DF c, float scale) {
    return __float2ll_rn(c.hi * scale) + __float2ll_rn(c.lo * scale);   // exact scaling by a power of 2
}

// Next-orbit current of one particle (closed-form weights, Appendix A): into the tile when
// `tiled`, else straight into the FP64 J.
__device__ __forceinline__ int scatter_df(const ParamsDF& pd, const TileDF& tl, bool tiled, const int c0[3],
                                          const int co[3], const DF x0[3], const DF beta[3], const DF w[3],
                                          double* __restrict__ J) {
    const int64_t N = pd.p.m.ncell;
    return for_each_segment(x0, beta, true, [&](const Segment<DF>& sg) {
        DF I[8];
        weights_from_ints(piece_integrals(sg, beta, false), I);
        if (tiled) {
            const int lx = co[0] + sg.cell[0] - tl.lo[0], ly = co[1] + sg.cell[1] - tl.lo[1];
            const int lz = co[2] + sg.cell[2] - tl.lo[2];
            const int ex = tl.ext[0], exy = tl.ext[0] * tl.ext[1];
            const int base = lx + ex * ly + exy * lz;
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int l = base + (k & 1) + ((k >> 1) & 1) * ex + (k >> 2) * exy;
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    atomicAdd(reinterpret_cast<unsigned long long*>(tl.jt + a * DF_TILE_CAP + l),
                              (unsigned long long)fixed64(w[a] * I[k], tl.scale[a]));
            }
        } else {
            const int c[3] = {c0[0] + sg.cell[0], c0[1] + sg.cell[1], c0[2] + sg.cell[2]};
            int64_t g[8];
            cell_nodes(c, pd.p.m, g);
#pragma unroll
            for (int k = 0; k < 8; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) atomicAdd(J + a * N + g[k], dbl_of(w[a] * I[k]));
        }
    });
}

// The FP32-pair iteration: G(v^p) for every particle, creeping ones listed for k_local (as in
// k_push), the e_v partial sums, and the orbit current of v^{p+1} = G(v^p) into Jnext.
__global__ void __launch_bounds__(THREADS, 4) k_push_df(ParamsDF pd, const double* __restrict__ xi,
                                                         const double* __restrict__ v, const double* __restrict__ P,
                                                         const double* __restrict__ vit,
                                                         const float4* __restrict__ table, double* __restrict__ vnew,
                                                         double* __restrict__ Jnext, int32_t* __restrict__ creep_list,
                                                         int* __restrict__ creep_count,
                                                         uint8_t* __restrict__ creep_flag,
                                                         const uint8_t* __restrict__ slide,
                                                         double* __restrict__ partials, int* __restrict__ status) {
    __shared__ double sm[32];
    __shared__ int order[THREADS];
    __shared__ int wcount[THREADS / 32][PIECE_CLASSES];
    __shared__ int sbox[9 * 32 + 9];
    __shared__ long long jt[3 * DF_TILE_CAP];
    const StepParams& p = pd.p;
    const int64_t np = p.np, nchunks = (np + THREADS - 1) / THREADS;
    double ev_num = 0.0, ev_den = 0.0, pieces_push = 0.0, pieces_scatter = 0.0;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const int64_t base = ch * THREADS;
        {
            const int64_t j = base + threadIdx.x;
            const int cls = j < np ? piece_class(p, xi, v, vit, j) : PIECE_CLASSES - 1;
            order[stable_class_rank(cls, wcount)] = threadIdx.x;
        }
        __syncthreads();
        const int64_t i = base + order[threadIdx.x];
        int ref[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) ref[a] = min(max((int)::floor(xi[a * np + base]), 0), p.m.n[a] - 1);
        // the particle's push; `scat` is set when its next orbit is scattered here
        bool scat = false;
        int c0[3] = {0, 0, 0}, co[3] = {0, 0, 0}, lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        float amax[3] = {0.f, 0.f, 0.f};
        DF off[3], beta2[3], w2[3];
        if (i < np) {
            double x0[3], vn[3], vi[3], Pn[3];
            DF vb[3], beta[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = xi[a * np + i];
                vn[a] = v[a * np + i];
                vi[a] = vit[a * np + i];
                Pn[a] = P[a * np + i];
                const double cf = ::floor(x0[a]);
                c0[a] = (int)cf;
                off[a] = df_of(x0[a] - cf);              // exact in FP64, then to a pair
                vb[a] = df_of(0.5 * (vi[a] + vn[a]));
                beta[a] = vb[a] * pd.dt_invH[a];
            }
            DF gphi[3], F[3];
            const int nseg = for_each_segment(off, beta, true, [&](const Segment<DF>& sg) {
                push_piece_df(pd, sg, c0, beta, vb, table, gphi, F);
            });
            if (nseg < 0) atomicOr(status, DEV_ERR_SEGMENTS);
            pieces_push += (double)nseg;
            // x^{n+1} in the cells of the start, A_h^{n+1}(x^{n+1}) by the point interpolant
            DF xe[3], r[3];
            int ce[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                xe[a] = off[a] + beta[a];
                const DF f = floor(xe[a]);
                ce[a] = c0[a] + (int)f;
                r[a] = xe[a] - f;
            }
            int64_t ge[8];
            cell_nodes(ce, p.m, ge);
            DF Ae[3];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const DF wx = (k & 1) ? r[0] : DF(1) - r[0];
                const DF wy = (k & 2) ? r[1] : DF(1) - r[1];
                const DF wz = (k & 4) ? r[2] : DF(1) - r[2];
                const DF wk = wx * wy * wz;
                const NodeDF n = load_node(table, ge[k]);
                Ae[0] += wk * n.A1[0];
                Ae[1] += wk * n.A1[1];
                Ae[2] += wk * n.A1[2];
            }
            double vw[3];
            bool finite = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double Pw = Pn[a] + dbl_of(pd.dt_q * (F[a] - gphi[a]));   // Eq. (orbit-P-update)
                vw[a] = (Pw - dbl_of(pd.q * Ae[a])) * p.inv_mass;              // Eq. (orbit-v-update)
                finite = finite && isfinite(vw[a]);
            }
            if (!finite) atomicOr(status, DEV_ERR_NONFINITE);
            // the local-solve gate of k_push, in FP64
            double beta_it[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) beta_it[a] = p.dt * 0.5 * (vi[a] + vn[a]) * p.invH[a];
            const double xk[3] = {x0[0] - p.koff, x0[1] - p.koff, x0[2] - p.koff};
            bool slow = false;
            if (p.hist) {
                double dn = 0.0, dold = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    dn = fmax(dn, ::fabs(vw[a] - vi[a]));
                    dold = fmax(dold, ::fabs(vi[a] - vnew[a * np + i]));
                }
                const double spd = sqrt(vi[0] * vi[0] + vi[1] * vi[1] + vi[2] * vi[2]);
                slow = dn > SLOW_RATIO * dold && dn > pd.p.slow_floor * spd;
            }
            const bool creep = p.accel && (is_creeping(xk, beta_it) || (slide[i] & SLIDE_CREPT) || slow);
            if (creep_flag) creep_flag[i] = creep ? 1 : 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) vnew[a * np + i] = vw[a];
            if (creep) {
                if (!creep_flag) {
                    const int k = atomicAdd(creep_count, 1);
                    creep_list[k] = (int32_t)i;
                }
            } else {
                double dnum = 0.0, dden = 0.0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = vw[a] - vi[a];
                    dnum += d * d;
                    dden += vw[a] * vw[a];
                    const DF vb2 = df_of(0.5 * (vw[a] + vn[a]));
                    beta2[a] = vb2 * pd.dt_invH[a];
                    w2[a] = vb2 * pd.q_dV;
                    amax[a] = fabsf(w2[a].hi);
                }
                ev_num += dnum;
                ev_den += dden;
                scat = true;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    co[a] = rel_cell_df(c0[a], ref[a], p.m.n[a]);
                    const DF xe2 = off[a] + beta2[a];
                    const int e0 = (int)floor(fmin(off[a], xe2)), e1 = (int)floor(fmax(off[a], xe2));
                    lo[a] = co[a] + e0;
                    hi[a] = co[a] + e1 + 1;
                }
            }
        }
        // the chunk's node box of the next orbits, and its fixed-point scales
        block_box_df(lo, hi, amax, sbox);
        TileDF tl;
        int64_t vol = 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            tl.lo[a] = lo[a];
            tl.ext[a] = hi[a] - lo[a] + 1;
            vol *= tl.ext[a] > 0 ? tl.ext[a] : 0;
            int e = 0;
            frexpf(amax[a], &e);                    // amax < 2^e: a contribution maps below 2^52
            tl.scale[a] = ldexpf(1.f, 52 - max(e, -60));
        }
        const bool tiled = vol > 0 && vol <= DF_TILE_CAP;
        tl.vol = tiled ? (int)vol : 0;
        tl.jt = jt;
        if (tiled) {
            for (int l = threadIdx.x; l < 3 * DF_TILE_CAP; l += blockDim.x) jt[l] = 0;
            __syncthreads();
        }
        if (scat) {
            const int ns = scatter_df(pd, tl, tiled, c0, co, off, beta2, w2, Jnext);
            if (ns < 0) atomicOr(status, DEV_ERR_SEGMENTS);
            pieces_scatter += (double)ns;
        }
        if (tiled) {
            __syncthreads();
            const int64_t N = p.m.ncell;
            const int ex = tl.ext[0], exy = tl.ext[0] * tl.ext[1];
            for (int l = threadIdx.x; l < tl.vol; l += blockDim.x) {
                const int lz = l / exy, rr = l - lz * exy, ly = rr / ex, lx = rr - ly * ex;
                const int64_t g = node_index(wrapi(ref[0] + tl.lo[0] + lx, p.m.n[0]),
                                             wrapi(ref[1] + tl.lo[1] + ly, p.m.n[1]),
                                             wrapi(ref[2] + tl.lo[2] + lz, p.m.n[2]), p.m);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const long long s = jt[a * DF_TILE_CAP + l];
                    if (s != 0) atomicAdd(Jnext + a * N + g, (double)s / (double)tl.scale[a]);
                }
            }
        }
        __syncthreads();   // order[] and the tile are rewritten by the next chunk
    }
    write_partial<double>(partials, S_EV_NUM, ev_num, sm, false);
    write_partial<double>(partials, S_EV_DEN, ev_den, sm, false);
    write_partial<double>(partials, S_PIECES_PUSH, pieces_push, sm, false);
    write_partial<double>(partials, S_PIECES_SCATTER, pieces_scatter, sm, false);
}

// FP64 gather table (12 doubles per node) -> pair table (A^n, A^{n+1}, grad phi as pairs).
__global__ void k_table_df(int64_t N, const double* __restrict__ t64, float4* __restrict__ tdf) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
        float f[20];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const double d = t64[12 * g + k];
            const float h = (float)d;
            f[2 * k] = h;
            f[2 * k + 1] = (float)(d - (double)h);
        }
        f[18] = f[19] = 0.f;
#pragma unroll
        for (int q = 0; q < DF_NODE4; ++q) tdf[DF_NODE4 * g + q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
    }
}

ParamsDF make_params_df(const Ctx& c) {
    ParamsDF pd;
    pd.p = make_params(c);
    pd.p.hist = c.cfg.picard_accel && c.run.hist;
    for (int a = 0; a < 3; ++a) {
        pd.dth[a] = pair_of(0.5 * c.cfg.dt / c.H[a]);
        pd.dt_invH[a] = pair_of(c.cfg.dt / c.H[a]);
        pd.invH[a] = pair_of(c.invH[a]);
    }
    pd.dt_q = pair_of(c.cfg.dt * c.q);
    pd.q = pair_of(c.q);
    pd.q_dV = pair_of(c.q / c.dV);
    return pd;
}

}  // namespace

void launch_table_df(Ctx& c) {
    k_table_df<<<mesh_blocks(c), THREADS, 0, c.stream>>>(c.m.ncell, c.table, reinterpret_cast<float4*>(c.table_pair));
    ++c.launches;
}

void launch_push_df(Ctx& c, const double* vit, double* vnew, double* Jnext) {
    const bool det = c.cfg.deterministic != 0;
    cudaMemsetAsync(c.creep_count, 0, 2 * sizeof(int), c.stream);   // count, k_local queue head
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>((c.np + THREADS - 1) / THREADS, (int64_t)c.sms * c.push_bps));
    nb = std::min(nb, MAX_BLOCKS);
    k_push_df<<<nb, THREADS, 0, c.stream>>>(make_params_df(c), c.xi, c.v, c.P, vit,
                                            reinterpret_cast<const float4*>(c.table_pair), vnew, Jnext, c.creep_list,
                                            c.creep_count, det ? c.creep_flag : nullptr, c.slide, c.partials,
                                            c.dev_status);
    ++c.launches;
}

}  // namespace pic
