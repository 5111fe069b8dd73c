// FP32 particle kernels of the mixed-precision Picard iterations (sm_103a).
//
// The mixed path runs the first Picard iterations of Algorithm 1 in single precision: the
// orbit breakpoints, the Appendix A/B orbit integrals, the gather, the canonical-momentum
// push and the orbit current are computed in FP32 from an FP32 working set, while the mesh
// solve (continuity, Crank--Nicolson), the reductions and the accumulation of J stay FP64.
// The FP64 kernels then refine the iterate to the FP64 tolerance and run the final sweep, so
// the accepted step is a solution of the FP64 discrete equations.
//
// FP32 working set (device order, structure of arrays, component stride `stride`):
//   cell[i]   packed cell index cx | cy << 10 | cz << 20 of the particle's start position;
//   off[c,i]  offset of the start position inside that cell, in [0, 1) (cell units);
//   v         v^n rounded to FP32;
//   vit, vnew the Picard iterates as increments dv = v^{n+1,p} - v^n.
// Positions relative to the cell keep ~1e-7-cell resolution for the knot tests at any mesh size.
// The iterates are increments because the push can produce them without P^n: the level-n
// canonical momentum is P^n = m v^n + q A_h^n(x^n) (Eq. (orbit-push)), so
//   m (v^{n+1} - v^n) = dt q (-grad phi_bar + (D A)^T v_bar) - q [A_h^{n+1}(x^{n+1}) - A_h^n(x^n)],
// and every FP32 rounding then scales with the small increment instead of with v itself.
#include <algorithm>
#include <climits>
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
    int64_t stride;   // component stride of the FP32 particle arrays (a multiple of CHUNK32)
    int det;          // deterministic mode: FP64 deposits go to acc (exact, order independent)
    ExactAcc acc;
    long long wait_cycles;   // bound of each wait for a chunk's bulk copies (SM clock cycles)
};

template <typename T>
__device__ __forceinline__ void write_partial32(double* partials, int slot, double v, double* sm) {
    double r = block_sum(v, sm);
    if (threadIdx.x == 0) partials[slot * MAX_BLOCKS + blockIdx.x] = r;
}

// ---- mesh access: the block's shared-memory tile, or the global arrays -------------------
//
// The particles are sorted by start cell, so the orbits of one chunk of consecutive
// particles touch a small box of mesh nodes.  The box is found per chunk by a block
// reduction (in node coordinates relative to the chunk's first cell, minimal image per
// periodic axis); when it fits TILE_CAP nodes, the chunk gathers A^n, A^{n+1} and
// grad_h phi from a shared-memory copy of the box and accumulates its orbit current in a
// shared fixed-point tile that is added to the FP64 J once per chunk.  Chunks whose box does
// not fit (very fast or scattered particles) use the global arrays directly.

constexpr int TILE_CAP = 320;  // nodes of a block's mesh tile
constexpr int CHUNK32 = 256;   // particles per chunk = threads per block
constexpr int PUSH32_MINB = 4; // resident blocks per SM the FP32 push is compiled for (64 registers)

struct Box {
    int lo[3];   // lowest node, relative to the chunk's reference cell
    int ex, exy; // extents: x, x*y
    int ext[3];
    int vol;
};

// Minimal-image offset of cell c from cell ref on a periodic axis of n cells.
__device__ __forceinline__ int rel_cell(int c, int ref, int n) {
    int d = c - ref;
    if (2 * d > n) d -= n;
    else if (2 * d < -n) d += n;
    return d;
}

// Node range [lo, hi] touched by the orbit x0 + s beta (0 <= s <= 1) of a particle whose
// cell sits at offset co from the reference cell: its pieces' stencil cells are floors of
// points on the orbit and the linear stencil of cell c is the nodes c, c + 1.
__device__ __forceinline__ void orbit_node_range(const int co[3], const float x0[3], const float beta[3], int lo[3],
                                                 int hi[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xe = x0[a] + beta[a];
        lo[a] = co[a] + (int)floorf(fminf(x0[a], xe));
        hi[a] = co[a] + (int)floorf(fmaxf(x0[a], xe)) + 1;
    }
}

// Bounding box of the block's node ranges and the block maxima of amax[3] (non-negative
// floats, reduced through their bit patterns); sm: 9 * 32 + 9 ints.  Every thread gets the
// result.
__device__ __forceinline__ Box block_box(int lo[3], int hi[3], float amax[3], int* sm) {
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
    Box b;
    int64_t vol = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        b.lo[a] = sm[288 + a];
        b.ext[a] = sm[291 + a] - b.lo[a] + 1;
        vol *= b.ext[a] > 0 ? b.ext[a] : 0;
        amax[a] = __int_as_float(sm[294 + a]);
    }
    const bool fits = vol <= TILE_CAP;
    b.ex = fits ? b.ext[0] : 0;
    b.exy = fits ? b.ext[0] * b.ext[1] : 0;
    b.vol = fits ? (int)vol : TILE_CAP + 1;
    return b;
}

// Local index of the lowest node of cell c (relative coordinates) in the tile; false if any
// of the cell's 8 nodes lies outside the box.
__device__ __forceinline__ bool tile_cell(const Box& b, const int c[3], int& base) {
    const int lx = c[0] - b.lo[0], ly = c[1] - b.lo[1], lz = c[2] - b.lo[2];
    base = lx + b.ex * ly + b.exy * lz;
    return lx >= 0 && ly >= 0 && lz >= 0 && lx + 1 < b.ext[0] && ly + 1 < b.ext[1] && lz + 1 < b.ext[2];
}

__device__ __forceinline__ int tile_off(const Box& b, int k) {
    return (k & 1) + ((k >> 1) & 1) * b.ex + (k >> 2) * b.exy;
}

// Global row of tile node l (wrapped onto the periodic mesh).
__device__ __forceinline__ int64_t tile_global(const Box& b, const int ref[3], const MeshDims& m, int l) {
    const int lz = l / b.exy, r = l - lz * b.exy, ly = r / b.ex, lx = r - ly * b.ex;
    return node_index(wrapi(ref[0] + b.lo[0] + lx, m.n[0]), wrapi(ref[1] + b.lo[1] + ly, m.n[1]),
                      wrapi(ref[2] + b.lo[2] + lz, m.n[2]), m);
}

// Nearest integer to x * scale for |x * scale| < 2^22: adding 1.5 * 2^23 puts the rounded
// integer in the low mantissa bits (the sum lies in [2^23, 2^24), where the spacing is 1).
__device__ __forceinline__ int to_fixed(float x, float scale) {
    return __float_as_int(fmaf(x, scale, 12582912.0f)) - 0x4B400000;
}

// Power-of-two scale of one component of the fixed-point current tile: every contribution
// |w_a| * I_nu (I_nu <= 1) of a chunk whose largest |w_a| is amax maps below 2^21 in
// magnitude, so a node's sum over the chunk stays below CHUNK32 * 2^21 <= 2^30.  Each
// component has its own scale (the transverse currents of a beam are far smaller).
__device__ __forceinline__ float fixed_scale(float amax) {
    int e = 0;
    frexpf(amax, &e);                 // amax < 2^e
    e = max(e, -100);
    return ldexpf(1.f, 21 - e);
}

// Mesh view of one chunk.  TILED: cells are relative to the reference cell and the table
// and current live in shared memory; otherwise cells are absolute (wrapped here) and the
// global table / FP64 current are used.
template <bool TILED>
struct MeshView {
    const float4* tab;   // 3 float4 per node
    int* jt;             // TILED: 3 x TILE_CAP current in fixed point (units of 1 / jscale[a])
    float jscale[3];     // TILED: per component, a power of two with |contribution| * jscale < 2^21
    double* J;           // !TILED: FP64 current, 3 x N
    ExactAcc acc;        // !TILED, deterministic mode: exact accumulator of J
    int det;
    Box box;
    MeshDims m;
    int* status;

    __device__ __forceinline__ bool nodes8(const int c[3], int g[8], int64_t gg[8]) const {
        if (TILED) {
            int base;
            const bool ok = tile_cell(box, c, base);
#pragma unroll
            for (int k = 0; k < 8; ++k) g[k] = base + tile_off(box, k);
            if (!ok) atomicOr(status, DEV_ERR_TILE);
            return ok;
        } else {
            Segment<float> s;
            s.cell[0] = c[0];
            s.cell[1] = c[1];
            s.cell[2] = c[2];
            segment_nodes8(s, m, gg);
            return true;
        }
    }
    __device__ __forceinline__ const float4* node(const int g[8], const int64_t gg[8], int k) const {
        return TILED ? tab + 3 * g[k] : tab + 3 * gg[k];
    }
    __device__ __forceinline__ void add(const int g[8], const int64_t gg[8], int k, float w0, float w1, float w2) const {
        if (TILED) {
            atomicAdd(jt + g[k], to_fixed(w0, jscale[0]));
            atomicAdd(jt + TILE_CAP + g[k], to_fixed(w1, jscale[1]));
            atomicAdd(jt + 2 * TILE_CAP + g[k], to_fixed(w2, jscale[2]));
        } else if (det) {
            exact_add(acc, gg[k], (double)w0);
            exact_add(acc, m.ncell + gg[k], (double)w1);
            exact_add(acc, 2 * m.ncell + gg[k], (double)w2);
        } else {
            atomicAdd(J + gg[k], (double)w0);
            atomicAdd(J + m.ncell + gg[k], (double)w1);
            atomicAdd(J + 2 * m.ncell + gg[k], (double)w2);
        }
    }
};

// Orbit current of one FP32 orbit (closed form, Appendix A): q v_bar S_bar / dV per node.
template <bool TILED>
__device__ __forceinline__ int scatter32(const MeshView<TILED>& mv, const int co[3], const float x0[3],
                                         const float beta[3], const float w[3]) {
    return for_each_segment(x0, beta, true, [&](const Segment<float>& sg) {
        float I[8];
        weights_from_ints(piece_integrals(sg, beta, false), I);
        const int c[3] = {co[0] + sg.cell[0], co[1] + sg.cell[1], co[2] + sg.cell[2]};
        int g[8];
        int64_t gg[8];
        if (!mv.nodes8(c, g, gg)) return;
        if (TILED) {
            // lane-dependent node order: lanes of one cell add to different nodes at each step
            const int r = threadIdx.x & 7;
#pragma unroll
            for (int bit = 1; bit < 8; bit <<= 1) {
                const bool sw = (r & bit) != 0;
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (k & bit) continue;
                    const float a0 = I[k], a1 = I[k | bit];
                    I[k] = sw ? a1 : a0;
                    I[k | bit] = sw ? a0 : a1;
                    const int g0 = g[k], g1 = g[k | bit];
                    g[k] = sw ? g1 : g0;
                    g[k | bit] = sw ? g0 : g1;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) mv.add(g, gg, k, w[0] * I[k], w[1] * I[k], w[2] * I[k]);
    });
}

// G(u) in FP32: the orbit push of Algorithm 1 with the FP32 gather table
// (per node: A^n (3), A^{n+1} (3), grad_h phi^{n+1/2} (3), 3 unused).  Returns the
// velocity increment dv = v^{n+1} - v^n of the pushed particle (see the file comment).
template <bool TILED>
__device__ __forceinline__ int push32(const Params32& p, const MeshView<TILED>& mv, const int co[3], const float x0[3],
                                      const float beta[3], const float vb[3], float dv[3]) {
    float gphi[3] = {0.f, 0.f, 0.f}, F[3] = {0.f, 0.f, 0.f};
    const int nseg = for_each_segment(x0, beta, true, [&](const Segment<float>& sg) {
        const PieceInts<float> I = piece_integrals(sg, beta, true);
        float W[8];
        weights_from_ints(I, W);
        const int c[3] = {co[0] + sg.cell[0], co[1] + sg.cell[1], co[2] + sg.cell[2]};
        int g[8];
        int64_t gg[8];
        if (!mv.nodes8(c, g, gg)) return;
        const float s = sg.s0, oms = 1.f - s, h = sg.h, hh2 = 0.5f * h * h;
        float am[8], cc[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float4* t4 = mv.node(g, gg, k);
            const float4 a = t4[0], b = t4[1], c4 = t4[2];
            const float an = a.x * vb[0] + a.y * vb[1] + a.z * vb[2];
            const float a1 = a.w * vb[0] + b.x * vb[1] + b.y * vb[2];
            am[k] = oms * an + s * a1;
            cc[k] = a1 - an;
            gphi[0] += W[k] * b.z;
            gphi[1] += W[k] * b.w;
            gphi[2] += W[k] * c4.x;
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
    // dA = A_h^{n+1}(x^{n+1}) - A_h^n(x^n): point interpolants at the end and start points
    float dA[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int end = 0; end < 2; ++end) {
        int ce[3];
        float r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float xe = end ? x0[a] + beta[a] : x0[a];
            const float f = floorf(xe);
            ce[a] = co[a] + (int)f;
            r[a] = xe - f;
        }
        int g[8];
        int64_t gg[8];
        if (!mv.nodes8(ce, g, gg)) continue;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float wx = (k & 1) ? r[0] : 1.f - r[0], wy = (k & 2) ? r[1] : 1.f - r[1];
            const float wz = (k & 4) ? r[2] : 1.f - r[2];
            const float w = wx * wy * wz;
            const float4* t4 = mv.node(g, gg, k);
            const float4 a = t4[0];
            if (end) {
                const float4 b = t4[1];
                dA[0] += w * a.w;
                dA[1] += w * b.x;
                dA[2] += w * b.y;
            } else {
                dA[0] -= w * a.x;
                dA[1] -= w * a.y;
                dA[2] -= w * a.z;
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) dv[a] = (p.dt * (p.q * (F[a] - gphi[a])) - p.q * dA[a]) * p.inv_mass;
    return nseg;
}

// Copy the box's nodes of the global FP32 table into the shared tile.
__device__ __forceinline__ void load_tile(const Box& b, const int ref[3], const MeshDims& m,
                                          const float4* __restrict__ table, float4* tab) {
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
        const int64_t g = tile_global(b, ref, m, l);
        tab[3 * l] = __ldg(table + 3 * g);
        tab[3 * l + 1] = __ldg(table + 3 * g + 1);
        tab[3 * l + 2] = __ldg(table + 3 * g + 2);
    }
}

__device__ __forceinline__ void zero_jtile(const Box& b, int* jt) {
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) jt[l] = jt[TILE_CAP + l] = jt[2 * TILE_CAP + l] = 0;
}

// Add the chunk's FP32 current tile to the FP64 J (nodes that received nothing are skipped).
__device__ __forceinline__ void flush_jtile(const Params32& p, const Box& b, const int ref[3], const int* jt,
                                            const float jscale[3], double* __restrict__ J) {
    const MeshDims& m = p.m;
    const double i0 = 1.0 / (double)jscale[0], i1 = 1.0 / (double)jscale[1], i2 = 1.0 / (double)jscale[2];
    for (int l = threadIdx.x; l < b.vol; l += blockDim.x) {
        const int j0 = jt[l], j1 = jt[TILE_CAP + l], j2 = jt[2 * TILE_CAP + l];
        if ((j0 | j1 | j2) == 0) continue;
        const int64_t g = tile_global(b, ref, m, l);
        if (p.det) {
            if (j0 != 0) exact_add(p.acc, g, i0 * j0);
            if (j1 != 0) exact_add(p.acc, m.ncell + g, i1 * j1);
            if (j2 != 0) exact_add(p.acc, 2 * m.ncell + g, i2 * j2);
        } else {
            if (j0 != 0) atomicAdd(J + g, i0 * j0);
            if (j1 != 0) atomicAdd(J + m.ncell + g, i1 * j1);
            if (j2 != 0) atomicAdd(J + 2 * m.ncell + g, i2 * j2);
        }
    }
}

// FP64 masters -> FP32 working set; first iterate v^{n+1,0} = 2 v^n - v^{n-1}, as an increment.
__global__ void k_to32(Params32 p, const double* __restrict__ xi, const double* __restrict__ v,
                       const double* __restrict__ vprev, int32_t* __restrict__ cell, float* __restrict__ off,
                       float* __restrict__ v32, float* __restrict__ vit32, double* __restrict__ partials) {
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
            off[a * p.stride + i] = (float)(x - c);
            packed |= ((int32_t)c & CELL_MASK) << (a * CELL_BITS);
            const double vv = v[a * np + i];
            v32[a * p.stride + i] = (float)vv;
            vit32[a * p.stride + i] = (float)(vv - vprev[a * np + i]);   // (2 v^n - v^{n-1}) - v^n
        }
        cell[i] = packed;
    }
    write_partial32<double>(partials, S_JSCALE, jsc, sm);
}

struct Chunk {
    int ref[3];   // cell of the chunk's first particle
    bool valid;   // this thread holds a particle
    int64_t i;
};

// Slot of thread t in its chunk.  Lanes of one warp take every 8th slot, so they sit in
// different cells of the sorted chunk (their shared-memory current updates rarely collide);
// the rotation by lane / 4 keeps the 32 lanes on 32 different shared-memory banks when they
// read the chunk's staged fields.
__device__ __forceinline__ int chunk_slot(int t) {
    const int l = t & 31, w = t >> 5;
    return 8 * l + ((w + (l >> 2)) & 7);
}

__device__ __forceinline__ Chunk chunk_of(int64_t ch, int64_t np, int32_t ref_cell) {
    Chunk k;
    k.i = ch * CHUNK32 + chunk_slot(threadIdx.x);
    k.valid = k.i < np;
    unpack_cell(ref_cell, k.ref);
    return k;
}

// ---- TMA staging of a chunk's particle fields (cp.async.bulk + mbarrier) ------------------

constexpr int NFIELD = 10;   // cell | offset (3) | v^n (3) | iterate increment (3)
constexpr int F_CELL = 0, F_OFF = 1, F_V = 4, F_IT = 7;
constexpr long long DRAIN_CYCLES = 2000000000LL;  // ~1 s: bound of the wait for the copies still in
                                                  // flight when a block gives up (always the full bound,
                                                  // so that no copy lands after the block has exited)

__device__ __forceinline__ uint32_t smem_u32(const void* ptr) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(ptr));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Order this thread's generic-proxy shared-memory accesses before later bulk copies.
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void bulk_store(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// Has phase `parity` of bar completed?  try_wait may suspend the thread for a while (until
// the phase completes or a hardware time limit passes); test_wait returns at once.
__device__ __forceinline__ bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ bool mbar_poll(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of bar to complete; false once more than `limit` clocks have passed
// without it.  The clock is read before every potentially suspending probe, so a limit
// shorter than the copy's latency gives up at once instead of sleeping through it.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    while (true) {
        if (mbar_poll(bar, parity)) return true;
        if (clock64() - t0 > limit) return false;
        if (mbar_try(bar, parity)) return true;
    }
}

// Bytes copied per field for chunk ch: the chunk's particles rounded up to 16 bytes (the
// arrays are padded to a multiple of CHUNK32 entries, so the rounding stays inside them).
__device__ __forceinline__ uint32_t chunk_bytes(int64_t ch, int64_t np) {
    const int64_t cnt = min((int64_t)CHUNK32, np - ch * CHUNK32);
    return (uint32_t)((cnt * 4 + 15) & ~(int64_t)15);
}

// Issued by one thread: the NFIELD fields of chunk ch into buf, completing on bar.
__device__ __forceinline__ void stage_chunk(const Params32& p, int64_t ch, uint32_t* buf, uint64_t* bar,
                                            const int32_t* cell, const float* off, const float* v32,
                                            const float* vit32) {
    const int64_t base = ch * CHUNK32;
    const uint32_t bytes = chunk_bytes(ch, p.np);
    mbar_arrive_tx(bar, bytes * NFIELD);
    bulk_load(buf + F_CELL * CHUNK32, cell + base, bytes, bar);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int64_t o = a * p.stride + base;
        bulk_load(buf + (F_OFF + a) * CHUNK32, off + o, bytes, bar);
        bulk_load(buf + (F_V + a) * CHUNK32, v32 + o, bytes, bar);
        bulk_load(buf + (F_IT + a) * CHUNK32, vit32 + o, bytes, bar);
    }
}

__device__ __forceinline__ float fld(const uint32_t* S, int f, int j) { return __uint_as_float(S[f * CHUNK32 + j]); }

// Orbit current of one chunk's orbits (x0 + s beta, weights w = q v_bar / dV) into J: through
// the shared tile when the chunk's box fits, else with FP64 atomics on J directly.
__device__ __forceinline__ void chunk_scatter(const Params32& p, const Chunk& k, const int cb[3], const float x0[3],
                                              const float beta[3], const float w[3], int* jt, int* sbox,
                                              double* __restrict__ J, int* __restrict__ status) {
    int co[3], lo[3], hi[3];
    float amax[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) co[a] = rel_cell(cb[a], k.ref[a], p.m.n[a]);
    if (k.valid) {
        orbit_node_range(co, x0, beta, lo, hi);
#pragma unroll
        for (int a = 0; a < 3; ++a) amax[a] = fabsf(w[a]);
    } else {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = INT_MAX;
            hi[a] = INT_MIN;
        }
    }
    const Box b = block_box(lo, hi, amax, sbox);
    if (b.vol <= TILE_CAP && amax[0] < 1e30f && amax[1] < 1e30f && amax[2] < 1e30f) {
        const float js[3] = {fixed_scale(amax[0]), fixed_scale(amax[1]), fixed_scale(amax[2])};
        zero_jtile(b, jt);
        __syncthreads();
        if (k.valid) {
            MeshView<true> mv{nullptr, jt, {js[0], js[1], js[2]}, nullptr, p.acc, p.det, b, p.m, status};
            if (scatter32(mv, co, x0, beta, w) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
        }
        __syncthreads();
        flush_jtile(p, b, k.ref, jt, js, J);
    } else if (k.valid) {
        MeshView<false> mv{nullptr, nullptr, {0.f, 0.f, 0.f}, J, p.acc, p.det, b, p.m, status};
        if (scatter32(mv, cb, x0, beta, w) < 0) atomicOr(status, DEV_ERR_SEGMENTS);
    }
}

// Orbit current of the FP32 iterate (first iteration of the step).
__global__ void __launch_bounds__(CHUNK32) k_scatter32(Params32 p, const int32_t* __restrict__ cell,
                                                       const float* __restrict__ off, const float* __restrict__ v32,
                                                       const float* __restrict__ vit32, double* __restrict__ J,
                                                       int* __restrict__ status) {
    __shared__ int jt[3 * TILE_CAP];
    __shared__ int sbox[9 * 32 + 10];
    const int64_t np = p.np, nchunks = (np + CHUNK32 - 1) / CHUNK32;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        const Chunk k = chunk_of(ch, np, __ldg(cell + ch * CHUNK32));
        int cb[3] = {0, 0, 0};
        float x0[3] = {0.f, 0.f, 0.f}, beta[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f};
        if (k.valid) {
            unpack_cell(cell[k.i], cb);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = off[a * p.stride + k.i];
                const float vb = v32[a * p.stride + k.i] + 0.5f * vit32[a * p.stride + k.i];
                beta[a] = p.dt * vb * p.invH[a];
                w[a] = p.q_dV * vb;
            }
        }
        chunk_scatter(p, k, cb, x0, beta, w, jt, sbox, J, status);
    }
}

// One FP32 Picard iteration: G(v^p), the e_v partial sums, and the orbit current of
// v^{p+1} = G(v^p) into Jnext.  Persistent blocks walk the chunks of CHUNK32 sorted
// particles; while a block works on one chunk, the bulk-copy engine stages the next chunk's
// fields into the other shared buffer, and the new iterate goes back by a bulk store.
__global__ void __launch_bounds__(CHUNK32, PUSH32_MINB) k_push32(Params32 p, const int32_t* __restrict__ cell,
                                                                 const float* __restrict__ off,
                                                                 const float* __restrict__ v32,
                                                                 const float* __restrict__ vit32,
                                                                 const float* __restrict__ table,
                                                                 float* __restrict__ vnew32,
                                                                 double* __restrict__ Jnext,
                                                                 double* __restrict__ partials,
                                                                 int* __restrict__ status) {
    __shared__ __align__(128) uint32_t stage[2][NFIELD * CHUNK32];
    __shared__ float4 tab[3 * TILE_CAP];
    __shared__ int jt[3 * TILE_CAP];
    __shared__ int sbox[9 * 32 + 10];
    __shared__ double sm[32];
    __shared__ __align__(8) uint64_t bar[2];
    const int64_t np = p.np, nchunks = (np + CHUNK32 - 1) / CHUNK32;
    const float4* table4 = reinterpret_cast<const float4*>(table);
    const int tid = threadIdx.x, j = chunk_slot(tid);
    if (tid == 0) {
        mbar_init(&bar[0]);
        mbar_init(&bar[1]);
        fence_mbar_init();
    }
    __syncthreads();
    if (tid == 0 && blockIdx.x < nchunks) stage_chunk(p, blockIdx.x, stage[0], &bar[0], cell, off, v32, vit32);
    float ev_num = 0.f, ev_den = 0.f;
    int it = 0, nchunk = 0, nglobal = 0;
    bool failed = false;
    for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x, ++it) {
        const int b = it & 1;
        const bool more = ch + gridDim.x < nchunks;
        if (tid == 0 && more) {
            bulk_wait_read();      // the previous chunk's iterate store has left the other buffer
            stage_chunk(p, ch + gridDim.x, stage[b ^ 1], &bar[b ^ 1], cell, off, v32, vit32);
        }
        if (!__syncthreads_and(mbar_wait(&bar[b], (it >> 1) & 1, p.wait_cycles))) {
            // a copy did not complete in time: report, let the copies in flight land (with the
            // full bound, whatever p.wait_cycles is), stop this block
            if (tid == 0) {
                atomicOr(status, DEV_ERR_TIMEOUT);
                mbar_wait(&bar[b], (it >> 1) & 1, DRAIN_CYCLES);
                if (more) mbar_wait(&bar[b ^ 1], ((it + 1) >> 1) & 1, DRAIN_CYCLES);
            }
            failed = true;
            break;
        }
        uint32_t* S = stage[b];
        const Chunk k = chunk_of(ch, np, (int32_t)S[F_CELL * CHUNK32]);
        int cb[3] = {0, 0, 0}, co[3], lo[3], hi[3];
        float x0[3] = {0.f, 0.f, 0.f}, vb[3] = {0.f, 0.f, 0.f}, beta[3] = {0.f, 0.f, 0.f};
        if (k.valid) {
            unpack_cell((int32_t)S[F_CELL * CHUNK32 + j], cb);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                x0[a] = fld(S, F_OFF + a, j);
                vb[a] = fld(S, F_V + a, j) + 0.5f * fld(S, F_IT + a, j);
                beta[a] = p.dt * vb[a] * p.invH[a];
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) co[a] = rel_cell(cb[a], k.ref[a], p.m.n[a]);
        if (k.valid) {
            orbit_node_range(co, x0, beta, lo, hi);
        } else {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = INT_MAX;
                hi[a] = INT_MIN;
            }
        }
        float unused[3] = {0.f, 0.f, 0.f};
        const Box bx = block_box(lo, hi, unused, sbox);
        const bool tiled = bx.vol <= TILE_CAP;
        ++nchunk;
        nglobal += tiled ? 0 : 1;
        if (tiled) load_tile(bx, k.ref, p.m, table4, tab);
        __syncthreads();
        float bn[3] = {0.f, 0.f, 0.f}, w[3] = {0.f, 0.f, 0.f};
        if (k.valid) {
            float dv[3];
            int ns;
            if (tiled) {
                MeshView<true> mv{tab, nullptr, {0.f, 0.f, 0.f}, nullptr, p.acc, p.det, bx, p.m, status};
                ns = push32(p, mv, co, x0, beta, vb, dv);
            } else {
                MeshView<false> mv{table4, nullptr, {0.f, 0.f, 0.f}, nullptr, p.acc, p.det, bx, p.m, status};
                ns = push32(p, mv, cb, x0, beta, vb, dv);
            }
            if (ns < 0) atomicOr(status, DEV_ERR_SEGMENTS);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float vn = fld(S, F_V + a, j);
                const float d = dv[a] - fld(S, F_IT + a, j);
                const float vw = vn + dv[a];
                ev_num += d * d;
                ev_den += vw * vw;
                S[(F_IT + a) * CHUNK32 + j] = __float_as_uint(dv[a]);   // staged for the bulk store
                const float vbn = vn + 0.5f * dv[a];
                bn[a] = p.dt * vbn * p.invH[a];
                w[a] = p.q_dV * vbn;
            }
            if (!(isfinite(dv[0]) && isfinite(dv[1]) && isfinite(dv[2]))) atomicOr(status, DEV_ERR_NONFINITE);
        }
        chunk_scatter(p, k, cb, x0, bn, w, jt, sbox, Jnext, status);
        fence_async_smem();   // this thread's accesses to S come before the bulk copies that follow
        __syncthreads();      // the new iterate is complete in S, and S is no longer read
        if (tid == 0) {
            const int64_t base = ch * CHUNK32;
            const uint32_t bytes = chunk_bytes(ch, np);
#pragma unroll
            for (int a = 0; a < 3; ++a) bulk_store(vnew32 + a * p.stride + base, S + (F_IT + a) * CHUNK32, bytes);
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait_all();
    if (failed) return;
    write_partial32<double>(partials, S_EV_NUM, (double)ev_num, sm);
    write_partial32<double>(partials, S_EV_DEN, (double)ev_den, sm);
    if (threadIdx.x == 0) {
        partials[S_CHUNKS32 * MAX_BLOCKS + blockIdx.x] = (double)nchunk;
        partials[S_CHUNKS32_GLOBAL * MAX_BLOCKS + blockIdx.x] = (double)nglobal;
    }
}

// FP64 gather table -> FP32 table (A^n, A^{n+1}, grad phi; 3 unused).
__global__ void k_table32(int64_t N, const double* __restrict__ t64, float* __restrict__ t32) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < N; g += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 9; ++k) t32[12 * g + k] = (float)t64[12 * g + k];
        t32[12 * g + 9] = t32[12 * g + 10] = t32[12 * g + 11] = 0.f;
    }
}

// FP32 iterate increment (component stride `stride`) -> FP64 iterate v^n + dv (stride np).
__global__ void k_from32(int64_t np, int64_t stride, const float* __restrict__ dv, const double* __restrict__ vn,
                         double* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        out[i] = vn[i] + (double)dv[i];
        out[np + i] = vn[np + i] + (double)dv[stride + i];
        out[2 * np + i] = vn[2 * np + i] + (double)dv[2 * stride + i];
    }
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
    p.stride = c.np32;
    p.det = c.cfg.deterministic;
    p.acc = ExactAcc{c.acc_hi, c.acc_lo, c.inv_u_J, c.dev_status};
    p.wait_cycles = c.wait_cycles;
    return p;
}

}  // namespace

void launch_to32(Ctx& c) {
    k_to32<<<particle_blocks(c), THREADS, 0, c.stream>>>(make_params32(c), c.xi, c.v, c.vprev, c.cell32,
                                                         c.off32, c.v32, c.vit32, c.partials);
    ++c.launches;
}

int push32_blocks(const Ctx& c) {
    const int64_t chunks = (c.np + CHUNK32 - 1) / CHUNK32;
    const int64_t cap = std::min<int64_t>((int64_t)c.sms * c.push32_bps, MAX_BLOCKS);
    return (int)std::max<int64_t>(1, std::min(chunks, cap));
}

void launch_scatter32(Ctx& c, double* J) {
    k_scatter32<<<push32_blocks(c), CHUNK32, 0, c.stream>>>(make_params32(c), c.cell32, c.off32, c.v32, c.vit32, J,
                                                              c.dev_status);
    ++c.launches;
    if (c.cfg.deterministic) launch_exact_finish(c, J, 3 * c.m.ncell, c.inv_u_J);
}

void launch_push32(Ctx& c, double* Jnext) {
    k_push32<<<push32_blocks(c), CHUNK32, 0, c.stream>>>(make_params32(c), c.cell32, c.off32, c.v32, c.vit32,
                                                           c.table32, c.vnew32, Jnext, c.partials, c.dev_status);
    ++c.launches;
    if (c.cfg.deterministic) launch_exact_finish(c, Jnext, 3 * c.m.ncell, c.inv_u_J);
}

void launch_table32(Ctx& c) {
    k_table32<<<mesh_blocks(c), THREADS, 0, c.stream>>>(c.m.ncell, c.table, c.table32);
    ++c.launches;
}

void launch_from32(Ctx& c, const float* a, double* b) {
    k_from32<<<particle_blocks(c), THREADS, 0, c.stream>>>(c.np, c.np32, a, c.v, b);
    ++c.launches;
}

}  // namespace pic
