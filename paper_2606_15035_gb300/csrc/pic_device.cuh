// Device-side building blocks of the orbit-averaged particle step (sm_103a).
//
// Positions are carried in cell units (xi = x / H per axis), so the knots of the
// tensor-product linear B-spline (r = 1, the shape of the paper's §5.4 test) are the
// integers and the mesh node g sits at integer coordinates.  A particle orbit over one
// step is the straight segment xi(s) = xi0 + s * beta, 0 <= s <= 1, with beta the
// unwrapped displacement in cell units (§4.2, Eq. (particle-orbit)).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pic {

// Error bits set in the device status word (read by the host at sync points).
enum : int {
    DEV_ERR_SEGMENTS = 1,   // more knot crossings in one step than MAX_SEGMENTS allows
    DEV_ERR_NONFINITE = 2,  // a non-finite velocity or residual appeared
    DEV_ERR_TILE = 4,       // an orbit left the mesh tile computed for its block (not expected)
    DEV_ERR_TIMEOUT = 8,    // a bounded wait on an asynchronous copy gave up
    DEV_ERR_RANGE = 16,     // a deposit beyond the exact accumulator's range (deterministic mode)
};

constexpr int MAX_SEGMENTS = 64;

struct MeshDims {
    int n[3];       // nodes per axis
    int64_t ncell;  // n0 * n1 * n2
};

__device__ __forceinline__ int wrapi(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

// Row index of node (ix, iy, iz) in the x-fastest mesh layout.
__device__ __forceinline__ int64_t node_index(int ix, int iy, int iz, const MeshDims& m) {
    return (int64_t)ix + (int64_t)m.n[0] * ((int64_t)iy + (int64_t)m.n[1] * iz);
}

// Wrap any position onto [0, n) (initial data).
template <typename T>
__device__ __forceinline__ T wrap_pos_any(T x, T n) {
    T w = x - n * floor(x / n);
    return w >= n ? w - n : w;
}

// Wrap onto [0, n) a position that is less than one box length outside it (an orbit
// moves far less than n cells per step).
template <typename T>
__device__ __forceinline__ T wrap_pos(T x, T n) {
    T w = x < T(0) ? x + n : (x >= n ? x - n : x);
    return w >= n ? w - n : (w < T(0) ? T(0) : w);
}

// One knot-free piece [s0, s0 + h] of an orbit: the stencil cell containing its midpoint
// and the normalised start coordinate r_{a,m} in that cell (Appendix A).
template <typename T>
struct Segment {
    T s0, h;
    int cell[3];
    T r[3];
};

// Visit the pieces of the orbit xi0 + s * beta between consecutive breakpoints.
// The breakpoints are {0, 1} and every s in (0, 1) at which some axis crosses a knot
// (§4.7, Eq. (breakpoint-set)); the three per-axis crossing sequences are already
// sorted, so they are merged on the fly.  Coincident crossings produce one breakpoint;
// an axis with beta_a = 0 contributes none.  With split = false the whole path [0, 1]
// is one piece; that form is only used with the Gauss rule (the unsplit comparison run
// of §5.4), whose samples find their own cell, so seg.cell / seg.r are not used then.
// Returns the number of pieces, or -1 if MAX_SEGMENTS was exceeded.
template <typename T, typename F>
__device__ __forceinline__ int for_each_segment(const T xi0[3], const T beta[3], bool split, F&& visit) {
    T snext[3], knot[3], step[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        snext[a] = T(2);
        knot[a] = T(0);
        step[a] = T(0);
        // the division is only needed when the orbit reaches the first knot ahead
        if (split && beta[a] > T(0)) {
            knot[a] = floor(xi0[a]) + T(1);
            step[a] = T(1);
            if (knot[a] - xi0[a] < beta[a]) snext[a] = (knot[a] - xi0[a]) / beta[a];
        } else if (split && beta[a] < T(0)) {
            knot[a] = ceil(xi0[a]) - T(1);
            step[a] = T(-1);
            if (knot[a] - xi0[a] > beta[a]) snext[a] = (knot[a] - xi0[a]) / beta[a];
        }
        if (!(snext[a] < T(1))) snext[a] = T(2);
    }
    T s0 = T(0);
    for (int it = 0; it < MAX_SEGMENTS; ++it) {
        T s1 = fmin(fmin(snext[0], snext[1]), fmin(snext[2], T(1)));
        T h = s1 - s0;
        if (h > T(0)) {
            Segment<T> seg;
            seg.s0 = s0;
            seg.h = h;
            T mid = T(0.5) * (s0 + s1);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                T c = floor(xi0[a] + mid * beta[a]);
                seg.cell[a] = (int)c;
                seg.r[a] = xi0[a] + s0 * beta[a] - c;
            }
            visit(seg);
        }
        if (s1 >= T(1)) return it + 1;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (snext[a] == s1) {
                knot[a] += step[a];
                const T dk = knot[a] - xi0[a];
                T sn = (beta[a] > T(0) ? dk < beta[a] : dk > beta[a]) ? dk / beta[a] : T(2);
                snext[a] = sn < T(1) ? sn : T(2);
            }
        }
        s0 = s1;
    }
    return -1;
}

// Per-axis linear weights on a piece: w_{a,0}(eta) = L0 + M0 eta, w_{a,1} = L1 + M1 eta,
// with L0 = 1 - r, M0 = -beta, L1 = r, M1 = beta (Appendix A).
template <typename T>
struct AxisPoly {
    T L[2], M[2];
};

template <typename T>
__device__ __forceinline__ AxisPoly<T> axis_poly(T r, T beta) {
    AxisPoly<T> p;
    p.L[0] = T(1) - r;
    p.M[0] = -beta;
    p.L[1] = r;
    p.M[1] = beta;
    return p;
}

// Quadratic product (La + Ma eta)(Lb + Mb eta) = d0 + d1 eta + d2 eta^2.
template <typename T>
struct Quad {
    T d0, d1, d2;
};

template <typename T>
__device__ __forceinline__ Quad<T> quad_product(T La, T Ma, T Lb, T Mb) {
    Quad<T> q;
    q.d0 = La * Lb;
    q.d1 = Ma * Lb + La * Mb;
    q.d2 = Ma * Mb;
    return q;
}

// I_nu = int_0^h (c0 + c1 eta + c2 eta^2 + c3 eta^3) d eta with the cubic being the
// product of a quadratic (two axes) and a linear factor (third axis) (Appendix A).
template <typename T>
__device__ __forceinline__ T segment_weight(const Quad<T>& q, T L, T M, T h) {
    T c0 = q.d0 * L;
    T c1 = q.d1 * L + q.d0 * M;
    T c2 = q.d2 * L + q.d1 * M;
    T c3 = q.d2 * M;
    return h * (c0 + h * (c1 * T(0.5) + h * (c2 * (T(1) / T(3)) + h * (c3 * T(0.25)))));
}

// The two bracketed integrals of I^D (Appendix B) for a transverse quadratic d:
// T0 = int_0^h d(eta) d eta, T1 = int_0^h eta d(eta) d eta.
template <typename T>
__device__ __forceinline__ void transverse_integrals(const Quad<T>& q, T h, T& t0, T& t1) {
    t0 = h * (q.d0 + h * (q.d1 * T(0.5) + h * (q.d2 * (T(1) / T(3)))));
    t1 = h * h * (q.d0 * T(0.5) + h * (q.d1 * (T(1) / T(3)) + h * (q.d2 * T(0.25))));
}

// Eight closed-form weights I_nu of one piece, nu = nx + 2 ny + 4 nz (Appendix A).
template <typename T>
__device__ __forceinline__ void segment_weights8(const Segment<T>& sg, const T beta[3], T I[8]) {
    AxisPoly<T> px = axis_poly(sg.r[0], beta[0]);
    AxisPoly<T> py = axis_poly(sg.r[1], beta[1]);
    AxisPoly<T> pz = axis_poly(sg.r[2], beta[2]);
#pragma unroll
    for (int ny = 0; ny < 2; ++ny)
#pragma unroll
        for (int nx = 0; nx < 2; ++nx) {
            Quad<T> qxy = quad_product(px.L[nx], px.M[nx], py.L[ny], py.M[ny]);
#pragma unroll
            for (int nz = 0; nz < 2; ++nz) I[nx + 2 * ny + 4 * nz] = segment_weight(qxy, pz.L[nz], pz.M[nz], sg.h);
        }
}

// Base integrals of one piece.  With w_a(eta) = r_a + beta_a eta the "upper" linear weight
// of axis a (w_{a,1} of Appendix A; w_{a,0} = 1 - w_a):
//   S1[a] = int_0^h w_a,   E1[a] = int_0^h eta w_a,
//   S2[j] = int_0^h w_p w_q,   E2[j] = int_0^h eta w_p w_q   ((p, q) = the axes other than j),
//   S3 = int_0^h w_x w_y w_z.
// Every closed-form integral of Appendices A and B is a signed sum of these, because each
// w_{a,0} = 1 - w_{a,1} (inclusion--exclusion).
template <typename T>
struct PieceInts {
    T h, S1[3], E1[3], S2[3], E2[3], S3;
};

template <typename T>
__device__ __forceinline__ PieceInts<T> piece_integrals(const Segment<T>& sg, const T beta[3], bool with_eta) {
    PieceInts<T> I;
    const T h = sg.h, h2 = h * h, h3 = h2 * h;
    I.h = h;
    const T c2 = T(0.5), c3 = T(1) / T(3), c4 = T(0.25);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        I.S1[a] = sg.r[a] * h + beta[a] * (c2 * h2);
        I.E1[a] = with_eta ? sg.r[a] * (c2 * h2) + beta[a] * (c3 * h3) : T(0);
    }
    T d0[3], d1[3], d2[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int p = j == 0 ? 1 : 0, q = j == 2 ? 1 : 2;
        d0[j] = sg.r[p] * sg.r[q];
        d1[j] = sg.r[p] * beta[q] + beta[p] * sg.r[q];
        d2[j] = beta[p] * beta[q];
        I.S2[j] = h * (d0[j] + h * (c2 * d1[j] + h * (c3 * d2[j])));
        I.E2[j] = with_eta ? h2 * (c2 * d0[j] + h * (c3 * d1[j] + h * (c4 * d2[j]))) : T(0);
    }
    // w_x w_y w_z = (d0 + d1 eta + d2 eta^2)_{xy} (r_z + beta_z eta)
    const T e0 = d0[2] * sg.r[2];
    const T e1 = d1[2] * sg.r[2] + d0[2] * beta[2];
    const T e2 = d2[2] * sg.r[2] + d1[2] * beta[2];
    const T e3 = d2[2] * beta[2];
    I.S3 = h * (e0 + h * (c2 * e1 + h * (c3 * e2 + h * (c4 * e3))));
    return I;
}

// The eight weights I_nu of Appendix A from the base integrals, nu = nx + 2 ny + 4 nz.
template <typename T>
__device__ __forceinline__ void weights_from_ints(const PieceInts<T>& I, T W[8]) {
    const T Sx = I.S1[0], Sy = I.S1[1], Sz = I.S1[2];
    const T Syz = I.S2[0], Sxz = I.S2[1], Sxy = I.S2[2], Sxyz = I.S3;
    W[7] = Sxyz;                       // (1,1,1)
    W[3] = Sxy - Sxyz;                 // (1,1,0)
    W[5] = Sxz - Sxyz;                 // (1,0,1)
    W[6] = Syz - Sxyz;                 // (0,1,1)
    W[1] = Sx - Sxy - W[5];            // (1,0,0)
    W[2] = Sy - Syz - W[3];            // (0,1,0)
    W[4] = Sz - Sxz - W[6];            // (0,0,1)
    W[0] = I.h - Sx - Sy - Sz + Sxy + Sxz + Syz - Sxyz;   // (0,0,0)
}

template <typename T>
__device__ __forceinline__ void segment_nodes8(const Segment<T>& sg, const MeshDims& m, int64_t g[8]) {
    int x0 = wrapi(sg.cell[0], m.n[0]), x1 = wrapi(sg.cell[0] + 1, m.n[0]);
    int y0 = wrapi(sg.cell[1], m.n[1]), y1 = wrapi(sg.cell[1] + 1, m.n[1]);
    int z0 = wrapi(sg.cell[2], m.n[2]), z1 = wrapi(sg.cell[2] + 1, m.n[2]);
    g[0] = node_index(x0, y0, z0, m);
    g[1] = node_index(x1, y0, z0, m);
    g[2] = node_index(x0, y1, z0, m);
    g[3] = node_index(x1, y1, z0, m);
    g[4] = node_index(x0, y0, z1, m);
    g[5] = node_index(x1, y0, z1, m);
    g[6] = node_index(x0, y1, z1, m);
    g[7] = node_index(x1, y1, z1, m);
}

// Point value of the 8 linear B-splines around a wrapped position (Eq. (Ah-mesh)).
template <typename T>
__device__ __forceinline__ void point_weights8(const T xi[3], const MeshDims& m, int64_t g[8], T w[8]) {
    int c[3];
    T r[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        T f = floor(xi[a]);
        c[a] = (int)f;
        r[a] = xi[a] - f;
    }
    Segment<T> sg;
    sg.cell[0] = c[0];
    sg.cell[1] = c[1];
    sg.cell[2] = c[2];
    segment_nodes8(sg, m, g);
#pragma unroll
    for (int nz = 0; nz < 2; ++nz)
#pragma unroll
        for (int ny = 0; ny < 2; ++ny)
#pragma unroll
            for (int nx = 0; nx < 2; ++nx) {
                T wx = nx ? r[0] : T(1) - r[0];
                T wy = ny ? r[1] : T(1) - r[1];
                T wz = nz ? r[2] : T(1) - r[2];
                w[nx + 2 * ny + 4 * nz] = wx * wy * wz;
            }
}

// ---- exact, order-independent accumulation (deterministic mode) --------------------------
//
// A deposit x is added as the integer N = round(x / u), u a power of two, split into
// N = hi * 2^40 + lo with 0 <= lo < 2^40; hi and lo go to two 64-bit integer accumulators.
// Integer addition is associative, so the sums do not depend on the order in which threads
// add, and the only rounding is that of each x to a multiple of u.  u is chosen from a bound W
// on the sum of |x| over all deposits to one entry, u = 2^(ceil(log2 W) - 102): then every
// |hi| sum stays below 2^63 and u / |x| is ~1e-21 for a typical deposit.
struct ExactAcc {
    long long* hi;    // one per entry
    long long* lo;
    double inv_u;     // 1 / u
    int* status;
};

__device__ __forceinline__ void exact_add(const ExactAcc& a, int64_t idx, double x) {
    const double t = x * a.inv_u;                       // exact: scaling by a power of two
    if (!(fabs(t) < 0x1p100)) {
        atomicOr(a.status, DEV_ERR_RANGE);
        return;
    }
    const double h = floor(t * 0x1p-40);                // exact
    const double l = t - h * 0x1p40;                    // in [0, 2^40], exact for |t| >= 2^40
    atomicAdd(reinterpret_cast<unsigned long long*>(a.hi + idx), (unsigned long long)(long long)h);
    atomicAdd(reinterpret_cast<unsigned long long*>(a.lo + idx), (unsigned long long)llrint(l));
}

// ---- "creeping" orbits --------------------------------------------------------------------

constexpr double BETA_CREEP = 0.1;   // cells
constexpr double D_KNOT = 1e-11;     // cells: starting this close to a knot also counts (and is
                                     // probed for sliding: about the rounding of a position
                                     // landed on a knot, with margin)

// On an axis where the orbit moves less than BETA_CREEP cells, does it get within 2 |beta|
// of the next knot ahead, or start within D_KNOT of any knot?  Those orbits cross a knot
// while barely moving, nearly do, or hover on a knot (an iterate can flip between
// crossing and not crossing).
__device__ __forceinline__ bool is_creeping(const double x0[3], const double beta[3]) {
    bool f = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double b = beta[a];
        const double d = b > 0.0 ? floor(x0[a]) + 1.0 - x0[a] : x0[a] - (ceil(x0[a]) - 1.0);
        const double near = fmin(x0[a] - floor(x0[a]), ceil(x0[a]) - x0[a]);
        f |= (fabs(b) < BETA_CREEP) && (((b != 0.0) && (d < 2.0 * fabs(b))) || (near < D_KNOT));
    }
    return f;
}

// ---- block reductions (fixed order, so results are reproducible for a fixed launch) ----

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Sum over the block; the result is valid in thread 0.  blockDim.x <= 1024.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* smem32) {
    v = warp_sum(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem32[wid] = v;
    __syncthreads();
    T r = T(0);
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? smem32[lane] : T(0);
        r = warp_sum(r);
    }
    return r;
}

template <typename T>
__device__ __forceinline__ T block_max(T v, T* smem32) {
    v = warp_max(v);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) smem32[wid] = v;
    __syncthreads();
    T r = T(0);
    if (wid == 0) {
        int nw = (blockDim.x + 31) >> 5;
        r = lane < nw ? smem32[lane] : T(0);
        r = warp_max(r);
    }
    return r;
}

}  // namespace pic
