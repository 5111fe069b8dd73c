// Device helpers shared by the FP64 push (particles.cu) and the FP32-pair push
// (particles_df.cu): the ordering of a chunk's particles by orbit-piece count, the per-particle
// slide byte, the slow-particle gate of the particle-local solves, and the per-block partials.
#pragma once

#include "pic_internal.h"

namespace pic {

constexpr uint8_t SLIDE_CREPT = 8;    // slide-byte bit 3: solved locally earlier in this step
constexpr double SLOW_RATIO = 0.25;   // a plain particle whose change did not shrink below this
                                      // of the previous one (and exceeds the launch's floor
                                      // times its speed) is solved locally from then on

// Orbit-piece classes for ordering the particles of a chunk: 1, 2, 3, >= 4 pieces, and a
// last class for the threads past the end of the particle array.
constexpr int PIECE_CLASSES = 5;

// Estimated number of pieces of an orbit x0 + s beta (1 + knots crossed), in FP32: only the
// order of the work depends on it, never a result.
__device__ __forceinline__ int piece_class_of(const StepParams& p, const double x0[3], const double beta[3]) {
    int pieces = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = (float)(x0[a] - p.koff);
        const float b = (float)beta[a];
        pieces += abs((int)floorf(x + b) - (int)floorf(x));
    }
    return min(pieces, PIECE_CLASSES - 1) - 1;
}

// The same for particle j under the iterate vit.
__device__ __forceinline__ int piece_class(const StepParams& p, const double* __restrict__ xi,
                                           const double* __restrict__ v, const double* __restrict__ vit, int64_t j) {
    const int64_t np = p.np;
    double x0[3], beta[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x0[a] = xi[a * np + j];
        beta[a] = p.dt * 0.5 * (vit[a * np + j] + v[a * np + j]) * p.invH[a];
    }
    return piece_class_of(p, x0, beta);
}

// Position of this thread's item in the block when items are ordered by class (stable: equal
// classes keep the thread order).  Uses wcount as scratch; ends with a barrier.
__device__ __forceinline__ int stable_class_rank(int cls, int (*wcount)[PIECE_CLASSES]) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned mine = 0;
#pragma unroll
    for (int c = 0; c < PIECE_CLASSES; ++c) {
        const unsigned m = __ballot_sync(0xffffffffu, cls == c);
        if (lane == 0) wcount[w][c] = __popc(m);
        if (cls == c) mine = m;
    }
    __syncthreads();
    int pos = __popc(mine & ((1u << lane) - 1u));
    for (int c = 0; c < cls; ++c)
        for (int v = 0; v < nw; ++v) pos += wcount[v][c];
    for (int v = 0; v < w; ++v) pos += wcount[v][cls];
    __syncthreads();
    return pos;
}

template <typename T>
__device__ __forceinline__ void write_partial(double* partials, int slot, double v, double* sm, bool is_max) {
    double r = is_max ? block_max(v, sm) : block_sum(v, sm);
    if (threadIdx.x == 0) partials[slot * MAX_BLOCKS + blockIdx.x] = r;
}

}  // namespace pic
