/*
 * pic.h -- C-ABI of the GB300 (sm_103a) energy-conserving unstaggered potential PIC step.
 *
 * The library advances the paper's method (arXiv 2606.15035, "An Energy-Conserving
 * Unstaggered Electromagnetic-Potential Particle-in-Cell Method, Part I"): a periodic box,
 * node-collocated potentials (phi, psi = d_t phi, A, U = d_t A) and charge rho, and
 * electron macro-particles carried by position x, velocity v and canonical momentum
 * P = m v + q A_h(x).  One call to pic_step runs Algorithm 1 ("Picard iteration for the
 * orbit-discrete-gradient CN potential PIC step") per time step:
 *   orbit-averaged current J^{n+1/2} (§4.2, Eq. (orbit-current)) ->
 *   charge from continuity (§3.2, Eq. (cn-continuity)) ->
 *   Crank--Nicolson potential update (§3.2, Eq. (cn-field-update)) ->
 *   orbit gather of grad phi and the orbit-discrete gradient D_i A (§4.3-§4.4,
 *   Eq. (gphibar-definition), Eq. (DA-def), Appendices A/B) ->
 *   canonical-momentum push (§4.4, Eq. (orbit-push)),
 * repeated until the current and velocity fixed-point errors fall below tolerance,
 * followed by one final consistency sweep (§5.4) whose state is committed.
 *
 * Conventions shared by every entry point
 *   - Mesh arrays are float64, x-fastest: node (ix, iy, iz) is element
 *     ix + nx * (iy + ny * iz).  Vector mesh fields are component-major: component c of
 *     node g is element c * ncell + g.
 *   - Particle arrays are float64 structure-of-arrays: component c of particle i is
 *     element c * np + i.  Positions are physical (in [0, L) after wrapping).
 *   - Pointers passed in are borrowed for the duration of the call only.  A flag
 *     `on_device` says whether they are device (1) or host (0) addresses.
 *   - All device work runs on the CUDA stream given to pic_init, in order.  Calls that
 *     return host values synchronise that stream.
 *   - Every call returns a pic_status; none aborts, traps or exits.  After an error,
 *     pic_last_error(ctx) gives a one-line reason.  A pic_step that fails leaves the
 *     state at the last committed step.
 *   - Spatial operators are the periodic second-order central difference D_a and the
 *     Laplacian Delta_h = sum_a D_a D_a, which give the identities the paper's theorems
 *     use (§3.3, §4.6).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pic_ctx pic_ctx;

typedef enum {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,             /* invalid argument or configuration */
    PIC_ERR_OOM = 2,             /* device allocation failed */
    PIC_ERR_CUDA = 3,            /* a CUDA runtime call failed */
    PIC_ERR_NO_CONVERGENCE = 4,  /* Picard reached picard_max without meeting picard_tol */
    PIC_ERR_NONFINITE = 5,       /* a non-finite residual or velocity appeared */
    PIC_ERR_SEGMENTS = 6,        /* an orbit crossed more knots in one step than supported */
    PIC_ERR_INTERNAL = 7,        /* a device-side consistency check failed (a mesh-tile bound) */
    PIC_ERR_TIMEOUT = 8,         /* a bounded device-side wait gave up (an asynchronous copy) */
} pic_status;

enum { PIC_FP64 = 0, PIC_MIXED = 1 };
enum { PIC_QUAD_CLOSED = 0, PIC_QUAD_GAUSS = 1 };

/* Run configuration.  Fill with pic_config_default, then override. */
typedef struct {
    int32_t n[3];                 /* mesh nodes per axis (periodic) */
    double L[3];                  /* box lengths; H_a = L_a / n_a */
    double dt;                    /* time step */
    double kappa, sigma1, sigma2; /* light speed and source coefficients (§2.1); sigma1 = kappa^2 sigma2 */
    double n0;                    /* immobile ion background density (§5.4) */
    double picard_tol;            /* tau: both fixed-point errors must be <= tau (Algorithm 1) */
    int32_t picard_max;           /* p_max: iterations p = 0 .. p_max */
    int32_t split_orbit_at_knots; /* 1: split at every crossed knot (conservative); 0: unsplit (Gauss only) */
    int32_t quadrature;           /* PIC_QUAD_CLOSED (Appendices A/B) or PIC_QUAD_GAUSS (§4.7) */
    int32_t nq;                   /* Gauss points per piece when quadrature = PIC_QUAD_GAUSS (1..16) */
    int32_t precision;            /* PIC_FP64, or PIC_MIXED: the first Picard iterations of each step
                                     in FP32 (orbit integrals, push, scatter; mesh solve and sums in
                                     FP64), then FP64 iterations to picard_tol and the FP64 final
                                     sweep; needs n_a <= 1024 */
    int32_t sort_every;           /* re-sort particles by cell every k steps (0: never) */
    int32_t diagnostics;          /* 1: accumulate the §5.1-§5.3 diagnostics during each step */
    int32_t accept_unconverged;   /* 1: commit a step that hit p_max (Algorithm 1 as printed) */
    int32_t picard_accel;         /* 1: particles whose orbit crosses (or nearly crosses) a knot on
                                     an axis where they move < 0.1 cells, or whose iterate change
                                     stopped shrinking below 1/4 of the previous one, get a
                                     particle-local solve of v = G_i(v) with the iteration's fields
                                     fixed (an accelerated fixed point, §4.8), for the rest of the
                                     step; all others, and every particle when 0, take the plain
                                     update v^{p+1} = G(v^p) of Algorithm 1 */
    double helmholtz_tol;         /* accuracy of the CN Helmholtz solve (Chebyshev, central2): each
                                     mesh phase runs the fewest steps whose error bound is below
                                     helmholtz_tol times the solution's norm, from the warm start's
                                     residual (at most the schedule that reduces any start by it).
                                     On a mesh whose sizes are all 2^p 3^q <= 1024 the central2
                                     solve is by FFT instead, exact per mode (the wide Laplacian's
                                     symbol), and this does not apply to it */
    double mixed_tol32;           /* PIC_MIXED: leave the FP32 iterations once e_v <= this */
    int32_t mixed_max32;          /* PIC_MIXED: at most this many FP32 iterations per step */
    int32_t deterministic;        /* 1: bitwise reproducible steps.  The particle sort is a stable
                                     radix sort, the current and charge deposits are exact sums in
                                     2 x 64-bit fixed point (integer atomics, order independent),
                                     creeping particles are solved in index order and the launch
                                     grids are the defaults (pic_autotune changes nothing).  The
                                     same inputs then give the same bits, run after run and alone
                                     or in an ensemble.  Needs |v| < 100 kappa. */
    int32_t shape_order;          /* B-spline degree r of the particle shape: 1 (default, the
                                     paper's test), 2 or 3 (§4.7, Table 2).  Nodes at the
                                     integers; knots at the integers for odd r and at the
                                     half-integers for even r; orbits are split at those knots.
                                     r > 1 needs quadrature = PIC_QUAD_GAUSS (exact on every
                                     piece when 2 nq - 1 >= 3 r) and precision = PIC_FP64 */
    int32_t ops;                  /* spatial operators: PIC_OPS_CENTRAL2 (default; D_a the central
                                     difference, Delta_h = sum_a D_a D_a) or PIC_OPS_SPECTRAL (the
                                     paper's Fourier operators, §3.3: D_a = i k_a with the Nyquist
                                     symbol zero, Delta_h = -|k|^2; the CN update is then solved
                                     exactly per mode by FFT).  Spectral needs every n_a = 2^p 3^q
                                     <= 1024 */
    double mixed_tol64;           /* PIC_MIXED: the FP64 iterations that follow the FP32 phase stop
                                     once e_v and e_J are both <= this (0: picard_tol).  The step
                                     is still closed by the FP64 final sweep from the accepted
                                     iterate v*, so its energy error is the second-order product
                                     (m / 2) sum_i (v_i^{n+1} - v_i^n) . (G(v*)_i - v*_i) of the
                                     step's velocity change and the fixed-point residual (the
                                     orbit's power balance and the field-energy balance hold
                                     exactly for the orbit of v*, §4.6, §4.8).  When this is > 0
                                     and diagnostics are off, an FP64 iterate v^{p+1} is also
                                     tried as v* directly once its residual is predicted <= this
                                     (from the ratio of residual to current change e_J that earlier
                                     trials measured, else from the contraction of the iterations
                                     so far): the final sweep then measures its own residual
                                     ||G(v*) - v*|| / ||G(v*)|| and commits only if that is <= this
                                     (residual history kind 3); otherwise the FP64 iterations
                                     continue from v^{p+1} */
    int32_t mixed_pair_max;       /* PIC_MIXED: after the FP32 phase, at most this many refinement
                                     iterations whose particle half (orbit integrals, gather, push,
                                     next-orbit current) runs in FP32-pair arithmetic (two floats
                                     per value, a 48-bit significand, on the FP32 pipes) before the
                                     FP64 iterations; they stop early once e_v and e_J are <=
                                     picard_tol or stop shrinking.  An FP32-pair iterate never ends
                                     the step by Algorithm 1's test, but with mixed_tol64 > 0 it
                                     can be tried as v* by the FP64 final sweep, which checks its
                                     residual in FP64.  1 (default): one such iteration, which
                                     replaces the FP64 iteration of the common step (the pair push
                                     costs about 0.85 of the FP64 one at 128^3); 0: FP64 refinement
                                     from the FP32 iterate.  Not used in deterministic mode */
} pic_config;

#define PIC_OPS_CENTRAL2 0
#define PIC_OPS_SPECTRAL 1

/* Initial particles of one species. */
typedef struct {
    int64_t np;       /* number of macro-particles */
    double q, m;      /* charge and mass per macro-particle */
    const double* x;  /* 3 * np positions (SoA, physical units) */
    const double* v;  /* 3 * np velocities (SoA) */
    int32_t on_device;
} pic_particles;

/* Optional device allocator (for example the caller's caching allocator).  When it is
 * absent the library uses cudaMalloc / cudaFree.  `stream` is the context's stream. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, size_t bytes, void* stream, void* user);
    void* user;
} pic_allocator;

typedef struct {
    int32_t steps_done;   /* steps committed by this call */
    int32_t iterations;   /* Picard iterations of the last step (p + 1 at convergence) */
    int32_t converged;    /* 1 if the last step met picard_tol */
    int32_t total_iterations; /* Picard iterations summed over the committed steps */
    double e_v, e_J;      /* the last step's final velocity and current fixed-point errors */
    int32_t iterations_fp32;       /* of the last step's iterations, those run in FP32 (PIC_MIXED) */
    int32_t total_iterations_fp32; /* FP32 iterations summed over the committed steps */
    int32_t iterations_pair;       /* of the last step's iterations, those run in FP32 pairs (PIC_MIXED) */
    int32_t total_iterations_pair; /* FP32-pair iterations summed over the committed steps */
} pic_step_info;

typedef struct {
    double K;      /* sum_i m |v_i|^2 / 2 (Eq. (particle-energy)) */
    double W;      /* sum_g (|E_g|^2 / (2 sigma1) + |B_g|^2 / (2 sigma2)) dV (Eq. (field-energy)) */
    double total;  /* K + W (Eq. (total-discrete-energy)) */
} pic_energy_t;

/* Diagnostics of the last committed step (valid when the config has diagnostics = 1). */
typedef struct {
    double gauge_max, gauge_rms;   /* G_h = psi / kappa^2 + div_h A at n+1 (Eq. (gauge-diagnostic)) */
    double gauss_max, gauss_rms;   /* R_h = div_h E - sigma1 rho at n+1 (Eq. (gauss-diagnostic)) */
    double continuity_max;         /* max |rho^{n+1} - rho^n + dt div_h J^{n+1/2}| */
    double RA_max, RA_rms;         /* chain-rule residual over particles (Eq. (RA-test)) */
    double partition_max;          /* max_i |sum_g Sbar_ig - 1| (Appendix A) */
    double particle_work;          /* sum_i q vbar_i . Ebar_i (Eq. (power-test), left) */
    double mesh_work;              /* sum_g J . E^{n+1/2} dV (Eq. (power-test), right) */
    double R_field, R_particle, R_total; /* Eq. (R-field), (R-particle), (R-total) */
    double K0, W0, K1, W1;         /* energies before and after the step */
    int32_t picard_iterations;
    double e_v, e_J;
} pic_diag_t;

/* A full state, for checkpoint/restart and for inspection.  Caller-owned buffers:
 * x, v, P, vprev: 3 * np each; phi, psi, rho: ncell each; A, U: 3 * ncell each.
 * Particles are in the order they were given to pic_init. */
typedef struct {
    double *x, *v, *P, *vprev;
    double *phi, *psi, *rho;
    double *A, *U;
    int32_t on_device;
} pic_state_view;

/* Outputs of one Picard-iteration body (pic_iterate).  Caller-owned buffers with the
 * same sizes as in pic_state_view; J has 3 * ncell entries. */
typedef struct {
    double *J, *rho, *phi, *psi, *A, *U;  /* mesh: J^{n+1/2,p} and the level-(n+1,p) fields */
    double *x, *P, *v;                    /* particles: x^{n+1,p}, P^{n+1,p}, v^{n+1,p+1} */
    int32_t on_device;
} pic_iterate_out;

/* Live per-phase timing of the library's own kernels (CUDA events on the context stream)
 * and a count of every kernel it launched, accumulated since the last reset. */
typedef struct {
    int64_t launches;            /* kernels launched */
    int64_t push_launches;       /* fused push + next-orbit scatter launches (Picard iterations) */
    double push_ms;              /* their summed event durations */
    int64_t commit_launches;     /* final-sweep push launches */
    double commit_ms;
    int64_t scatter_launches;    /* first orbit-current scatter of each step */
    double scatter_ms;
    double mesh_ms;              /* continuity, CN Helmholtz solve, back-substitution, gather table */
    double sort_ms;              /* counting sort by cell */
    int64_t particle_pushes;     /* sum over push launches of the particle count */
    int64_t push_pieces;         /* knot-free orbit pieces integrated by those pushes */
    int64_t scatter_pieces;      /* orbit pieces integrated by their next-orbit scatters */
    int64_t push32_launches;     /* FP32 push + scatter launches (PIC_MIXED) */
    double push32_ms;
    int64_t local_launches;      /* particle-local solve launches (picard_accel = 1), one per FP64 push */
    double local_ms;             /* their summed event durations (not part of push_ms) */
    int64_t local_solves;        /* creeping particles solved by them */
    int64_t local_evals;         /* push evaluations those solves made (probes, first, iterations) */
    int64_t push32_chunks;       /* chunks of 256 particles pushed by the FP32 push launches */
    int64_t push32_chunks_global;/* ... of them whose orbits' mesh box exceeded the shared-memory
                                    tile, so that they gathered and scattered in global memory */
    int64_t pushpair_launches;   /* FP32-pair push + scatter launches (PIC_MIXED refinement) */
    double pushpair_ms;          /* their summed event durations */
    int64_t local_failed;        /* local solves whose best residual stayed above 1e-10 of the
                                    particle's speed (their pinned components aside, the residual
                                    stays in the committed step as an energy defect) */
    int64_t local_failed_unpinned; /* ... of them with no component within 1e-6 cells of a knot,
                                    so none was pinned */
} pic_profile_t;

/* Fill cfg with defaults: 8^3 nodes, box 2 pi / 3, dt = 0.1, kappa = sigma1 = sigma2 = 1,
 * n0 = 1, tau = 1e-13, p_max = 16, split closed-form orbits, FP64, sort every step,
 * diagnostics off, local solves on, Chebyshev reduction 1e-17, mixed: FP32 phase to 1e-9,
 * at most 8 FP32 iterations, one FP32-pair refinement iteration, FP64 refinement to picard_tol, not
 * deterministic, linear shapes (r = 1), central-difference operators. */
pic_status pic_config_default(pic_config* cfg);

/* Create a context: copies the particles to the device, sorts them by cell, deposits
 * rho^0 = sum_i q S_g(x_i)/dV + n0 with the null modes of Delta_h removed, solves
 * -Delta_h phi^0 = sigma1 rho^0, sets psi = A = U = 0, P = m v and v^{n-1} = v (§5.4).
 * `alloc` may be NULL.  `stream` is a cudaStream_t (NULL: the legacy default stream). */
pic_status pic_init(const pic_config* cfg, const pic_particles* particles,
                    const pic_allocator* alloc, void* stream, pic_ctx** out);

/* Advance nsteps time steps (Algorithm 1 plus the final consistency sweep of §5.4).
 * `info` may be NULL.  Returns PIC_ERR_NO_CONVERGENCE (state kept at the last committed
 * step) when a step reaches picard_max unless accept_unconverged is set. */
pic_status pic_step(pic_ctx* ctx, int32_t nsteps, pic_step_info* info);

/* Kinetic, field and total energy of the current state (§4.1), FP64 sums. */
pic_status pic_energy(pic_ctx* ctx, pic_energy_t* out);

/* Diagnostics of the last committed step (§5.1-§5.3).  PIC_ERR_ARG if none is available. */
pic_status pic_diagnostics(pic_ctx* ctx, pic_diag_t* out);

/* Copy the full state out (checkpoint) / in (restart).  pic_set_state also accepts a
 * state that was not produced by the library; it does not re-solve any field. */
pic_status pic_get_state(pic_ctx* ctx, const pic_state_view* dst);
pic_status pic_set_state(pic_ctx* ctx, const pic_state_view* src);

/* Run one body of the Algorithm 1 loop from the given end-of-step velocity iterate
 * v^{n+1,p} (3 * np, particles in pic_init order) without committing anything, and copy
 * out the orbit current, the new mesh fields and the pushed particles. */
pic_status pic_iterate(pic_ctx* ctx, const double* v_iter, int32_t on_device, const pic_iterate_out* out);

/* Particle positions exactly as stored, in cell units xi = x / H (3 * np, pic_init order,
 * wrapped to [0, n_a)): the orbit breakpoints and knot tests of §4.7 use these values. */
pic_status pic_get_positions(pic_ctx* ctx, double* xi, int32_t on_device);

/* The counterpart of pic_get_positions: set the particle positions in cell units (3 * np,
 * pic_init order, each in [0, n_a); values outside are wrapped periodically) without the
 * physical-unit conversion of pic_set_state, whose x / H rounds.  Call it after pic_set_state:
 * pic_get_state + pic_get_positions then restore a state bit for bit (checkpoint-and-recompute
 * of a run whose trajectory must repeat exactly, as the adjoint's backward pass does).  Not a
 * part of the paper's method; PIC_ERR_ARG on a NULL pointer. */
pic_status pic_set_positions(pic_ctx* ctx, const double* xi, int32_t on_device);

/* After a pic_step that did not converge: its last Picard iterate v^{n+1,p} and the image
 * G(v^{n+1,p}) (3 * np each, particles in pic_init order); their difference is each
 * particle's fixed-point residual (Algorithm 1).  PIC_ERR_ARG after a converged step. */
pic_status pic_get_iterate(pic_ctx* ctx, double* v_iter, double* g_iter, int32_t on_device);

/* Right after a pic_step that committed its last step: the end-of-step velocity iterate
 * v^{n+1,p+1} whose orbit that step's final consistency sweep used (Algorithm 1 and §5.4:
 * x^{n+1} = x^n + dt (v^{n+1,p+1} + v^n) / 2 and P^{n+1} come from that orbit; the committed
 * v^{n+1} is its image G(v^{n+1,p+1})), into v_iter (3 * np, pic_init order), and per
 * particle the sliding bits of that step into slide (np bytes, pic_init order): bit a set
 * means that component a landed exactly on a knot (the particle-local solve of picard_accel
 * found no root that double precision resolves; the committed v_a is then the iterate's and
 * P_a = m v_a + q A_h,a(x^{n+1})).  Either pointer may be NULL (not both).  Lets a caller
 * check the accepted step against the method's own equations: G(v) = v within picard_tol
 * for the components that do not slide.  PIC_ERR_ARG if no committed step precedes the call
 * (a failed step, pic_set_state, pic_iterate or pic_autotune came after it). */
pic_status pic_get_accepted(pic_ctx* ctx, double* v_iter, uint8_t* slide, int32_t on_device);

/* Bound, in SM clock cycles, of each wait of the FP32 push (precision = PIC_MIXED) for the
 * bulk copies that stage a chunk of particles in shared memory (default 2e9, about 1 s).
 * When a wait runs out, the block records PIC_ERR_TIMEOUT, waits for its copies still in
 * flight (always with the default bound, so that no copy lands after the block has exited)
 * and stops; the step returns PIC_ERR_TIMEOUT and keeps the committed state.  A short bound
 * is how a caller (or a test) checks that path without a fault.  PIC_ERR_ARG for cycles < 1. */
pic_status pic_set_wait_limit(pic_ctx* ctx, int64_t cycles);

/* ---- Adjoint of the step (reverse mode) ---------------------------------------------------
 *
 * For a scalar L of the state after a step, the adjoint maps lambda' = dL/d(state n+1) to
 * lambda = dL/d(state n) through Algorithm 1's implicit step: the accepted iterate v* solves
 * v* = G(v*; state n), and the implicit-function theorem gives its adjoint mu from the
 * transposed fixed point mu = F_v*^T (lambda' + mu on v^{n+1}), F being the final sweep
 * (§5.4).  The per-particle derivatives of the orbit integrals (Appendices A and B, with the
 * motion of every knot-crossing breakpoint, §4.3) come from forward-mode dual numbers through
 * the same closed forms; the mesh half is the transposed continuity and Crank--Nicolson update
 * (the Helmholtz operator is symmetric).  Positions' adjoints are per physical unit.  The
 * adjoint of v^{n-1} is zero (it only sets the first Picard iterate). */
typedef struct {
    int32_t iterations;   /* sweeps (applications of F^T) made by the transposed solve */
    double residual;      /* its final ||P r|| / ||mu||: r = F_v*^T(lambda' + mu) - mu the residual,
                             P the preconditioner, so the size of one more correction */
} pic_vjp_info;

/* lam_prev = (d state^{n+1} / d state^n)^T lam_next for the step that the last pic_step
 * committed (call it right after that pic_step: the context keeps level n and v* until the next
 * step begins).  Views as in pic_state_view (NULL members of lam_next are zero; NULL members of
 * lam_prev are not written).  Needs closed-form linear orbits and central differences.  A
 * component that slid onto a knot in that step is differentiated through the sliding
 * equations (its iterate is the landing velocity 2 d H / dt - v^n, its momentum m v + q A_h).
 * The transposed fixed point is solved by restarted GMRES (restart length 40, fewer when its
 * basis would pass 4 GiB), preconditioned with the transpose of the forward iteration's
 * splitting: the particles that the step solved locally get their 3 x 3 block
 * (I - (dG_i/dv_i)^T)^{-1}, all others the identity.  PIC_ERR_NO_CONVERGENCE if it does not
 * reach 1e-11 in 400 sweeps (the message lists the residual at each restart).  Allocates its
 * work buffers (about 51 np + 50 ncell doubles, plus the basis of 3 np (restart + 1) doubles)
 * on first use. */
pic_status pic_step_vjp(pic_ctx* ctx, const pic_state_view* lam_next, const pic_state_view* lam_prev,
                        pic_vjp_info* info);

/* lam = dW/d(state) of the current state, W the field energy (Eq. (field-energy)): nonzero for
 * phi, A and U only (the other members, when given, are zeroed). */
pic_status pic_energy_vjp(pic_ctx* ctx, const pic_state_view* lam);

/* The adjoint of pic_init's map from the initial particles (x^0, v^0) to the initial state
 * (§5.4: rho^0 deposited and projected, phi^0 from Poisson, P^0 = m v^0, v^{-1} = v^0):
 * lam_x0, lam_v0 (3 * np each, pic_init order) from the state adjoint lam0.  Only valid while
 * the context still holds pic_init's state. */
pic_status pic_init_vjp(pic_ctx* ctx, const pic_state_view* lam0, double* lam_x0, double* lam_v0, int32_t on_device);

/* Switch live profiling on (1) or off (0).  If `out` is non-NULL the accumulated profile is
 * copied there (after synchronising the stream) and the accumulators are reset. */
pic_status pic_profile(pic_ctx* ctx, int32_t enable, pic_profile_t* out);

/* Residual history of the last pic_step call (the last step it ran): for each Picard
 * iteration k, e_v[k] and e_J[k] (Algorithm 1's fixed-point errors of the update made by
 * iteration k: ||v^{k+1} - v^k|| and the change of the orbit current between the two
 * iterates, relative; FP32 iterations record the previous update's current change, +inf at
 * the first) and fp32[k] = 1 if the iteration ran in FP32, 2 if its particle half ran in FP32
 * pairs (PIC_MIXED), 3 for a final sweep that measured the residual ||G(v*) - v*|| / ||G(v*)||
 * of its own iterate (PIC_MIXED, see mixed_tol64; e_J is then not measured, NaN), else 0
 * (FP64).  Writes at
 * most `cap` entries into each non-NULL array and returns the number of iterations (which
 * may exceed cap), or -1 for a NULL context. */
int32_t pic_residual_history(const pic_ctx* ctx, int32_t cap, double* e_v, double* e_J, int32_t* fp32);

/* Choose the launch grids of the particle kernels for this context by measurement: the
 * FP64 push (blocks per SM in {2, 4, 8, 16}; default 8) and, for PIC_MIXED, the FP32 chunk
 * push ({4, 8, 16}; default 16), each timed over two launches on the context's stream from
 * one Algorithm 1 iteration body at the current state (scratch buffers only; the committed
 * state is unchanged).  Results are cached per process by mesh, particle count (in buckets
 * of 16384) and precision, so further contexts of the same shape reuse them without timing.
 * The chosen values are returned through the non-NULL pointers. */
pic_status pic_autotune(pic_ctx* ctx, int32_t* push_blocks_per_sm, int32_t* push32_blocks_per_sm);

/* ---- Ensembles of independent runs -------------------------------------------------------
 *
 * Many small runs do not fill the GPU one at a time.  An ensemble holds `nruns` contexts,
 * each created by pic_init from cfgs[i] and particles[i] on a stream of its own that the
 * ensemble creates (non-blocking), with device memory from `alloc` (may be NULL: cudaMalloc).
 * The runs may differ in mesh, particle count and every other setting.  No data is shared
 * between runs; each run computes exactly what pic_step would compute for it alone. */
typedef struct pic_ensemble pic_ensemble;

/* PIC_ERR_ARG for nruns < 1 or NULL arrays; otherwise the first failing pic_init's status
 * (nothing is kept then). */
pic_status pic_ensemble_init(int32_t nruns, const pic_config* cfgs, const pic_particles* particles,
                             const pic_allocator* alloc, pic_ensemble** out);

/* Advance every run by nsteps time steps.  The runs' Picard iterations interleave: the host
 * polls the runs' streams and queues a run's next iteration as soon as its previous one has
 * completed, so the runs' kernels overlap on the GPU.  A run that fails (any pic_step error)
 * stops at its last committed step while the others continue.  infos[i] / statuses[i]
 * (either may be NULL) receive each run's pic_step-style summary and final status.  Returns
 * PIC_OK, or the status of the lowest-numbered failed run (reason: pic_ensemble_last_error). */
pic_status pic_ensemble_step(pic_ensemble* e, int32_t nsteps, pic_step_info* infos, pic_status* statuses);

/* Number of runs (-1 for NULL); run i as a context for every other call of this header
 * (pic_energy, pic_get_state, ...; not pic_destroy: the ensemble owns it), NULL if out of range. */
int32_t pic_ensemble_size(const pic_ensemble* e);
pic_ctx* pic_ensemble_run(pic_ensemble* e, int32_t i);
const char* pic_ensemble_last_error(const pic_ensemble* e);
void pic_ensemble_destroy(pic_ensemble* e);

/* Largest mesh (nodes) accepted by pic_cn_update_static. */
#define PIC_STATIC_MAX_CELLS 32768

/* The Crank--Nicolson update of (phi, psi, A, U) for given sources, without allocating.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc where they need the update (a fixed, pre-committed device-memory budget, a
 * host thread that must not enter the CUDA allocator because it can synchronise the device,
 * or a plugin whose host application owns all device allocations).  It computes what
 * pic_step's mesh phase computes with the central-difference operators (PIC_OPS_CENTRAL2
 * only: Delta_h is the wide Laplacian sum_a D_a D_a; a context configured with
 * PIC_OPS_SPECTRAL solves the same equations with the Fourier operators and gets a
 * different update), (I - a Delta_h) F^{n+1} = (I + a Delta_h) F^n + dt W^n +
 * (dt^2 kappa^2 sigma / 2) src with a = kappa^2 dt^2 / 4 (src = rho_half for phi with sigma1,
 * J for A with sigma2), by the library's Chebyshev iteration (the fewest steps whose error
 * bound is below helmholtz_tol, at most 1024), then W^{n+1} = 2 (F^{n+1} - F^n) / dt - W^n.
 * (pic_step solves the same system by FFT on 2^p 3^q meshes; the results agree to the
 * solves' rounding.)
 *
 * Arguments: n, L: mesh nodes and box lengths (host); every array pointer is a DEVICE
 * pointer in the library's mesh layout (x-fastest; A, U, J component-major, 3 * ncell).
 * Inputs phi, psi, rho_half (ncell) and A, U, J (3 * ncell); outputs phi1, psi1 (ncell) and
 * A1, U1 (3 * ncell), which must not overlap the inputs.  Work is queued on `stream`; the
 * call returns without synchronising.
 *
 * Memory: working storage is one fixed __device__ array of 16 * PIC_STATIC_MAX_CELLS doubles
 * (4 MiB) that every device loading the library holds until the process exits; no call
 * allocates or frees device memory.  Every call looks that array's address up on the current
 * device (cudaGetSymbolAddress, which allocates nothing), so the address is never stale, even
 * after a device reset; the first call on a device may load the library's device code there,
 * so make it before any stream capture.  Every call on a device shares the array and nothing
 * in it needs to start at zero (each call writes what it reads), but two calls whose work
 * overlaps on the GPU (different streams, or before the earlier one finished) race on it.
 *
 * Errors: PIC_ERR_ARG for a null pointer, invalid sizes or constants,
 * n0 * n1 * n2 > PIC_STATIC_MAX_CELLS, or a helmholtz_tol that needs more than 1024 Chebyshev
 * steps; PIC_ERR_CUDA if a launch or the address look-up fails. */
pic_status pic_cn_update_static(const int32_t n[3], const double L[3], double dt, double kappa, double sigma1,
                                double sigma2, double helmholtz_tol, const double* phi, const double* psi,
                                const double* A, const double* U, const double* rho_half, const double* J,
                                double* phi1, double* psi1, double* A1, double* U1, void* stream);

/* Measured FMA throughput of the current device, in flop/s (an FMA counts 2): FP64 and FP32
 * independent FMA chains over a grid of 16 blocks per SM, timed with CUDA events on `stream`
 * after one warm-up launch.  The FP64 particle kernels are bound by the FP64 pipe, and their
 * roofline divides by an arithmetic peak; this is the measurement behind it.  Synchronises the
 * stream; makes one 8-byte stream-ordered allocation for the duration of the call. */
pic_status pic_probe_fma_rates(void* stream, double* fp64_flops, double* fp32_flops);

/* One-line description of the last error on this context ("" if none). */
const char* pic_last_error(const pic_ctx* ctx);

/* Free every device buffer of the context (on its stream) and the context itself. */
void pic_destroy(pic_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PIC_H */
