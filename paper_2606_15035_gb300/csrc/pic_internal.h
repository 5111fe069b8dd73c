// Host-side context and kernel launchers of the PIC library (internal).
#pragma once

#include <cstdint>
#include <string>
#include <utility>
#include <cmath>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pic.h"
#include "pic_device.cuh"

namespace pic {

// Reduction slots: each kernel writes one partial per block into partials[slot * MAX_BLOCKS + b];
// finalize() folds them in a fixed order into results[slot].
enum Slot : int {
    S_EV_NUM = 0,  // sum |v^{p+1} - v^p|^2
    S_EV_DEN,      // sum |v^{p+1}|^2
    S_EVL_NUM,     // the same two sums over the locally solved particles (k_local)
    S_EVL_DEN,
    S_EJ_NUM,      // sum |J^p - J^{p-1}|^2
    S_EJ_DEN,      // sum |J^p|^2
    S_JSCALE,      // sum |v^n|
    S_K1,          // sum m |v^{n+1}|^2 / 2
    S_PWORK,       // sum q vbar . Ebar
    S_RA_SQ,       // sum |R_A|^2
    S_RA_MAX,      // max |R_A| (component)
    S_PU_MAX,      // max |sum Sbar - 1|
    S_MWORK,       // sum J . E^{n+1/2} dV
    S_W,           // field energy at n+1 (diagnostics)
    S_W0,          // field energy of the current state
    S_G_MAX,
    S_G_SQ,
    S_R_MAX,
    S_R_SQ,
    S_CONT_MAX,
    S_K,           // kinetic energy of the current state
    S_PIECES_PUSH,     // orbit pieces visited by the push (profiling)
    S_PIECES_SCATTER,  // orbit pieces visited by the scatter of the next orbit (profiling)
    S_LOCAL_SOLVES,    // particle-local solves made by k_local (profiling)
    S_LOCAL_EVALS,     // push evaluations made by those solves (profiling)
    S_LOCAL_FAILED,    // solves that ended above FAIL_RES of the speed (profiling)
    S_LOCAL_FAILED_FREE,  // ... of them with no component pinned to a knot (profiling)
    S_CHUNKS32,        // particle chunks pushed by the FP32 push (profiling)
    S_CHUNKS32_GLOBAL, // ... of which gathered and scattered through global memory (box too big)
    S_PROJ0,       // 8 null-mode projections (init)
    S_NULLSTAT = S_PROJ0 + 8,
    NSLOT
};

constexpr int MAX_BLOCKS = 4096;

// Floors of the slow-particle test of the particle-local solves, as fractions of the speed: a
// particle is slow when its change did not shrink below SLOW_RATIO of the previous one and
// exceeds the floor.  In the first FP64 iteration after the FP32 ones the previous change is
// the last FP32 one, so the floor sits above the FP32 iterate's rounding (increments good to
// ~1e-10 of the speed): only particles that the FP32 loop left unconverged pass it.
constexpr double SLOW_FLOOR = 1e-12;
constexpr double SLOW_FLOOR_AFTER32 = 1e-8;
constexpr int THREADS = 256;

struct StepParams {
    MeshDims m;
    double H[3], invH[3];
    double dt, q, mass, inv_mass, q_dV;  // q_dV = q / dV
    int64_t np;
    int split;                 // split orbits at knots
    int nq;                    // Gauss points (Gauss quadrature only)
    int accel;                 // particle-local solves for creeping particles
    int hist;                  // vnew holds v^{p-1} (slow particles are found against it)
    double slow_floor;         // a slow particle's change also exceeds this times its speed
    int order;                 // B-spline degree r of the shape (1, 2, 3)
    double koff;               // knot offset: 0 (odd r, knots at the integers) or 0.5 (even r)
    int det;                   // deterministic mode: deposits go to acc (exact, order independent)
    ExactAcc acc;
};

constexpr int FFT_MAX = 1024;       // largest mesh size per axis with spectral operators
constexpr int FFT_MAX_STAGES = 16;

// Host-side state of the time step in progress (see step_begin / iter_issue / iter_finish).
struct StepRun {
    int cur = 0, prev = 1, next = 2;   // J buffers: current iterate, previous, next
    bool fp32 = false;                 // the next iteration runs in FP32 (PIC_MIXED)
    bool hist = false;                 // vnew holds the previous iterate v^{p-1}
    bool after32 = false;              // the iteration in flight is the first FP64 one after FP32
    bool trial = false;                // the next issue is a final sweep of v^{p+1} that measures
                                       // its residual (PIC_MIXED), instead of an iteration
    bool final_done = false;           // that sweep was accepted: the step only needs its commit
    double e_v32_first = 0.0, rho32 = 0.0;   // FP32 phase: first e_v, contraction e_v[1] / e_v[0]
    double e_v64_prev = 0.0;           // e_v of the previous FP64 iteration
    double trial_eJ = 0.0;             // e_J of the iteration whose iterate the trial sweeps
    bool began32 = false;              // the step began with FP32 iterations (PIC_MIXED)
    bool pair = false;                 // the next iteration's particle half runs in FP32 pairs
    bool pair_issued = false;          // the iteration in flight ran in FP32 pairs
    int ppair = 0;                     // FP32-pair iterations done in this step
    double e_vpair_prev = INFINITY;
    int p64 = 0;                       // FP64 iterations done in this step
    bool iterating = true;             // the Picard loop is still running
    bool converged = false;
    int p = 0, p32 = 0;                // iteration index, FP32 iterations done
    double e_v = 0.0, e_J = 0.0, jscale = 0.0, e_v32_prev = INFINITY;
    void rotate() {
        const int old_prev = prev;
        prev = cur;
        cur = next;
        next = old_prev;
    }
};

struct Ctx {
    pic_config cfg;
    cudaStream_t stream = nullptr;
    pic_allocator alloc{};
    bool has_alloc = false;
    std::string err;

    MeshDims m{};
    int sms = 152;
    int push_bps = 8;     // grid of the FP64 particle kernels: blocks per SM (pic_autotune)
    int push32_bps = 16;  // grid of the FP32 chunk kernels: blocks per SM (pic_autotune)
    double H[3], invH[3], dV = 0, volume = 0;
    int64_t np = 0;
    double q = 0, mass = 0;

    // particles, FP64 SoA (3 * np each)
    double *xi = nullptr, *v = nullptr, *P = nullptr, *vprev = nullptr;
    double *vit = nullptr, *vnew = nullptr, *xi_new = nullptr, *P_new = nullptr;
    const double *last_v = nullptr, *last_g = nullptr;   // last Picard iterate and the next one
    double* gsave = nullptr;         // G(v^p) of the locally solved particles (diagnostics)
    bool last_failed = false;        // the last step hit picard_max
    bool have_accepted = false;      // vit and slide hold the last committed step's final-sweep
                                     // iterate and sliding marks (until the next step begins)
    long long wait_cycles = 2000000000LL;   // bound of k_push32's waits on its bulk copies
    uint8_t* slide = nullptr;        // per particle, bit a: component a slides along a knot
    int32_t* creep_list = nullptr;   // creeping particles of the current iteration (local solves)
    int* creep_count = nullptr;
    int64_t *id = nullptr, *id_tmp = nullptr;
    double* sort_tmp = nullptr;          // 3 * np
    int32_t *key = nullptr, *count = nullptr, *offset = nullptr, *cursor = nullptr;
    int32_t* scan_tmp = nullptr;         // block totals of the scan

    // mesh, FP64.  F = [phi | A_x | A_y | A_z] and W = [psi | U_x | U_y | U_z] (4 * ncell).
    double *F0 = nullptr, *W0 = nullptr, *rho0 = nullptr;
    double *F1 = nullptr, *F1b = nullptr, *W1 = nullptr, *rho1 = nullptr;
    double *cheb_d = nullptr, *rhs0 = nullptr, *rhs = nullptr;
    double *J[3] = {nullptr, nullptr, nullptr};
    double* table = nullptr;             // 12 * ncell gather table

    // FP32 working set of the mixed path (allocated only for PIC_MIXED)
    std::vector<double> hist_ev, hist_eJ;   // residuals of the last step's iterations
    std::vector<int32_t> hist_fp32;
    StepRun run;
    double trial_kappa = 0.0;          // PIC_MIXED: measured ||G(v*) - v*|| / e_J of trial sweeps
    // spectral operators (ops = PIC_OPS_SPECTRAL): transforms of level n [phi, A | psi, U | rho]
    // (9 N), of level n+1 and D phi^{n+1/2} (12 N), of J (3 N), residual scratch (3 N), the
    // real D phi^{n+1/2} (3 N), and the FFT plan of each axis
    double2 *spec0 = nullptr, *spec1 = nullptr, *specJ = nullptr, *specR = nullptr;
    double* spec_gphi = nullptr;
    double2* fft_tw[3] = {nullptr, nullptr, nullptr};
    int fft_radix[3][FFT_MAX_STAGES] = {};
    int fft_nst[3] = {0, 0, 0};
    // central-difference operators on a 2^p 3^q mesh: the CN Helmholtz solve of each mesh phase
    // by FFT (4 N complex scratch, per-axis symbols sin^2(2 pi m / n_a) / H_a^2)
    bool helm_fft = false;
    double2* helm_spec = nullptr;
    double* helm_s2 = nullptr;
    // deterministic mode: exact deposit accumulators (3 N each), their scales, creeping flags,
    // and the radix-sort work arrays
    long long *acc_hi = nullptr, *acc_lo = nullptr;
    double inv_u_J = 1.0, inv_u_rho = 1.0;
    uint8_t* creep_flag = nullptr;
    int32_t *rs_key[2] = {nullptr, nullptr}, *rs_val[2] = {nullptr, nullptr}, *rs_hist = nullptr, *rs_offs = nullptr;
    int32_t* rs_scan_tmp = nullptr;
    int64_t np32 = 0;   // component stride of the FP32 arrays: np rounded up to 256 entries
    int32_t* cell32 = nullptr;
    float *off32 = nullptr, *v32 = nullptr, *vit32 = nullptr, *vnew32 = nullptr;   // iterates: increments
    float* table32 = nullptr;            // 12 * ncell
    float* table_pair = nullptr;         // 20 * ncell: A^n, A^{n+1}, grad phi as FP32 pairs (+ pad)

    // reductions and status
    double *partials = nullptr, *results = nullptr;
    int* dev_status = nullptr;
    double* host_results = nullptr;      // pinned, NSLOT
    int* host_status = nullptr;          // pinned

    // Chebyshev schedule for the CN Helmholtz solve
    int cheb_iters = 0;
    double cheb_alpha[1024], cheb_beta[1024];
    double* cheb_coef_dev = nullptr;   // alpha (1024) | beta (1024) on the device, for k_cheb_all
    int cheb_coop_blocks = 0;          // co-resident blocks for the cooperative solve (0: none)
    double cheb_lmax = 1.0;            // largest eigenvalue of I - a Delta_h
    double cheb_rate = 0.0;            // 1 / log(1 / rho) of the Chebyshev bound (0: one step)
    double* cheb_red = nullptr;        // per-block sums of the cooperative solve (8 per block)

    // adjoint (pic_step_vjp / pic_init_vjp), allocated on first use: particles (3 np each) the
    // adjoints of x^{n+1} (cell units), v^{n+1}, P^{n+1}, of v* (two buffers), of x^n, the
    // sweep's adjoint of v* g and the preconditioner's blocks B (9 np), a scratch; mesh: the gather table's
    // adjoint (9 N), the level-(n+1) inputs and level-n outputs, the Helmholtz buffers, J's adjoint
    bool fresh_init = false;             // the state is pic_init's (no step or set_state since)
    double *adj_xe = nullptr, *adj_v = nullptr, *adj_P = nullptr, *adj_mu = nullptr, *adj_mu2 = nullptr;
    double *adj_xi = nullptr, *adj_g = nullptr, *adj_B = nullptr, *adj_tmp = nullptr, *adj_vn = nullptr, *adj_Pn = nullptr;
    double *adj_tab = nullptr, *adj_F1 = nullptr, *adj_W1 = nullptr, *adj_rho1 = nullptr;
    double *adj_t = nullptr, *adj_pn = nullptr, *adj_y = nullptr, *adj_ys = nullptr, *adj_J = nullptr;
    double *adj_F0 = nullptr, *adj_W0 = nullptr, *adj_rho0 = nullptr;
    double *adj_b0 = nullptr, *adj_w = nullptr, *adj_V = nullptr;   // the transposed solve's Krylov basis
    double *adj_h = nullptr, *adj_part = nullptr;                     // its dot products (device)
    int adj_m = 0;                                                    // restart length (basis size - 1)

    // live profiling: event pairs per phase, resolved at the next stream synchronisation
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
    pic_profile_t prof_acc{};
    int64_t launches = 0;

    // bookkeeping
    int64_t steps = 0;
    bool have_diag = false;
    pic_diag_t diag{};
    bool have_energy = false;
    double K_n = 0, W_n = 0;
};

enum ProfPhase : int { PH_PUSH = 0, PH_COMMIT, PH_SCATTER, PH_MESH, PH_SORT, PH_PUSH32, PH_LOCAL, PH_PUSHPAIR };

// ---- launchers (particles.cu) ----
void launch_init_positions(Ctx& c, const double* x_dev);
void launch_point_deposit(Ctx& c);
void launch_set_positions(Ctx& c, const double* src_dev);
void launch_sort(Ctx& c);
void launch_first_scatter(Ctx& c, double* J, const double* v_iter_or_null);
void launch_push(Ctx& c, const double* vit, double* vnew, double* Jnext, bool commit, bool diag);
// The particle-local solves of the creeping particles that the last (non-commit) push listed.
void launch_local(Ctx& c, const double* vit, double* vnew, double* Jnext);
void launch_kinetic(Ctx& c);
void launch_unpermute(Ctx& c, const double* src_soa3, double* dst_soa3, double scale0, double scale1, double scale2);
void launch_patch_local(Ctx& c, double* g);
// dst[id[i]] = slide[i] & 7 (the sliding bits of each particle, in caller order).
void launch_slide_out(Ctx& c, uint8_t* dst);
void launch_permute_in(Ctx& c, const double* src_soa3, double* dst_soa3, double s0, double s1, double s2);
void set_gauss_rule(int nq);

// ---- launchers (particles_df.cu): the FP32-pair refinement push ----
void launch_table_df(Ctx& c);
void launch_push_df(Ctx& c, const double* vit, double* vnew, double* Jnext);

// ---- launchers (adjoint.cu) ----
void launch_adj_scatter(Ctx& c, const double* xi, const double* v, const double* vstar, const double* lam_P,
                        const double* lam_v, const double* mu, double* lam_tab);
void launch_adj_mesh_rhs(Ctx& c, const double* lam_tab, const double* lF1, const double* lW1, double* t, double* pn);
void launch_adj_mesh_out(Ctx& c, const double* y, const double* pn, const double* lW1, const double* lrho1,
                         double* lF0, double* lW0, double* lrho0, double* lJ);
void launch_adj_derivs(Ctx& c, const double* xi, const double* v, const double* vstar, const double* lJ,
                       const double* lam_P, const double* lam_v, const double* lam_xe, const double* mu,
                       double* lam_xi, double* g, double* lvn, double* lPn, double* B);
void launch_adj_precond(Ctx& c, const double* B, const double* r, double* z);
void launch_adj_apply(Ctx& c, int64_t n, const double* z, const double* g, const double* b0, double* w);
void launch_adj_mdot(Ctx& c, int64_t n, const double* w, const double* V, int64_t ldv, int nv, double* part,
                     double* out);
void launch_adj_combine(Ctx& c, int64_t n, double* w, const double* V, int64_t ldv, int nv, const double* h,
                        double sign);
int adj_blocks(const Ctx& c, int64_t n);
void launch_adj_axpy(Ctx& c, int64_t n, double* y, const double* x, double s);
void launch_adj_deposit(Ctx& c, const double* xi, const double* lam_dep, double* lam_xi);
void launch_energy_grad(Ctx& c, double* lF, double* lW);

// ---- launchers (particles32.cu) ----
void launch_to32(Ctx& c);
void launch_scatter32(Ctx& c, double* J);
void launch_push32(Ctx& c, double* Jnext);
void launch_exact_finish(Ctx& c, double* out, int64_t n, double inv_u);   // acc -> out, acc = 0
// spectral operators (spectral.cu)
bool fft_factor(int n, int* radix, int& nst);
void spec_twiddles(int n, std::vector<double2>& tw);
void launch_spec_begin(Ctx& c);
void launch_spec_mesh_phase(Ctx& c, const double* Jcur, const double* Jprev);
void launch_spec_energy(Ctx& c, const double* F, const double* W, int slot);
void launch_spec_diag(Ctx& c, const double* Jfinal);
void launch_spec_poisson(Ctx& c);
void launch_helmholtz_fft(Ctx& c, const double* b, double* x, int nf, double a);
int radix_tiles(int64_t np);
int push32_blocks(const Ctx& c);   // grid of the FP32 chunk kernels (partials per block)
void launch_table32(Ctx& c);
void launch_from32(Ctx& c, const float* a, double* b);

// ---- launchers (mesh.cu) ----
void launch_rhs0(Ctx& c);
void launch_source(Ctx& c, const double* Jcur, const double* Jprev);
// Partials of |Jnew - Jold|^2 and |Jnew|^2 (the current fixed-point error of one update).
void launch_jdiff(Ctx& c, const double* Jnew, const double* Jold);
void launch_helmholtz(Ctx& c, const double* b, double c_id, double c_lap, int nfields, int iters,
                      const double* alpha, const double* beta, double** x_io, double** x_spare);
void launch_backsub_table(Ctx& c, bool diag);
void launch_helmholtz_cn(Ctx& c, double** x_io, double** x_spare, double tol);
void launch_helmholtz_fft_refined(Ctx& c, double* x);
int cheb_coop_capacity(const Ctx& c);
void launch_null_project(Ctx& c, double* f, double add_const);
void launch_mesh_energy(Ctx& c, const double* F, const double* W, int slot);
void launch_mesh_diag(Ctx& c, const double* Jfinal);
void launch_finalize(Ctx& c, int slot0, int nslots, int nblocks, bool is_max);
void launch_fill(Ctx& c, double* p, int64_t n, double value);
void launch_scale_copy(Ctx& c, double* dst, const double* src, int64_t n, double s);

// Chebyshev iteration for a symmetric operator with spectrum in [lmin, lmax] (pic_abi.cu):
// cheb_steps is the step count that brings the error bound 2 rho^k / (1 + rho^{2k}),
// rho = (sqrt(lmax / lmin) - 1) / (sqrt(lmax / lmin) + 1), below eps; cheb_schedule writes the
// three-term recurrence coefficients of min(cheb_steps, cap) steps and returns that count.
int cheb_steps(double lmin, double lmax, double eps);
int cheb_schedule(double lmin, double lmax, double eps, double* alpha, double* beta, int cap);

// Kernel parameters of the FP64 particle kernels for this context (particles.cu).
StepParams make_params(const Ctx& c);

int particle_blocks(const Ctx& c);
int local_blocks(const Ctx& c);
int mesh_blocks(const Ctx& c);

}  // namespace pic
