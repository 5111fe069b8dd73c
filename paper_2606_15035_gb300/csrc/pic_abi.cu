// C-ABI of the PIC library: context management and the host side of Algorithm 1.
//
// Every entry point validates its arguments, runs its device work on the context's
// stream, converts CUDA failures and device status bits into a pic_status, and records a
// one-line reason in ctx->err.  No entry point aborts.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <tuple>
#include <new>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "pic_internal.h"

using namespace pic;

struct pic_ctx {
    Ctx c;
    std::vector<std::pair<void*, size_t>> allocs;
};

namespace {

pic_status fail(pic_ctx* ctx, pic_status s, const std::string& why) {
    if (ctx) ctx->c.err = why;
    return s;
}

void* dev_alloc(pic_ctx* ctx, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (ctx->c.has_alloc) {
        p = ctx->c.alloc.alloc(bytes, (void*)ctx->c.stream, ctx->c.alloc.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) ctx->allocs.emplace_back(p, bytes);
    return p;
}

void free_all(pic_ctx* ctx) {
    for (auto& a : ctx->allocs) {
        if (ctx->c.has_alloc) ctx->c.alloc.free(a.first, a.second, (void*)ctx->c.stream, ctx->c.alloc.user);
        else cudaFree(a.first);
    }
    ctx->allocs.clear();
    if (ctx->c.host_results) cudaFreeHost(ctx->c.host_results);
    if (ctx->c.host_status) cudaFreeHost(ctx->c.host_status);
    ctx->c.host_results = nullptr;
    ctx->c.host_status = nullptr;
}

// Largest sin^2(2 pi m / n) over integer m, and the smallest positive one.
void sin2_range(int n, double& mx, double& mn_pos) {
    mx = 0.0;
    mn_pos = 0.0;
    for (int m = 0; m < n; ++m) {
        double s = std::sin(2.0 * M_PI * m / n);
        s = s * s;
        if (s < 1e-24) continue;
        mx = std::max(mx, s);
        mn_pos = mn_pos == 0.0 ? s : std::min(mn_pos, s);
    }
}

}  // namespace

namespace pic {

int cheb_steps(double lmin, double lmax, double eps) {
    const double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    if (delta <= 1e-14 * theta) return 1;
    const double kap = lmax / lmin;
    const double rho = (std::sqrt(kap) - 1.0) / (std::sqrt(kap) + 1.0);
    const double k = std::ceil(std::log(2.0 / eps) / std::log(1.0 / rho)) + 1.0;
    return k > 1e9 ? 1000000000 : std::max(1, (int)k);
}

int cheb_schedule(double lmin, double lmax, double eps, double* alpha, double* beta, int cap) {
    double theta = 0.5 * (lmax + lmin), delta = 0.5 * (lmax - lmin);
    if (delta <= 1e-14 * theta) {
        alpha[0] = 0.0;
        beta[0] = 1.0 / theta;
        return 1;
    }
    const int k = std::min(cheb_steps(lmin, lmax, eps), cap);
    double sigma = theta / delta;
    double rprev = 1.0 / sigma;
    alpha[0] = 0.0;
    beta[0] = 1.0 / theta;
    for (int j = 1; j < k; ++j) {
        double r = 1.0 / (2.0 * sigma - rprev);
        alpha[j] = r * rprev;
        beta[j] = 2.0 * r / delta;
        rprev = r;
    }
    return k;
}

}  // namespace pic

namespace {

pic_status check_cuda(pic_ctx* ctx, const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return PIC_OK;
}

// ---- live profiling ----
cudaEvent_t take_event(Ctx& c) {
    if (!c.ev_pool.empty()) {
        cudaEvent_t e = c.ev_pool.back();
        c.ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Brackets one phase with events on the context stream when profiling is on.
struct ProfScope {
    Ctx& c;
    int phase;
    cudaEvent_t e0 = nullptr;
    ProfScope(Ctx& c_, int ph) : c(c_), phase(ph) {
        if (c.prof) {
            e0 = take_event(c);
            cudaEventRecord(e0, c.stream);
        }
    }
    ~ProfScope() {
        if (c.prof) {
            cudaEvent_t e1 = take_event(c);
            cudaEventRecord(e1, c.stream);
            c.ev_pending.push_back({phase, {e0, e1}});
        }
    }
};

// After a stream synchronisation: fold the pending event pairs into the accumulators.
void prof_resolve(Ctx& c) {
    for (auto& pe : c.ev_pending) {
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, pe.second.first, pe.second.second);
        switch (pe.first) {
            case PH_PUSH: c.prof_acc.push_ms += ms; c.prof_acc.push_launches += 1; c.prof_acc.particle_pushes += c.np; break;
            case PH_COMMIT: c.prof_acc.commit_ms += ms; c.prof_acc.commit_launches += 1; break;
            case PH_SCATTER: c.prof_acc.scatter_ms += ms; c.prof_acc.scatter_launches += 1; break;
            case PH_MESH: c.prof_acc.mesh_ms += ms; break;
            case PH_SORT: c.prof_acc.sort_ms += ms; break;
            case PH_PUSH32: c.prof_acc.push32_ms += ms; c.prof_acc.push32_launches += 1; break;
            case PH_LOCAL: c.prof_acc.local_ms += ms; c.prof_acc.local_launches += 1; break;
            case PH_PUSHPAIR: c.prof_acc.pushpair_ms += ms; c.prof_acc.pushpair_launches += 1; break;
            default: break;
        }
        c.ev_pool.push_back(pe.second.first);
        c.ev_pool.push_back(pe.second.second);
    }
    c.ev_pending.clear();
}

// Copy results + status to the host and wait.
// Queue the copy of the result slots and the status word to the pinned host buffers.
void queue_results(Ctx& c) {
    cudaMemcpyAsync(c.host_results, c.results, sizeof(double) * NSLOT, cudaMemcpyDeviceToHost, c.stream);
    cudaMemcpyAsync(c.host_status, c.dev_status, sizeof(int), cudaMemcpyDeviceToHost, c.stream);
}

// Wait for the stream, then turn CUDA errors and device status bits into a status.
pic_status wait_results(pic_ctx* ctx, const char* where) {
    Ctx& c = ctx->c;
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return fail(ctx, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    if (c.prof) prof_resolve(c);
    pic_status s = check_cuda(ctx, where);
    if (s != PIC_OK) return s;
    int st = *c.host_status;
    if (st & DEV_ERR_SEGMENTS)
        return fail(ctx, PIC_ERR_SEGMENTS, std::string(where) + ": an orbit crossed more knots than supported in one step");
    if (st & DEV_ERR_NONFINITE) return fail(ctx, PIC_ERR_NONFINITE, std::string(where) + ": non-finite particle velocity");
    if (st & DEV_ERR_RANGE)
        return fail(ctx, PIC_ERR_NONFINITE, std::string(where) + ": a deposit beyond the exact accumulator's range "
                                                               "(a speed above 100 kappa in deterministic mode)");
    if (st & DEV_ERR_TIMEOUT)
        return fail(ctx, PIC_ERR_TIMEOUT, std::string(where) + ": a bulk copy into shared memory did not complete");
    if (st & DEV_ERR_TILE)
        return fail(ctx, PIC_ERR_INTERNAL, std::string(where) + ": an orbit left the mesh tile of its block");
    return PIC_OK;
}

pic_status sync_results(pic_ctx* ctx, const char* where) {
    queue_results(ctx->c);
    return wait_results(ctx, where);
}

pic_status validate(const pic_config* cfg) {
    for (int a = 0; a < 3; ++a)
        if (cfg->n[a] < 1 || !(cfg->L[a] > 0.0)) return PIC_ERR_ARG;
    if ((int64_t)cfg->n[0] * cfg->n[1] * cfg->n[2] >= (int64_t)1 << 31) return PIC_ERR_ARG;
    if (!(cfg->dt > 0.0) || !(cfg->kappa > 0.0) || !(cfg->sigma1 > 0.0) || !(cfg->sigma2 > 0.0)) return PIC_ERR_ARG;
    if (!(cfg->picard_tol > 0.0) || cfg->picard_max < 0) return PIC_ERR_ARG;
    if (cfg->quadrature != PIC_QUAD_CLOSED && cfg->quadrature != PIC_QUAD_GAUSS) return PIC_ERR_ARG;
    if (cfg->quadrature == PIC_QUAD_CLOSED && !cfg->split_orbit_at_knots) return PIC_ERR_ARG;
    if (cfg->quadrature == PIC_QUAD_GAUSS && (cfg->nq < 1 || cfg->nq > 16)) return PIC_ERR_ARG;
    if (cfg->precision != PIC_FP64 && cfg->precision != PIC_MIXED) return PIC_ERR_ARG;
    if (cfg->precision == PIC_MIXED) {
        if (cfg->quadrature != PIC_QUAD_CLOSED || cfg->n[0] > 1024 || cfg->n[1] > 1024 || cfg->n[2] > 1024)
            return PIC_ERR_ARG;
        if (!(cfg->mixed_tol32 > 0.0) || cfg->mixed_max32 < 1 || !(cfg->mixed_tol64 >= 0.0)) return PIC_ERR_ARG;
        if (cfg->mixed_pair_max < 0) return PIC_ERR_ARG;
    }
    if (!(cfg->helmholtz_tol > 0.0) || cfg->sort_every < 0) return PIC_ERR_ARG;
    if (cfg->shape_order < 1 || cfg->shape_order > 3) return PIC_ERR_ARG;
    if (cfg->ops != PIC_OPS_CENTRAL2 && cfg->ops != PIC_OPS_SPECTRAL) return PIC_ERR_ARG;
    if (cfg->ops == PIC_OPS_SPECTRAL) {
        int radix[FFT_MAX_STAGES], nst = 0;
        for (int a = 0; a < 3; ++a)
            if (!fft_factor(cfg->n[a], radix, nst)) return PIC_ERR_ARG;
    }
    if (cfg->shape_order > 1 && (cfg->quadrature != PIC_QUAD_GAUSS || cfg->precision != PIC_FP64)) return PIC_ERR_ARG;
    return PIC_OK;
}

void setup_geometry(Ctx& c) {
    c.m.n[0] = c.cfg.n[0];
    c.m.n[1] = c.cfg.n[1];
    c.m.n[2] = c.cfg.n[2];
    c.m.ncell = (int64_t)c.cfg.n[0] * c.cfg.n[1] * c.cfg.n[2];
    c.volume = 1.0;
    for (int a = 0; a < 3; ++a) {
        c.H[a] = c.cfg.L[a] / c.cfg.n[a];
        c.invH[a] = 1.0 / c.H[a];
        c.volume *= c.cfg.L[a];
    }
    c.dV = c.H[0] * c.H[1] * c.H[2];
    // CN Helmholtz operator I - a Delta_h: spectrum [1, 1 + a sum_a max sin^2 / H_a^2].
    double a = 0.25 * c.cfg.kappa * c.cfg.kappa * c.cfg.dt * c.cfg.dt;
    double lmax = 1.0;
    for (int ax = 0; ax < 3; ++ax) {
        double mx, mn;
        sin2_range(c.cfg.n[ax], mx, mn);
        lmax += a * mx * c.invH[ax] * c.invH[ax];
    }
    c.cheb_iters = cheb_schedule(1.0, lmax, c.cfg.helmholtz_tol, c.cheb_alpha, c.cheb_beta, 1024);
    c.cheb_lmax = lmax;
    const double rho = (std::sqrt(lmax) - 1.0) / (std::sqrt(lmax) + 1.0);
    c.cheb_rate = (c.cheb_iters > 1 && rho > 0.0) ? 1.0 / std::log(1.0 / rho) : 0.0;
}

#define ALLOC(ptr, type, count)                                                          \
    do {                                                                                 \
        (ptr) = (type*)dev_alloc(ctx, sizeof(type) * (size_t)(count));                   \
        if (!(ptr)) return fail(ctx, PIC_ERR_OOM, "device allocation of " #ptr " failed"); \
    } while (0)

pic_status allocate(pic_ctx* ctx) {
    Ctx& c = ctx->c;
    const int64_t np3 = 3 * std::max<int64_t>(c.np, 1), N = c.m.ncell;
    ALLOC(c.xi, double, np3);
    ALLOC(c.v, double, np3);
    ALLOC(c.P, double, np3);
    ALLOC(c.vprev, double, np3);
    ALLOC(c.vit, double, np3);
    ALLOC(c.vnew, double, np3);
    ALLOC(c.xi_new, double, np3);
    ALLOC(c.P_new, double, np3);
    ALLOC(c.sort_tmp, double, np3);
    ALLOC(c.creep_list, int32_t, std::max<int64_t>(c.np, 1));
    ALLOC(c.gsave, double, np3);
    ALLOC(c.slide, uint8_t, std::max<int64_t>(c.np, 1));
    ALLOC(c.creep_count, int, 2);   // creeping count, queue head of the local solves
    ALLOC(c.id, int64_t, std::max<int64_t>(c.np, 1));
    ALLOC(c.id_tmp, int64_t, std::max<int64_t>(c.np, 1));
    ALLOC(c.key, int32_t, std::max<int64_t>(c.np, 1));
    ALLOC(c.count, int32_t, N);
    ALLOC(c.offset, int32_t, N);
    ALLOC(c.cursor, int32_t, N);
    ALLOC(c.scan_tmp, int32_t, (N + 1023) / 1024 + 1);
    ALLOC(c.F0, double, 4 * N);
    ALLOC(c.W0, double, 4 * N);
    ALLOC(c.rho0, double, N);
    ALLOC(c.F1, double, 4 * N);
    ALLOC(c.F1b, double, 4 * N);
    ALLOC(c.W1, double, 4 * N);
    ALLOC(c.rho1, double, N);
    ALLOC(c.cheb_d, double, 4 * N);
    ALLOC(c.cheb_coef_dev, double, 2048);
    cudaMemcpyAsync(c.cheb_coef_dev, c.cheb_alpha, sizeof(double) * 1024, cudaMemcpyHostToDevice, c.stream);
    cudaMemcpyAsync(c.cheb_coef_dev + 1024, c.cheb_beta, sizeof(double) * 1024, cudaMemcpyHostToDevice, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "chebyshev coefficients");
    c.cheb_coop_blocks = cheb_coop_capacity(c);
    cudaGetLastError();
    ALLOC(c.cheb_red, double, 8 * (int64_t)std::max(1, c.cheb_coop_blocks));
    ALLOC(c.rhs0, double, 4 * N);
    ALLOC(c.rhs, double, 4 * N);
    for (int k = 0; k < 3; ++k) ALLOC(c.J[k], double, 3 * N);
    ALLOC(c.table, double, 12 * N);
    if (c.cfg.precision == PIC_MIXED) {
        // padded so that every chunk of 256 particles starts 16-byte aligned in every array
        c.np32 = std::max<int64_t>((c.np + 255) / 256 * 256, 256);
        ALLOC(c.cell32, int32_t, c.np32);
        ALLOC(c.off32, float, 3 * c.np32);
        ALLOC(c.v32, float, 3 * c.np32);
        ALLOC(c.vit32, float, 3 * c.np32);
        ALLOC(c.vnew32, float, 3 * c.np32);
        for (const void* q : {(const void*)c.cell32, (const void*)c.off32, (const void*)c.v32,
                              (const void*)c.vit32, (const void*)c.vnew32})
            if (reinterpret_cast<uintptr_t>(q) % 16 != 0)
                return fail(ctx, PIC_ERR_ARG, "the allocator returned a pointer that is not 16-byte aligned");
        ALLOC(c.table32, float, 12 * N);
        if (c.cfg.mixed_pair_max > 0 && !c.cfg.deterministic) ALLOC(c.table_pair, float, 20 * N);
    }
    if (c.cfg.deterministic) {
        ALLOC(c.acc_hi, long long, 3 * N);
        ALLOC(c.acc_lo, long long, 3 * N);
        cudaMemsetAsync(c.acc_hi, 0, sizeof(long long) * 3 * N, c.stream);
        cudaMemsetAsync(c.acc_lo, 0, sizeof(long long) * 3 * N, c.stream);
        ALLOC(c.creep_flag, uint8_t, std::max<int64_t>(c.np, 1));
        const int64_t np1 = std::max<int64_t>(c.np, 1);
        const int64_t nh = (int64_t)256 * radix_tiles(c.np);
        for (int k = 0; k < 2; ++k) {
            ALLOC(c.rs_key[k], int32_t, np1);
            ALLOC(c.rs_val[k], int32_t, np1);
        }
        ALLOC(c.rs_hist, int32_t, nh);
        ALLOC(c.rs_offs, int32_t, nh);
        ALLOC(c.rs_scan_tmp, int32_t, (nh + 1023) / 1024 + 1);
        // scales of the exact accumulators: bounds on the sum of |deposit| into one entry,
        // sum_i |q| |vbar_i| / dV (speeds below 100 kappa) for J and sum_i |q| / dV for rho
        const double wq = std::max<double>((double)c.np, 1.0) * std::fabs(c.q) / c.dV;
        auto inv_u = [](double W) {
            int e = 0;
            std::frexp(std::max(W, 1e-300), &e);   // W < 2^e
            return std::ldexp(1.0, 102 - e);
        };
        c.inv_u_J = inv_u(wq * 100.0 * c.cfg.kappa);
        c.inv_u_rho = inv_u(wq);
    }
    // central differences on a mesh the FFT takes: the CN Helmholtz solves go through it
    if (c.cfg.ops == PIC_OPS_CENTRAL2) {
        bool ok = true;
        for (int a = 0; a < 3; ++a) {
            int radix[FFT_MAX_STAGES], nst = 0;
            ok = ok && fft_factor(c.m.n[a], radix, nst);
        }
        c.helm_fft = ok;
    }
    if (c.helm_fft) {
        ALLOC(c.helm_spec, double2, 4 * N);
        ALLOC(c.helm_s2, double, c.m.n[0] + c.m.n[1] + c.m.n[2]);
        std::vector<double> s2;
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < c.m.n[a]; ++i) {
                const double sn = std::sin(2.0 * M_PI * i / c.m.n[a]);
                s2.push_back(sn * sn * c.invH[a] * c.invH[a]);
            }
        cudaMemcpyAsync(c.helm_s2, s2.data(), sizeof(double) * s2.size(), cudaMemcpyHostToDevice, c.stream);
        if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "helmholtz symbols");
    }
    if (c.cfg.ops == PIC_OPS_SPECTRAL) {
        ALLOC(c.spec0, double2, 9 * N);
        ALLOC(c.spec1, double2, 12 * N);
        ALLOC(c.specJ, double2, 3 * N);
        ALLOC(c.specR, double2, 3 * N);
        ALLOC(c.spec_gphi, double, 3 * N);
    }
    if (c.cfg.ops == PIC_OPS_SPECTRAL || c.helm_fft) {
        for (int a = 0; a < 3; ++a) {
            fft_factor(c.m.n[a], c.fft_radix[a], c.fft_nst[a]);
            std::vector<double2> tw;
            spec_twiddles(c.m.n[a], tw);
            ALLOC(c.fft_tw[a], double2, c.m.n[a]);
            cudaMemcpyAsync(c.fft_tw[a], tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice, c.stream);
            if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "twiddles");
        }
    }
    ALLOC(c.partials, double, (size_t)NSLOT * MAX_BLOCKS);
    ALLOC(c.results, double, NSLOT);
    ALLOC(c.dev_status, int, 1);
    if (cudaMallocHost(&c.host_results, sizeof(double) * NSLOT) != cudaSuccess ||
        cudaMallocHost(&c.host_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, PIC_ERR_OOM, "pinned host allocation failed");
    }
    cudaMemsetAsync(c.partials, 0, sizeof(double) * (size_t)NSLOT * MAX_BLOCKS, c.stream);
    cudaMemsetAsync(c.results, 0, sizeof(double) * NSLOT, c.stream);
    cudaMemsetAsync(c.dev_status, 0, sizeof(int), c.stream);
    return check_cuda(ctx, "allocate");
}

// out = sigma1 (-Delta_h)^+ rhs on the non-null modes, by Chebyshev iteration from zero (rhs
// must have no null-mode part; out is projected off them).  spare: a scratch mesh field.
void poisson_into(Ctx& c, const double* rhs, double* out, double* spare) {
    const int64_t N = c.m.ncell;
    double lmax = 0.0, lmin = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        double mx, mn;
        sin2_range(c.cfg.n[ax], mx, mn);
        lmax += mx * c.invH[ax] * c.invH[ax];
        if (mn > 0.0) {
            double v = mn * c.invH[ax] * c.invH[ax];
            lmin = lmin == 0.0 ? v : std::min(lmin, v);
        }
    }
    launch_fill(c, out, N, 0.0);
    if (!(lmin > 0.0)) return;
    std::vector<double> al(4096), be(4096);
    const int it = cheb_schedule(lmin / c.cfg.sigma1, lmax / c.cfg.sigma1, c.cfg.helmholtz_tol, al.data(), be.data(), 4096);
    double* x = out;
    double* sp = spare;
    launch_helmholtz(c, rhs, 0.0, 1.0 / c.cfg.sigma1, 1, it, al.data(), be.data(), &x, &sp);
    if (x != out) cudaMemcpyAsync(out, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream);
    launch_null_project(c, out, 0.0);
}

// -Delta_h phi = sigma1 rho on the non-null modes by Chebyshev iteration (rho projected).
pic_status solve_poisson(pic_ctx* ctx) {
    Ctx& c = ctx->c;
    const int64_t N = c.m.ncell;
    if (c.cfg.ops == PIC_OPS_SPECTRAL) {
        launch_spec_poisson(c);
        return check_cuda(ctx, "poisson");
    }
    double lmax = 0.0, lmin = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
        double mx, mn;
        sin2_range(c.cfg.n[ax], mx, mn);
        lmax += mx * c.invH[ax] * c.invH[ax];
        if (mn > 0.0) {
            double v = mn * c.invH[ax] * c.invH[ax];
            lmin = lmin == 0.0 ? v : std::min(lmin, v);
        }
    }
    // (0 I - (1/sigma1) Delta_h) phi = rho  <=>  -Delta_h phi = sigma1 rho; initial guess 0
    cudaMemcpyAsync(c.rhs, c.rho0, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream);
    launch_fill(c, c.F0, N, 0.0);
    if (lmin > 0.0) {
        std::vector<double> al(4096), be(4096);
        int it = cheb_schedule(lmin / c.cfg.sigma1, lmax / c.cfg.sigma1, c.cfg.helmholtz_tol, al.data(), be.data(), 4096);
        double* x = c.F0;
        double* spare = c.F1b;
        launch_helmholtz(c, c.rhs, 0.0, 1.0 / c.cfg.sigma1, 1, it, al.data(), be.data(), &x, &spare);
        if (x != c.F0) cudaMemcpyAsync(c.F0, x, sizeof(double) * N, cudaMemcpyDeviceToDevice, c.stream);
        launch_null_project(c, c.F0, 0.0);
    }
    return check_cuda(ctx, "poisson");
}

}  // namespace


namespace {

// Energy of the current state into results[S_K], results[S_W0].
void queue_energy(Ctx& c) {
    launch_kinetic(c);
    launch_finalize(c, S_K, 1, particle_blocks(c), false);
    if (c.cfg.ops == PIC_OPS_SPECTRAL) launch_spec_energy(c, c.F0, c.W0, S_W0);
    else launch_mesh_energy(c, c.F0, c.W0, S_W0);
    launch_finalize(c, S_W0, 1, mesh_blocks(c), false);
}

// Per-step mesh set-up: the CN right-hand-side part of level n (stencils), or the transforms
// of level n (spectral operators).
void mesh_begin(Ctx& c) {
    if (c.cfg.ops == PIC_OPS_SPECTRAL) launch_spec_begin(c);
    else launch_rhs0(c);
}

// The mesh half of one Algorithm 1 iteration: continuity, CN solve (warm-started from F1),
// back-substitution and the gather table.
// tol: the Chebyshev solve's relative accuracy (helmholtz_tol when not positive).
void mesh_phase(Ctx& c, const double* Jcur, const double* Jprev, double tol = 0.0) {
    ProfScope ps(c, PH_MESH);
    if (c.cfg.ops == PIC_OPS_SPECTRAL) {
        launch_spec_mesh_phase(c, Jcur, Jprev);
        return;
    }
    launch_source(c, Jcur, Jprev);
    if (c.helm_fft) {
        launch_helmholtz_fft_refined(c, c.F1);   // to roundoff: the tolerance does not apply
    } else {
        launch_helmholtz_cn(c, &c.F1, &c.F1b, tol > 0.0 ? std::max(tol, c.cfg.helmholtz_tol) : c.cfg.helmholtz_tol);
    }
    launch_backsub_table(c, false);
}

// PIC_MIXED: the fields of an FP32 iteration need no more accuracy than its iterate has
// (e_v >= ~1e-9), and those of an FP64 refinement iteration no more than a thousandth of
// mixed_tol64; the final sweep's mesh phase, which the committed step uses, keeps
// helmholtz_tol.
constexpr double MESH_TOL32 = 1e-10;

// ---- one time step as a sequence of issue / finish phases --------------------------------
//
// step_begin queues the start of a step; then, until the iteration loop ends, iter_issue
// queues one Algorithm 1 iteration and iter_finish (after the stream has been waited for)
// evaluates its residuals; final_issue queues the final sweep and final_finish commits.
// A single context runs the phases back to back (run_step); an ensemble interleaves them
// over its runs so that their kernels overlap on the GPU.

void step_begin(Ctx& c) {
    StepRun& r = c.run;
    const int64_t N = c.m.ncell, np = c.np;
    r = StepRun{};
    // a device error of an earlier call (reported then) does not outlive it: the committed
    // state was kept, so the context is usable again
    cudaMemsetAsync(c.dev_status, 0, sizeof(int), c.stream);
    c.have_accepted = false;
    c.fresh_init = false;
    if (np > 0 && c.cfg.sort_every > 0 && c.steps % c.cfg.sort_every == 0) {
        ProfScope ps(c, PH_SORT);
        launch_sort(c);
    }
    if (c.cfg.diagnostics) queue_energy(c);
    mesh_begin(c);
    cudaMemcpyAsync(c.F1, c.F0, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, c.stream);
    if (np > 0) cudaMemsetAsync(c.slide, 0, (size_t)np, c.stream);   // sliding marks live one step
    c.hist_ev.clear();
    c.hist_eJ.clear();
    c.hist_fp32.clear();
    // PIC_MIXED: the iterations run in FP32 until they reach mixed_tol32 (or stop improving),
    // then in FP64 from the FP32 iterate.
    r.fp32 = c.cfg.precision == PIC_MIXED && np > 0;
    r.began32 = r.fp32;
    cudaMemsetAsync(c.J[r.cur], 0, sizeof(double) * 3 * N, c.stream);
    {
        ProfScope ps(c, PH_SCATTER);
        if (r.fp32) {
            launch_to32(c);
            launch_scatter32(c, c.J[r.cur]);
        } else {
            launch_first_scatter(c, c.J[r.cur], nullptr);
        }
    }
    launch_finalize(c, S_JSCALE, 1, particle_blocks(c), false);
}

// The trial final sweep (PIC_MIXED, see iter_finish): the final sweep of v* = v^{p+1} with
// the residual sums of v* itself; final_issue then has nothing left to queue if it passes.
void trial_issue(Ctx& c) {
    StepRun& r = c.run;
    std::swap(c.vit, c.vnew);
    mesh_phase(c, c.J[r.next], nullptr);
    {
        ProfScope ps(c, PH_COMMIT);
        launch_push(c, c.vit, c.vnew, nullptr, true, false);
    }
    launch_finalize(c, S_EV_NUM, 2, particle_blocks(c), false);
    queue_results(c);
}

// Queue iteration r.p and the copy of its residual sums.
void iter_issue(Ctx& c) {
    StepRun& r = c.run;
    if (r.trial) {
        trial_issue(c);
        return;
    }
    const int64_t N = c.m.ncell;
    const double mesh_tol = r.fp32 ? MESH_TOL32
                            : (r.began32 && c.cfg.mixed_tol64 > 0.0 ? 1e-3 * c.cfg.mixed_tol64 : 0.0);
    mesh_phase(c, c.J[r.cur], r.p > 0 ? c.J[r.prev] : nullptr, mesh_tol);
    if (r.fp32) {
        launch_table32(c);
        cudaMemsetAsync(c.J[r.next], 0, sizeof(double) * 3 * N, c.stream);
        {
            ProfScope ps(c, PH_PUSH32);
            launch_push32(c, c.J[r.next]);
        }
        launch_finalize(c, S_EV_NUM, 2, push32_blocks(c), false);
        launch_finalize(c, S_EJ_NUM, 2, mesh_blocks(c), false);
        if (c.prof) launch_finalize(c, S_CHUNKS32, 2, push32_blocks(c), false);
    } else {
        cudaMemsetAsync(c.J[r.next], 0, sizeof(double) * 3 * N, c.stream);
        r.pair_issued = r.pair;
        if (r.pair) {
            // PIC_MIXED refinement: the particle half in FP32 pairs from the pair table
            launch_table_df(c);
            ProfScope ps(c, PH_PUSHPAIR);
            launch_push_df(c, c.vit, c.vnew, c.J[r.next]);
        } else {
            ProfScope ps(c, PH_PUSH);
            launch_push(c, c.vit, c.vnew, c.J[r.next], false, false);
        }
        if (c.cfg.picard_accel) {
            ProfScope ps(c, PH_LOCAL);
            launch_local(c, c.vit, c.vnew, c.J[r.next]);
        }
        // the current fixed-point error of this update: J(v^{p+1}) against J(v^p)
        launch_jdiff(c, c.J[r.next], c.J[r.cur]);
        launch_finalize(c, S_EV_NUM, 2, particle_blocks(c), false);
        if (c.cfg.picard_accel) launch_finalize(c, S_EVL_NUM, 2, local_blocks(c), false);
        launch_finalize(c, S_EJ_NUM, 2, mesh_blocks(c), false);
        if (c.prof) launch_finalize(c, S_PIECES_PUSH, 2, particle_blocks(c), false);
        if (c.prof && c.cfg.picard_accel) launch_finalize(c, S_LOCAL_SOLVES, 4, local_blocks(c), false);
        c.last_v = c.vit;
        c.last_g = c.vnew;
    }
    queue_results(c);
}

// After iter_issue's work has completed: residuals, convergence, buffer rotation.  Sets
// r.iterating = false when the loop is over (converged, or p_max reached).
pic_status iter_finish(pic_ctx* ctx) {
    Ctx& c = ctx->c;
    StepRun& r = c.run;
    const int64_t N = c.m.ncell;
    const double* h = c.host_results;
    if (r.trial) {
        // the trial final sweep of v* = v^{p+1}: its own residual ||G(v*) - v*|| / ||G(v*)||
        r.trial = false;
        const double num = h[S_EV_NUM], den = h[S_EV_DEN];
        const double res = den > 0.0 ? std::sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
        c.hist_ev.push_back(res);
        c.hist_eJ.push_back(NAN);
        c.hist_fp32.push_back(3);
        if (!std::isfinite(res)) return fail(ctx, PIC_ERR_NONFINITE, "pic_step: non-finite residual of the final sweep");
        // the measured ratio of residual to current change, for the next predictions (a larger
        // one at once, a smaller one halfway, so that one quiet step does not license the next)
        if (r.trial_eJ > 0.0 && std::isfinite(r.trial_eJ))
            c.trial_kappa = std::max(res / r.trial_eJ, 0.5 * c.trial_kappa);
        if (res <= c.cfg.mixed_tol64) {
            r.e_v = res;
            r.converged = true;
            r.iterating = false;
            r.final_done = true;
            r.after32 = false;
            return PIC_OK;
        }
        // rejected: the FP64 iterations continue from v^{p+1} (now in vit) as after any
        // iteration; the sweep's mesh fields are those of J(v^{p+1}), the next one's warm start
        r.e_v64_prev = r.e_v;
        ++r.p64;
        r.after32 = false;
        r.hist = r.p64 >= (r.began32 ? 2 : 1);
        r.rotate();
        if (r.p == c.cfg.picard_max) {
            r.iterating = false;
            return PIC_OK;
        }
        ++r.p;
        return PIC_OK;
    }
    if (r.p == 0) r.jscale = std::sqrt((double)N) * std::fabs(c.q) * h[S_JSCALE] / c.volume;
    {
        // FP64 iterations: the change of the orbit current made by this update, J(v^{p+1})
        // against J(v^p) (k_jdiff), the same update e_v measures.  FP32 iterations: the
        // mesh phase's J^p against J^{p-1} (one update late; they stop on e_v alone).
        double num = std::sqrt(h[S_EJ_NUM]), den = std::sqrt(h[S_EJ_DEN]) + r.jscale;
        const double ej = den > 0.0 ? num / den : (num > 0.0 ? INFINITY : 0.0);
        r.e_J = (r.fp32 && r.p == 0) ? INFINITY : ej;
    }
    if (r.fp32) {
        if (c.prof) {
            c.prof_acc.push32_chunks += (int64_t)h[S_CHUNKS32];
            c.prof_acc.push32_chunks_global += (int64_t)h[S_CHUNKS32_GLOBAL];
        }
        r.e_v = h[S_EV_DEN] > 0.0 ? std::sqrt(h[S_EV_NUM] / h[S_EV_DEN]) : 0.0;
        c.hist_ev.push_back(r.e_v);
        c.hist_eJ.push_back(r.e_J);
        c.hist_fp32.push_back(1);
        if (!std::isfinite(r.e_v)) return fail(ctx, PIC_ERR_NONFINITE, "pic_step: non-finite FP32 residual");
        ++r.p32;
        if (r.p32 == 1) r.e_v32_first = r.e_v;
        else if (r.p32 == 2 && r.e_v32_first > 0.0) r.rho32 = r.e_v / r.e_v32_first;
        // the FP32 iterations' e_J measures the change that iteration p - 1 made to v, so e_v
        // alone says that the FP32 iterate has reached the FP32 noise floor
        const bool reached = r.e_v <= c.cfg.mixed_tol32;
        const bool stalled = r.p32 > 1 && r.e_v > 0.5 * r.e_v32_prev;
        r.e_v32_prev = r.e_v;
        std::swap(c.vit32, c.vnew32);
        r.rotate();
        if (reached || stalled || r.p32 >= c.cfg.mixed_max32) {
            // continue in FP64 from the FP32 iterate; its current is recomputed in FP64 (the
            // fixed-point rounding of the FP32 current would cost one more FP64 iteration)
            launch_from32(c, c.vit32, c.vnew);   // vnew is free until the next push
            cudaMemsetAsync(c.J[r.cur], 0, sizeof(double) * 3 * N, c.stream);
            {
                ProfScope ps(c, PH_SCATTER);
                launch_first_scatter(c, c.J[r.cur], c.vnew);   // also copies the iterate into vit
            }
            // the previous FP32 iterate as v^{p-1}: the first FP64 iteration already sends the
            // particles that the FP32 loop left unconverged (a change that did not shrink, above
            // the FP32 rounding) to the particle-local solve
            launch_from32(c, c.vnew32, c.vnew);
            r.fp32 = false;
            r.hist = c.cfg.picard_accel != 0;
            r.after32 = true;
            r.pair = c.table_pair != nullptr;   // FP32-pair refinement next, if configured
        }
    } else {
        if (c.prof) {
            c.prof_acc.push_pieces += (int64_t)h[S_PIECES_PUSH];
            c.prof_acc.scatter_pieces += (int64_t)h[S_PIECES_SCATTER];
            if (c.cfg.picard_accel) {
                c.prof_acc.local_solves += (int64_t)h[S_LOCAL_SOLVES];
                c.prof_acc.local_evals += (int64_t)h[S_LOCAL_EVALS];
                c.prof_acc.local_failed += (int64_t)h[S_LOCAL_FAILED];
                c.prof_acc.local_failed_unpinned += (int64_t)h[S_LOCAL_FAILED_FREE];
            }
        }
        double num = h[S_EV_NUM], den = h[S_EV_DEN];
        if (c.cfg.picard_accel) {
            num += h[S_EVL_NUM];
            den += h[S_EVL_DEN];
        }
        r.e_v = den > 0.0 ? std::sqrt(num / den) : 0.0;
        c.hist_ev.push_back(r.e_v);
        c.hist_eJ.push_back(r.e_J);
        c.hist_fp32.push_back(r.pair_issued ? 2 : 0);
        if (!std::isfinite(r.e_v) || (r.p > 0 && !std::isfinite(r.e_J)))
            return fail(ctx, PIC_ERR_NONFINITE, "pic_step: non-finite Picard residual");
        if (r.pair_issued) {
            // An FP32-pair iteration never ends the step by Algorithm 1's test: the FP64
            // iterations that follow, or the FP64 final sweep of a trial, check the iterate in
            // FP64.  The pair phase ends once its iterate meets picard_tol (its
            // fixed point is the FP64 one to ~1e-15 of the speed), stops shrinking, or has run
            // mixed_pair_max iterations.
            ++r.ppair;
            const bool met = r.e_v <= c.cfg.picard_tol && r.e_J <= c.cfg.picard_tol;
            const bool stalled = r.ppair > 1 && r.e_v > 0.5 * r.e_vpair_prev;
            r.e_vpair_prev = r.e_v;
            if (met || stalled || r.ppair >= c.cfg.mixed_pair_max) r.pair = false;
        }
        // PIC_MIXED: the FP64 refinement that follows the FP32 phase stops at mixed_tol64
        const double tol = (r.began32 && c.cfg.mixed_tol64 > 0.0) ? c.cfg.mixed_tol64 : c.cfg.picard_tol;
        if (!r.pair_issued && r.e_v <= tol && r.e_J <= tol) {
            r.converged = true;
            r.iterating = false;
            return PIC_OK;
        }
        // PIC_MIXED: the FP64 or FP32-pair iterate v^{p+1} is tried as v* when its predicted
        // residual is within mixed_tol64; the FP64 final sweep of the trial measures that
        // residual and commits only if it is within (trial_issue).  The prediction: the residual left by an update is
        // driven by the change of the current it made, so once a trial has measured the ratio
        // kappa = ||G(v*) - v*|| / e_J, 2 kappa e_J; before that, the contraction seen so far
        // (the FP32 phase's e_v[1] / e_v[0] after the first FP64 iteration, else the last two
        // FP64 e_v) times e_v.
        if (r.began32 && c.cfg.mixed_tol64 > 0.0 && !c.cfg.diagnostics) {
            double pred = INFINITY;
            if (c.trial_kappa > 0.0 && std::isfinite(r.e_J)) {
                pred = 2.0 * c.trial_kappa * r.e_J;
            } else {
                const double rho = r.after32 ? r.rho32 : (r.e_v64_prev > 0.0 ? r.e_v / r.e_v64_prev : 0.0);
                if (rho > 0.0 && rho < 1.0) pred = rho * r.e_v;
            }
            if (pred <= c.cfg.mixed_tol64) {
                r.trial = true;
                r.trial_eJ = r.e_J;
                return PIC_OK;
            }
        }
        r.e_v64_prev = r.e_v;
        if (r.p == c.cfg.picard_max) {
            r.iterating = false;
            return PIC_OK;
        }
        std::swap(c.vit, c.vnew);
        // vnew now holds v^p, the iterate before the next one.  After an FP32 phase the first
        // FP64 change is the FP32 rounding of each particle, not its own contraction: the
        // second FP64 iteration skips the slow-particle test (the first ran it against the last
        // FP32 change, above the rounding floor), the third resumes it.
        ++r.p64;
        r.after32 = false;
        r.hist = r.p64 >= (r.began32 ? 2 : 1);
        r.rotate();
    }
    if (r.p == c.cfg.picard_max) {   // the last iteration ran in FP32
        r.iterating = false;
        return PIC_OK;
    }
    ++r.p;
    return PIC_OK;
}

// The loop is over: record the step info; refuse an unconverged step unless accepted.
pic_status iter_close(pic_ctx* ctx, pic_step_info* last) {
    Ctx& c = ctx->c;
    const StepRun& r = c.run;
    if (last) {
        last->iterations = std::min(r.p, c.cfg.picard_max) + 1;
        last->iterations_fp32 = r.p32;
        last->iterations_pair = r.ppair;
        last->converged = r.converged ? 1 : 0;
        last->e_v = r.e_v;
        last->e_J = r.e_J;
    }
    c.last_failed = !r.converged;
    if (!r.converged && !c.cfg.accept_unconverged) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "pic_step: Picard not converged after %d iterations (e_v=%.3e, e_J=%.3e)",
                      c.cfg.picard_max + 1, r.e_v, r.e_J);
        return fail(ctx, PIC_ERR_NO_CONVERGENCE, buf);
    }
    return PIC_OK;
}

// Final consistency sweep (§5.4): orbit of v^{n+1,p+1}, whose current is in J[next].
void final_issue(Ctx& c) {
    const StepRun& r = c.run;
    if (r.final_done) {   // the trial final sweep already ran and passed
        queue_results(c);
        return;
    }
    const bool diag = c.cfg.diagnostics != 0;
    std::swap(c.vit, c.vnew);
    double* Jfin = c.J[r.next];
    mesh_phase(c, Jfin, nullptr);
    {
        ProfScope ps(c, PH_COMMIT);
        launch_push(c, c.vit, c.vnew, nullptr, true, diag);
    }
    if (diag) {
        launch_finalize(c, S_K1, 3, particle_blocks(c), false);   // K1, PWORK, RA_SQ
        launch_finalize(c, S_RA_MAX, 2, particle_blocks(c), true);
        if (c.cfg.ops == PIC_OPS_SPECTRAL) launch_spec_diag(c, Jfin);
        else launch_mesh_diag(c, Jfin);
        launch_finalize(c, S_MWORK, 2, mesh_blocks(c), false);    // MWORK, W
        launch_finalize(c, S_G_MAX, 1, mesh_blocks(c), true);
        launch_finalize(c, S_G_SQ, 1, mesh_blocks(c), false);
        launch_finalize(c, S_R_MAX, 1, mesh_blocks(c), true);
        launch_finalize(c, S_R_SQ, 1, mesh_blocks(c), false);
        launch_finalize(c, S_CONT_MAX, 1, mesh_blocks(c), true);
    }
    queue_results(c);
}

// After final_issue's work has completed: commit level n+1 and the diagnostics.
void final_finish(Ctx& c) {
    const StepRun& r = c.run;
    const int64_t N = c.m.ncell, np = c.np;
    // commit: level n+1 becomes level n; v^{n-1} <- v^n
    std::swap(c.F0, c.F1);
    std::swap(c.W0, c.W1);
    std::swap(c.rho0, c.rho1);
    std::swap(c.xi, c.xi_new);
    std::swap(c.P, c.P_new);
    std::swap(c.vprev, c.v);
    std::swap(c.v, c.vnew);
    c.steps += 1;
    c.have_accepted = true;   // vit: the final sweep's iterate; slide: this step's sliding marks
    if (c.cfg.diagnostics) {
        const double* h = c.host_results;
        pic_diag_t& d = c.diag;
        const double dt = c.cfg.dt;
        d.K0 = h[S_K];
        d.W0 = h[S_W0];
        d.K1 = h[S_K1];
        d.W1 = h[S_W];
        d.particle_work = h[S_PWORK];
        d.mesh_work = h[S_MWORK];
        d.R_field = d.W1 - d.W0 + dt * d.mesh_work;
        d.R_particle = d.K1 - d.K0 - dt * d.particle_work;
        d.R_total = (d.K1 + d.W1) - (d.K0 + d.W0);
        d.RA_max = h[S_RA_MAX];
        d.RA_rms = np > 0 ? std::sqrt(h[S_RA_SQ] / (3.0 * np)) : 0.0;
        d.partition_max = h[S_PU_MAX];
        d.gauge_max = h[S_G_MAX];
        d.gauge_rms = std::sqrt(h[S_G_SQ] / (double)N);
        d.gauss_max = h[S_R_MAX];
        d.gauss_rms = std::sqrt(h[S_R_SQ] / (double)N);
        d.continuity_max = h[S_CONT_MAX];
        d.picard_iterations = std::min(r.p, c.cfg.picard_max) + 1;
        d.e_v = r.e_v;
        d.e_J = r.e_J;
        c.have_diag = true;
    }
}

// One time step.  On failure nothing of the committed state (F0, W0, rho0, xi, v, P, vprev)
// has changed except the particle order, which get_state undoes.
pic_status run_step(pic_ctx* ctx, pic_step_info* last) {
    Ctx& c = ctx->c;
    step_begin(c);
    while (c.run.iterating) {
        iter_issue(c);
        pic_status s = wait_results(ctx, c.run.fp32 ? "pic_step (fp32)" : "pic_step");
        if (s == PIC_OK) s = iter_finish(ctx);
        if (s != PIC_OK) return s;
    }
    pic_status s = iter_close(ctx, last);
    if (s != PIC_OK) return s;
    final_issue(c);
    s = wait_results(ctx, "pic_step final sweep");
    if (s != PIC_OK) return s;
    final_finish(c);
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_config_default(pic_config* cfg) {
    if (!cfg) return PIC_ERR_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    const double side = 2.0 * M_PI / 3.0;
    for (int a = 0; a < 3; ++a) {
        cfg->n[a] = 8;
        cfg->L[a] = side;
    }
    cfg->dt = 0.1;
    cfg->kappa = cfg->sigma1 = cfg->sigma2 = 1.0;
    cfg->n0 = 1.0;
    cfg->picard_tol = 1e-13;
    cfg->picard_max = 16;
    cfg->split_orbit_at_knots = 1;
    cfg->quadrature = PIC_QUAD_CLOSED;
    cfg->nq = 16;
    cfg->precision = PIC_FP64;
    cfg->sort_every = 1;
    cfg->diagnostics = 0;
    cfg->accept_unconverged = 0;
    cfg->picard_accel = 1;
    cfg->mixed_tol32 = 1e-9;
    cfg->mixed_max32 = 8;
    cfg->mixed_pair_max = 1;
    cfg->deterministic = 0;
    cfg->shape_order = 1;
    cfg->ops = PIC_OPS_CENTRAL2;
    cfg->helmholtz_tol = 1e-17;
    return PIC_OK;
}

pic_status pic_init(const pic_config* cfg, const pic_particles* particles, const pic_allocator* alloc, void* stream,
                    pic_ctx** out) {
    if (!cfg || !particles || !out) return PIC_ERR_ARG;
    *out = nullptr;
    if (validate(cfg) != PIC_OK) return PIC_ERR_ARG;
    if (particles->np < 0 || (particles->np > 0 && (!particles->x || !particles->v)) || !(particles->m > 0.0))
        return PIC_ERR_ARG;
    if (alloc && (!alloc->alloc || !alloc->free)) return PIC_ERR_ARG;
    pic_ctx* ctx = new (std::nothrow) pic_ctx();
    if (!ctx) return PIC_ERR_OOM;
    Ctx& c = ctx->c;
    c.cfg = *cfg;
    c.stream = (cudaStream_t)stream;
    if (alloc) {
        c.alloc = *alloc;
        c.has_alloc = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return PIC_ERR_CUDA;
    }
    c.np = particles->np;
    c.q = particles->q;
    c.mass = particles->m;
    setup_geometry(c);
    pic_status s = allocate(ctx);
    if (s != PIC_OK) {
        free_all(ctx);
        delete ctx;
        return s;
    }
    if (cfg->quadrature == PIC_QUAD_GAUSS) set_gauss_rule(cfg->nq);
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kind = particles->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (np > 0) {
        // positions to the scratch buffer, then wrapped cell units; velocities straight in
        cudaMemcpyAsync(c.sort_tmp, particles->x, sizeof(double) * 3 * np, kind, c.stream);
        cudaMemcpyAsync(c.v, particles->v, sizeof(double) * 3 * np, kind, c.stream);
        launch_init_positions(c, c.sort_tmp);
        if (c.cfg.sort_every > 0) {
            cudaMemcpyAsync(c.vprev, c.v, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, c.stream);
            cudaMemcpyAsync(c.P, c.v, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, c.stream);
            launch_sort(c);
        }
    }
    // rho^0 = sum q S / dV + n0, null modes removed; phi^0 from Poisson; psi = A = U = 0
    launch_fill(c, c.rho0, N, 0.0);
    if (np > 0) launch_point_deposit(c);
    launch_null_project(c, c.rho0, c.cfg.n0);
    s = solve_poisson(ctx);
    if (s == PIC_OK) {
        launch_fill(c, c.F0 + N, 3 * N, 0.0);
        launch_fill(c, c.W0, 4 * N, 0.0);
        if (np > 0) {
            // v^{n-1} = v^0 and P = m v + q A_h(x) = m v since A^0 = 0
            cudaMemcpyAsync(c.vprev, c.v, sizeof(double) * 3 * np, cudaMemcpyDeviceToDevice, c.stream);
            launch_scale_copy(c, c.P, c.v, 3 * np, c.mass);
        }
    }
    if (s == PIC_OK) s = sync_results(ctx, "pic_init");
    if (s != PIC_OK) {
        free_all(ctx);
        delete ctx;
        return s;
    }
    c.fresh_init = true;
    *out = ctx;
    return PIC_OK;
}


pic_status pic_step(pic_ctx* ctx, int32_t nsteps, pic_step_info* info) {
    if (!ctx || nsteps < 0) return PIC_ERR_ARG;
    ctx->c.err.clear();
    pic_step_info local{};
    pic_step_info last{};
    pic_status s = PIC_OK;
    for (int k = 0; k < nsteps; ++k) {
        s = run_step(ctx, &last);
        if (s != PIC_OK) break;
        local.steps_done += 1;
        local.total_iterations += last.iterations;
        local.total_iterations_fp32 += last.iterations_fp32;
        local.total_iterations_pair += last.iterations_pair;
    }
    local.iterations = last.iterations;
    local.iterations_fp32 = last.iterations_fp32;
    local.iterations_pair = last.iterations_pair;
    local.converged = last.converged;
    local.e_v = last.e_v;
    local.e_J = last.e_J;
    if (info) *info = local;
    return s;
}

pic_status pic_energy(pic_ctx* ctx, pic_energy_t* out) {
    if (!ctx || !out) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    queue_energy(c);
    pic_status s = sync_results(ctx, "pic_energy");
    if (s != PIC_OK) return s;
    out->K = c.host_results[S_K];
    out->W = c.host_results[S_W0];
    out->total = out->K + out->W;
    return PIC_OK;
}

pic_status pic_diagnostics(pic_ctx* ctx, pic_diag_t* out) {
    if (!ctx || !out) return PIC_ERR_ARG;
    if (!ctx->c.have_diag) return fail(ctx, PIC_ERR_ARG, "pic_diagnostics: no step with diagnostics = 1 has run");
    *out = ctx->c.diag;
    return PIC_OK;
}

pic_status pic_get_state(pic_ctx* ctx, const pic_state_view* dst) {
    if (!ctx || !dst) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kind = dst->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (np > 0) {
        double* outs[4] = {dst->x, dst->v, dst->P, dst->vprev};
        const double* srcs[4] = {c.xi, c.v, c.P, c.vprev};
        for (int k = 0; k < 4; ++k) {
            if (!outs[k]) continue;
            double sc[3] = {1.0, 1.0, 1.0};
            if (k == 0) sc[0] = c.H[0], sc[1] = c.H[1], sc[2] = c.H[2];
            launch_unpermute(c, srcs[k], c.sort_tmp, sc[0], sc[1], sc[2]);
            cudaMemcpyAsync(outs[k], c.sort_tmp, sizeof(double) * 3 * np, kind, c.stream);
        }
    }
    if (dst->phi) cudaMemcpyAsync(dst->phi, c.F0, sizeof(double) * N, kind, c.stream);
    if (dst->A) cudaMemcpyAsync(dst->A, c.F0 + N, sizeof(double) * 3 * N, kind, c.stream);
    if (dst->psi) cudaMemcpyAsync(dst->psi, c.W0, sizeof(double) * N, kind, c.stream);
    if (dst->U) cudaMemcpyAsync(dst->U, c.W0 + N, sizeof(double) * 3 * N, kind, c.stream);
    if (dst->rho) cudaMemcpyAsync(dst->rho, c.rho0, sizeof(double) * N, kind, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_get_state");
    return check_cuda(ctx, "pic_get_state");
}

pic_status pic_set_state(pic_ctx* ctx, const pic_state_view* src) {
    if (!ctx || !src) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    const int64_t np = c.np, N = c.m.ncell;
    if (np > 0 && (!src->x || !src->v || !src->P || !src->vprev)) return PIC_ERR_ARG;
    if (!src->phi || !src->psi || !src->rho || !src->A || !src->U) return PIC_ERR_ARG;
    const cudaMemcpyKind kind = src->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (np > 0) {
        // the given order becomes the device order (identity permutation)
        cudaMemcpyAsync(c.sort_tmp, src->x, sizeof(double) * 3 * np, kind, c.stream);
        launch_init_positions(c, c.sort_tmp);
        cudaMemcpyAsync(c.v, src->v, sizeof(double) * 3 * np, kind, c.stream);
        cudaMemcpyAsync(c.P, src->P, sizeof(double) * 3 * np, kind, c.stream);
        cudaMemcpyAsync(c.vprev, src->vprev, sizeof(double) * 3 * np, kind, c.stream);
    }
    cudaMemcpyAsync(c.F0, src->phi, sizeof(double) * N, kind, c.stream);
    cudaMemcpyAsync(c.F0 + N, src->A, sizeof(double) * 3 * N, kind, c.stream);
    cudaMemcpyAsync(c.W0, src->psi, sizeof(double) * N, kind, c.stream);
    cudaMemcpyAsync(c.W0 + N, src->U, sizeof(double) * 3 * N, kind, c.stream);
    cudaMemcpyAsync(c.rho0, src->rho, sizeof(double) * N, kind, c.stream);
    c.have_diag = false;
    c.have_accepted = false;
    c.fresh_init = false;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_set_state");
    return check_cuda(ctx, "pic_set_state");
}

pic_status pic_iterate(pic_ctx* ctx, const double* v_iter, int32_t on_device, const pic_iterate_out* out) {
    if (!ctx || !v_iter || !out) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = out->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double* vgiven = nullptr;
    cudaMemsetAsync(c.dev_status, 0, sizeof(int), c.stream);
    c.have_accepted = false;   // vit and slide are overwritten below
    if (np > 0) {
        cudaMemcpyAsync(c.vnew, v_iter, sizeof(double) * 3 * np, kin, c.stream);
        launch_permute_in(c, c.vnew, c.sort_tmp, 1.0, 1.0, 1.0);   // caller order -> device order
        vgiven = c.sort_tmp;
    }
    mesh_begin(c);
    cudaMemcpyAsync(c.F1, c.F0, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, c.stream);
    cudaMemsetAsync(c.J[0], 0, sizeof(double) * 3 * N, c.stream);
    if (np > 0) launch_first_scatter(c, c.J[0], vgiven);
    mesh_phase(c, c.J[0], nullptr);
    if (np > 0) {
        cudaMemsetAsync(c.slide, 0, (size_t)np, c.stream);   // no local solves in a single body
        launch_push(c, c.vit, c.vnew, nullptr, true, false);
    }
    pic_status s = sync_results(ctx, "pic_iterate");
    if (s != PIC_OK) return s;
    if (out->J) cudaMemcpyAsync(out->J, c.J[0], sizeof(double) * 3 * N, kout, c.stream);
    if (out->rho) cudaMemcpyAsync(out->rho, c.rho1, sizeof(double) * N, kout, c.stream);
    if (out->phi) cudaMemcpyAsync(out->phi, c.F1, sizeof(double) * N, kout, c.stream);
    if (out->A) cudaMemcpyAsync(out->A, c.F1 + N, sizeof(double) * 3 * N, kout, c.stream);
    if (out->psi) cudaMemcpyAsync(out->psi, c.W1, sizeof(double) * N, kout, c.stream);
    if (out->U) cudaMemcpyAsync(out->U, c.W1 + N, sizeof(double) * 3 * N, kout, c.stream);
    if (np > 0) {
        double* outs[3] = {out->x, out->P, out->v};
        const double* srcs[3] = {c.xi_new, c.P_new, c.vnew};
        for (int k = 0; k < 3; ++k) {
            if (!outs[k]) continue;
            double sc[3] = {1.0, 1.0, 1.0};
            if (k == 0) sc[0] = c.H[0], sc[1] = c.H[1], sc[2] = c.H[2];
            launch_unpermute(c, srcs[k], c.sort_tmp, sc[0], sc[1], sc[2]);
            cudaMemcpyAsync(outs[k], c.sort_tmp, sizeof(double) * 3 * np, kout, c.stream);
        }
    }
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_iterate");
    return check_cuda(ctx, "pic_iterate");
}

pic_status pic_get_positions(pic_ctx* ctx, double* xi, int32_t on_device) {
    if (!ctx || !xi) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.np == 0) return PIC_OK;
    launch_unpermute(c, c.xi, c.sort_tmp, 1.0, 1.0, 1.0);
    cudaMemcpyAsync(xi, c.sort_tmp, sizeof(double) * 3 * c.np,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_get_positions");
    return check_cuda(ctx, "pic_get_positions");
}

pic_status pic_set_positions(pic_ctx* ctx, const double* xi, int32_t on_device) {
    if (!ctx || !xi) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.np == 0) return PIC_OK;
    cudaMemcpyAsync(c.sort_tmp, xi, sizeof(double) * 3 * c.np,
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.stream);
    launch_set_positions(c, c.sort_tmp);
    c.have_diag = false;
    c.have_accepted = false;
    c.fresh_init = false;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_set_positions");
    return check_cuda(ctx, "pic_set_positions");
}

pic_status pic_get_iterate(pic_ctx* ctx, double* v_iter, double* g_iter, int32_t on_device) {
    if (!ctx || !v_iter || !g_iter) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.np == 0) return PIC_OK;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (!c.last_v || !c.last_g || !c.last_failed)
        return fail(ctx, PIC_ERR_ARG, "pic_get_iterate: only available after a pic_step that did not converge");
    // the image G(v^p): the next iterate with the locally solved particles' plain image
    // restored, assembled in P_new (3 * np, unused between steps)
    cudaMemcpyAsync(c.P_new, c.last_g, sizeof(double) * 3 * c.np, cudaMemcpyDeviceToDevice, c.stream);
    if (c.cfg.picard_accel) launch_patch_local(c, c.P_new);
    launch_unpermute(c, c.P_new, c.sort_tmp, 1.0, 1.0, 1.0);
    cudaMemcpyAsync(g_iter, c.sort_tmp, sizeof(double) * 3 * c.np, kind, c.stream);
    launch_unpermute(c, c.last_v, c.sort_tmp, 1.0, 1.0, 1.0);
    cudaMemcpyAsync(v_iter, c.sort_tmp, sizeof(double) * 3 * c.np, kind, c.stream);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_get_iterate");
    return check_cuda(ctx, "pic_get_iterate");
}

pic_status pic_get_accepted(pic_ctx* ctx, double* v_iter, uint8_t* slide, int32_t on_device) {
    if (!ctx || (!v_iter && !slide)) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (!c.have_accepted)
        return fail(ctx, PIC_ERR_ARG, "pic_get_accepted: only available right after a committed pic_step");
    if (c.np == 0) return PIC_OK;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (v_iter) {
        launch_unpermute(c, c.vit, c.sort_tmp, 1.0, 1.0, 1.0);
        cudaMemcpyAsync(v_iter, c.sort_tmp, sizeof(double) * 3 * c.np, kind, c.stream);
    }
    if (slide) {
        // the bytes go through the free scratch array sort_tmp (8 * 3 * np bytes >= np)
        uint8_t* tmp = reinterpret_cast<uint8_t*>(c.sort_tmp);
        launch_slide_out(c, tmp);
        cudaMemcpyAsync(slide, tmp, (size_t)c.np, kind, c.stream);
    }
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_get_accepted");
    return check_cuda(ctx, "pic_get_accepted");
}

// ---- adjoint --------------------------------------------------------------------------------

}  // extern "C"

namespace {

pic_status adj_alloc(pic_ctx* ctx) {
    Ctx& c = ctx->c;
    if (c.adj_tab) return PIC_OK;
    const int64_t np3 = 3 * std::max<int64_t>(c.np, 1), N = c.m.ncell;
    ALLOC(c.adj_xe, double, np3);
    ALLOC(c.adj_v, double, np3);
    ALLOC(c.adj_P, double, np3);
    ALLOC(c.adj_mu, double, np3);
    ALLOC(c.adj_mu2, double, np3);
    ALLOC(c.adj_xi, double, np3);
    ALLOC(c.adj_g, double, np3);
    ALLOC(c.adj_tmp, double, np3);
    ALLOC(c.adj_vn, double, np3);
    ALLOC(c.adj_Pn, double, np3);
    ALLOC(c.adj_B, double, 3 * np3);
    ALLOC(c.adj_F1, double, 4 * N);
    ALLOC(c.adj_W1, double, 4 * N);
    ALLOC(c.adj_rho1, double, N);
    ALLOC(c.adj_t, double, 4 * N);
    ALLOC(c.adj_pn, double, 4 * N);
    ALLOC(c.adj_y, double, 4 * N);
    ALLOC(c.adj_ys, double, 4 * N);
    ALLOC(c.adj_J, double, 3 * N);
    ALLOC(c.adj_F0, double, 4 * N);
    ALLOC(c.adj_W0, double, 4 * N);
    ALLOC(c.adj_rho0, double, N);
    ALLOC(c.adj_tab, double, 9 * N);
    // the transposed solve's restart length: 40, or fewer where the basis would pass 4 GiB
    const size_t vec = sizeof(double) * (size_t)np3;
    c.adj_m = (int)std::max<size_t>(4, std::min<size_t>(40, ((size_t)4 << 30) / vec - 1));
    ALLOC(c.adj_b0, double, np3);
    ALLOC(c.adj_w, double, np3);
    ALLOC(c.adj_V, double, (size_t)(c.adj_m + 1) * np3);
    ALLOC(c.adj_h, double, 2 * (c.adj_m + 2));
    ALLOC(c.adj_part, double, (size_t)(c.adj_m + 2) * MAX_BLOCKS);
    return check_cuda(ctx, "adjoint buffers");
}

// Particle array (3 np, caller order, host or device) -> device order, times s per component.
void adj_in(Ctx& c, const double* src, cudaMemcpyKind kind, double* dst, const double s[3]) {
    if (src) {
        cudaMemcpyAsync(c.sort_tmp, src, sizeof(double) * 3 * c.np, kind, c.stream);
        launch_permute_in(c, c.sort_tmp, dst, s[0], s[1], s[2]);
    } else {
        cudaMemsetAsync(dst, 0, sizeof(double) * 3 * c.np, c.stream);
    }
}

void adj_out(Ctx& c, const double* src, double* dst, cudaMemcpyKind kind, const double s[3]) {
    if (!dst) return;
    launch_unpermute(c, src, c.sort_tmp, s[0], s[1], s[2]);
    cudaMemcpyAsync(dst, c.sort_tmp, sizeof(double) * 3 * c.np, kind, c.stream);
}

void mesh_in(Ctx& c, const double* src, cudaMemcpyKind kind, double* dst, int64_t n) {
    if (src) cudaMemcpyAsync(dst, src, sizeof(double) * n, kind, c.stream);
    else cudaMemsetAsync(dst, 0, sizeof(double) * n, c.stream);
}

void mesh_out(Ctx& c, const double* src, double* dst, cudaMemcpyKind kind, int64_t n) {
    if (dst) cudaMemcpyAsync(dst, src, sizeof(double) * n, kind, c.stream);
}

// One transposed sweep at (level n, v*) for the velocity-output adjoint lam_v + mu: the mesh
// adjoints (adj_F0, adj_W0, adj_rho0, adj_J), and per particle adj_xi, adj_g, adj_B.
void adj_sweep(Ctx& c, const double* xi_n, const double* v_n, const double* vstar) {
    const int64_t N = c.m.ncell;
    const double a = 0.25 * c.cfg.kappa * c.cfg.kappa * c.cfg.dt * c.cfg.dt;
    cudaMemsetAsync(c.adj_tab, 0, sizeof(double) * 9 * N, c.stream);
    launch_adj_scatter(c, xi_n, v_n, vstar, c.adj_P, c.adj_v, c.adj_mu, c.adj_tab);
    launch_adj_mesh_rhs(c, c.adj_tab, c.adj_F1, c.adj_W1, c.adj_t, c.adj_pn);
    cudaMemsetAsync(c.adj_y, 0, sizeof(double) * 4 * N, c.stream);
    double* y = c.adj_y;
    double* ys = c.adj_ys;
    launch_helmholtz(c, c.adj_t, 1.0, a, 4, c.cheb_iters, c.cheb_alpha, c.cheb_beta, &y, &ys);
    launch_adj_mesh_out(c, y, c.adj_pn, c.adj_W1, c.adj_rho1, c.adj_F0, c.adj_W0, c.adj_rho0, c.adj_J);
    launch_adj_derivs(c, xi_n, v_n, vstar, c.adj_J, c.adj_P, c.adj_v, c.adj_xe, c.adj_mu, c.adj_xi, c.adj_g, c.adj_vn,
                      c.adj_Pn, c.adj_B);
}

// The transposed fixed point (I - K) mu = b0 (g(mu) = K mu + b0 is a sweep's adjoint of v*) by
// restarted GMRES, right-preconditioned with the forward step's splitting (launch_adj_precond).
// Each restart cycle starts from the true residual r = g(mu) - mu and checks |P r| / |mu|, the
// size of a preconditioned correction relative to mu, against tol.  On success c.adj_mu holds
// mu and the last sweep's outputs are those at mu.
pic_status adj_solve(pic_ctx* ctx, const double* xi_n, const double* v_n, const double* vstar, double tol,
                     int max_sweeps, int* sweeps_out, double* res_out) {
    Ctx& c = ctx->c;
    const int64_t n = 3 * c.np;
    const int m = c.adj_m;
    const size_t vb = sizeof(double) * (size_t)n;
    double* V = c.adj_V;
    double* sol = c.adj_mu2;
    std::vector<double> hb(2 * (m + 2), 0.0);
    auto fetch = [&](int count) {
        cudaMemcpyAsync(hb.data(), c.adj_h, sizeof(double) * count, cudaMemcpyDeviceToHost, c.stream);
        return sync_results(ctx, "pic_step_vjp");
    };
    int sweeps = 0;
    cudaMemsetAsync(c.adj_mu, 0, vb, c.stream);
    adj_sweep(c, xi_n, v_n, vstar);
    ++sweeps;
    cudaMemcpyAsync(c.adj_b0, c.adj_g, vb, cudaMemcpyDeviceToDevice, c.stream);
    cudaMemsetAsync(sol, 0, vb, c.stream);
    launch_adj_mdot(c, n, c.adj_b0, c.adj_b0, n, 1, c.adj_part, c.adj_h);
    pic_status s = fetch(1);
    if (s != PIC_OK) return s;
    if (!std::isfinite(hb[0])) return fail(ctx, PIC_ERR_NONFINITE, "pic_step_vjp: non-finite adjoint");
    *sweeps_out = sweeps;
    *res_out = 0.0;
    if (hb[0] == 0.0) return PIC_OK;   // mu = 0, and the sweep just made is at mu
    std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), gam(m + 1), y(m);
    auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
    std::string trace;
    double res = INFINITY, best = INFINITY, target_ratio = 1e-4;
    for (int cycle = 0;; ++cycle) {
        // the true residual r = g(mu) - mu (b0 at mu = 0) in V_0, and the check
        if (cycle == 0) {
            cudaMemcpyAsync(V, c.adj_b0, vb, cudaMemcpyDeviceToDevice, c.stream);
        } else {
            cudaMemcpyAsync(c.adj_mu, sol, vb, cudaMemcpyDeviceToDevice, c.stream);
            adj_sweep(c, xi_n, v_n, vstar);
            ++sweeps;
            launch_scale_copy(c, V, c.adj_g, n, 1.0);
            launch_adj_axpy(c, n, V, sol, -1.0);
        }
        launch_adj_precond(c, c.adj_B, V, c.adj_w);
        launch_adj_mdot(c, n, V, V, n, 1, c.adj_part, c.adj_h);
        launch_adj_mdot(c, n, c.adj_w, c.adj_w, n, 1, c.adj_part, c.adj_h + 1);
        launch_adj_mdot(c, n, sol, sol, n, 1, c.adj_part, c.adj_h + 2);
        s = fetch(3);
        if (s != PIC_OK) return s;
        const double beta = std::sqrt(hb[0]);
        res = cycle == 0 ? INFINITY : (hb[2] > 0.0 ? std::sqrt(hb[1] / hb[2]) : (hb[1] > 0.0 ? INFINITY : 0.0));
        if (!std::isfinite(beta) || (cycle > 0 && std::isnan(res)))
            return fail(ctx, PIC_ERR_NONFINITE, "pic_step_vjp: non-finite adjoint");
        best = std::min(best, res);
        if (cycle > 0) {
            char buf[48];
            std::snprintf(buf, sizeof(buf), "%s%d: %.2e", trace.empty() ? "" : ", ", sweeps, res);
            trace += buf;
        }
        if (res <= tol || beta == 0.0) break;
        if (sweeps >= max_sweeps) {
            return fail(ctx, PIC_ERR_NO_CONVERGENCE,
                        "pic_step_vjp: the transposed fixed point did not converge (sweeps: residual " + trace + ")");
        }
        // the reduction of |r| this cycle aims at: enough for tol, if the ratio of the checked
        // residual to |r| stays as it is
        if (cycle > 0) target_ratio = std::min(1e-4, std::max(1e-10, 0.25 * tol / res));
        launch_scale_copy(c, V, V, n, 1.0 / beta);
        std::fill(gam.begin(), gam.end(), 0.0);
        gam[0] = beta;
        int j = 0;
        while (j < m && sweeps < max_sweeps) {
            double* vj = V + (size_t)j * n;
            double* vj1 = V + (size_t)(j + 1) * n;
            launch_adj_precond(c, c.adj_B, vj, c.adj_mu);   // z_j = P v_j
            adj_sweep(c, xi_n, v_n, vstar);
            ++sweeps;
            launch_adj_apply(c, n, c.adj_mu, c.adj_g, c.adj_b0, vj1);   // (I - K) z_j
            // classical Gram--Schmidt, twice
            launch_adj_mdot(c, n, vj1, V, n, j + 1, c.adj_part, c.adj_h);
            launch_adj_combine(c, n, vj1, V, n, j + 1, c.adj_h, -1.0);
            launch_adj_mdot(c, n, vj1, V, n, j + 1, c.adj_part, c.adj_h + (m + 2));
            launch_adj_combine(c, n, vj1, V, n, j + 1, c.adj_h + (m + 2), -1.0);
            launch_adj_mdot(c, n, vj1, vj1, n, 1, c.adj_part, c.adj_h + (m + 1));
            s = fetch(2 * (m + 2));
            if (s != PIC_OK) return s;
            for (int k = 0; k <= j; ++k) Hij(k, j) = hb[k] + hb[m + 2 + k];
            const double hn = std::sqrt(hb[m + 1]);
            if (!std::isfinite(hn)) return fail(ctx, PIC_ERR_NONFINITE, "pic_step_vjp: non-finite adjoint");
            Hij(j + 1, j) = hn;
            if (hn > 0.0) launch_scale_copy(c, vj1, vj1, n, 1.0 / hn);
            for (int k = 0; k < j; ++k) {
                const double a = Hij(k, j), b = Hij(k + 1, j);
                Hij(k, j) = cs[k] * a + sn[k] * b;
                Hij(k + 1, j) = -sn[k] * a + cs[k] * b;
            }
            const double a = Hij(j, j), b = Hij(j + 1, j), rr = std::hypot(a, b);
            cs[j] = rr > 0.0 ? a / rr : 1.0;
            sn[j] = rr > 0.0 ? b / rr : 0.0;
            Hij(j, j) = rr;
            Hij(j + 1, j) = 0.0;
            gam[j + 1] = -sn[j] * gam[j];
            gam[j] = cs[j] * gam[j];
            ++j;
            if (std::fabs(gam[j]) <= target_ratio * beta || hn == 0.0) break;
        }
        // mu += P V y, H y = gam (upper triangular)
        for (int k = j - 1; k >= 0; --k) {
            double t = gam[k];
            for (int l = k + 1; l < j; ++l) t -= Hij(k, l) * y[l];
            y[k] = Hij(k, k) != 0.0 ? t / Hij(k, k) : 0.0;
        }
        cudaMemcpyAsync(c.adj_h, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, c.stream);
        cudaMemsetAsync(c.adj_w, 0, vb, c.stream);
        launch_adj_combine(c, n, c.adj_w, V, n, j, c.adj_h, 1.0);
        launch_adj_precond(c, c.adj_B, c.adj_w, c.adj_mu);
        launch_adj_axpy(c, n, sol, c.adj_mu, 1.0);
        s = sync_results(ctx, "pic_step_vjp");   // y is host memory
        if (s != PIC_OK) return s;
    }
    *sweeps_out = sweeps;
    *res_out = res;
    return PIC_OK;
}

}  // namespace

extern "C" {

pic_status pic_step_vjp(pic_ctx* ctx, const pic_state_view* lam_next, const pic_state_view* lam_prev,
                        pic_vjp_info* info) {
    if (!ctx || !lam_next || !lam_prev) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    c.err.clear();
    if (!c.have_accepted)
        return fail(ctx, PIC_ERR_ARG, "pic_step_vjp: only available right after a committed pic_step");
    if (c.cfg.quadrature != PIC_QUAD_CLOSED || c.cfg.shape_order != 1 || c.cfg.ops != PIC_OPS_CENTRAL2)
        return fail(ctx, PIC_ERR_ARG, "pic_step_vjp: needs the closed-form linear orbits and central differences");
    pic_status s = adj_alloc(ctx);
    if (s != PIC_OK) return s;
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kin = lam_next->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = lam_prev->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const double one[3] = {1.0, 1.0, 1.0};
    const double toc[3] = {c.H[0], c.H[1], c.H[2]};        // d/dxi = H d/dx
    const double tox[3] = {c.invH[0], c.invH[1], c.invH[2]};
    // level n and the accepted iterate, as the committed step left them (device order)
    const double* xi_n = c.xi_new;
    const double* v_n = c.vprev;
    const double* vstar = c.vit;
    cudaMemsetAsync(c.dev_status, 0, sizeof(int), c.stream);
    if (np > 0) {
        adj_in(c, lam_next->x, kin, c.adj_xe, toc);
        adj_in(c, lam_next->v, kin, c.adj_v, one);
        adj_in(c, lam_next->P, kin, c.adj_P, one);
        cudaMemsetAsync(c.adj_mu, 0, sizeof(double) * 3 * np, c.stream);
    }
    mesh_in(c, lam_next->phi, kin, c.adj_F1, N);
    mesh_in(c, lam_next->A, kin, c.adj_F1 + N, 3 * N);
    mesh_in(c, lam_next->psi, kin, c.adj_W1, N);
    mesh_in(c, lam_next->U, kin, c.adj_W1 + N, 3 * N);
    mesh_in(c, lam_next->rho, kin, c.adj_rho1, N);
    s = sync_results(ctx, "pic_step_vjp");
    if (s != PIC_OK) return s;
    // the transposed fixed point for mu, to 1e-11 relative: the sweep's own rounding (FP64
    // atomics in an order that varies between calls) sets a floor near 1e-14 of mu per sweep
    int sweeps = 0;
    double res = 0.0;
    if (np > 0) {
        s = adj_solve(ctx, xi_n, v_n, vstar, 1e-11, 400, &sweeps, &res);
        if (s != PIC_OK) return s;
    } else {
        adj_sweep(c, xi_n, v_n, vstar);   // the mesh-only adjoint
        sweeps = 1;
    }
    if (np > 0) {
        adj_out(c, c.adj_xi, lam_prev->x, kout, tox);
        adj_out(c, c.adj_vn, lam_prev->v, kout, one);
        adj_out(c, c.adj_Pn, lam_prev->P, kout, one);
        if (lam_prev->vprev) cudaMemsetAsync(lam_prev->vprev, 0, sizeof(double) * 3 * np, c.stream);
    }
    mesh_out(c, c.adj_F0, lam_prev->phi, kout, N);
    mesh_out(c, c.adj_F0 + N, lam_prev->A, kout, 3 * N);
    mesh_out(c, c.adj_W0, lam_prev->psi, kout, N);
    mesh_out(c, c.adj_W0 + N, lam_prev->U, kout, 3 * N);
    mesh_out(c, c.adj_rho0, lam_prev->rho, kout, N);
    s = sync_results(ctx, "pic_step_vjp");
    if (s != PIC_OK) return s;
    if (info) {
        info->iterations = sweeps;
        info->residual = res;
    }
    return PIC_OK;
}

pic_status pic_energy_vjp(pic_ctx* ctx, const pic_state_view* lam) {
    if (!ctx || !lam) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (c.cfg.ops != PIC_OPS_CENTRAL2) return fail(ctx, PIC_ERR_ARG, "pic_energy_vjp: needs central differences");
    pic_status s = adj_alloc(ctx);
    if (s != PIC_OK) return s;
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kout = lam->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    launch_energy_grad(c, c.adj_F0, c.adj_W0);
    mesh_out(c, c.adj_F0, lam->phi, kout, N);
    mesh_out(c, c.adj_F0 + N, lam->A, kout, 3 * N);
    mesh_out(c, c.adj_W0, lam->psi, kout, N);
    mesh_out(c, c.adj_W0 + N, lam->U, kout, 3 * N);
    double* zeros[5] = {lam->x, lam->v, lam->P, lam->vprev, lam->rho};
    const int64_t counts[5] = {3 * np, 3 * np, 3 * np, 3 * np, N};
    for (int k = 0; k < 5; ++k) {
        if (!zeros[k] || counts[k] == 0) continue;
        if (lam->on_device) cudaMemsetAsync(zeros[k], 0, sizeof(double) * counts[k], c.stream);
        else std::memset(zeros[k], 0, sizeof(double) * counts[k]);
    }
    return sync_results(ctx, "pic_energy_vjp");
}

pic_status pic_init_vjp(pic_ctx* ctx, const pic_state_view* lam0, double* lam_x0, double* lam_v0, int32_t on_device) {
    if (!ctx || !lam0) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    c.err.clear();
    if (!c.fresh_init)
        return fail(ctx, PIC_ERR_ARG, "pic_init_vjp: the state must be pic_init's (no step or set_state since)");
    if (c.cfg.ops != PIC_OPS_CENTRAL2 || c.cfg.shape_order != 1)
        return fail(ctx, PIC_ERR_ARG, "pic_init_vjp: needs central differences and linear shapes");
    pic_status s = adj_alloc(ctx);
    if (s != PIC_OK) return s;
    const int64_t np = c.np, N = c.m.ncell;
    const cudaMemcpyKind kin = lam0->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const double one[3] = {1.0, 1.0, 1.0};
    const double tox[3] = {c.invH[0], c.invH[1], c.invH[2]};
    // phi^0 = sigma1 (-Delta_h)^+ rho^0 and rho^0 = (deposit + n0) off the null modes: both
    // maps are symmetric, so lam_dep = P (lam_rho + sigma1 (-Delta_h)^+ P lam_phi)
    mesh_in(c, lam0->phi, kin, c.adj_t, N);
    mesh_in(c, lam0->rho, kin, c.adj_rho1, N);
    launch_null_project(c, c.adj_t, 0.0);
    poisson_into(c, c.adj_t, c.adj_y, c.adj_ys);
    launch_adj_axpy(c, N, c.adj_rho1, c.adj_y, 1.0);
    launch_null_project(c, c.adj_rho1, 0.0);
    if (np > 0) {
        // positions: the direct adjoint plus the deposit's transpose (cell units, device order)
        cudaMemsetAsync(c.adj_xi, 0, sizeof(double) * 3 * np, c.stream);
        launch_adj_deposit(c, c.xi, c.adj_rho1, c.adj_xi);
        adj_in(c, lam0->x, kin, c.adj_xe, one);
        launch_unpermute(c, c.adj_xi, c.adj_tmp, tox[0], tox[1], tox[2]);   // caller order, physical
        launch_permute_in(c, c.adj_tmp, c.adj_g, 1.0, 1.0, 1.0);           // back to device order
        launch_adj_axpy(c, 3 * np, c.adj_xe, c.adj_g, 1.0);
        adj_out(c, c.adj_xe, lam_x0, kout, one);
        // velocities: v^0 sets v, v^{-1} = v^0 and P^0 = m v^0 (A^0 = 0)
        adj_in(c, lam0->v, kin, c.adj_v, one);
        adj_in(c, lam0->vprev, kin, c.adj_g, one);
        launch_adj_axpy(c, 3 * np, c.adj_v, c.adj_g, 1.0);
        adj_in(c, lam0->P, kin, c.adj_g, one);
        launch_adj_axpy(c, 3 * np, c.adj_v, c.adj_g, c.mass);
        adj_out(c, c.adj_v, lam_v0, kout, one);
    }
    return sync_results(ctx, "pic_init_vjp");
}

pic_status pic_set_wait_limit(pic_ctx* ctx, int64_t cycles) {
    if (!ctx || cycles < 1) return PIC_ERR_ARG;
    ctx->c.wait_cycles = (long long)cycles;
    return PIC_OK;
}

pic_status pic_profile(pic_ctx* ctx, int32_t enable, pic_profile_t* out) {
    if (!ctx) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) return check_cuda(ctx, "pic_profile");
    prof_resolve(c);
    if (out) {
        *out = c.prof_acc;
        out->launches = c.launches;
        c.prof_acc = pic_profile_t{};
        c.launches = 0;
    }
    c.prof = enable != 0;
    return check_cuda(ctx, "pic_profile");
}

int32_t pic_residual_history(const pic_ctx* ctx, int32_t cap, double* e_v, double* e_J, int32_t* fp32) {
    if (!ctx) return -1;
    const Ctx& c = ctx->c;
    const int32_t n = (int32_t)c.hist_ev.size();
    for (int32_t k = 0; k < n && k < cap; ++k) {
        if (e_v) e_v[k] = c.hist_ev[k];
        if (e_J) e_J[k] = c.hist_eJ[k];
        if (fp32) fp32[k] = c.hist_fp32[k];
    }
    return n;
}

// ---- autotuning of the particle-kernel grids ---------------------------------------------------

}  // extern "C"

namespace {

struct TuneKey {
    int n[3];
    int64_t np_bucket;
    int precision;
    bool operator<(const TuneKey& o) const {
        return std::tie(n[0], n[1], n[2], np_bucket, precision) <
               std::tie(o.n[0], o.n[1], o.n[2], o.np_bucket, o.precision);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;   // -> (push_bps, push32_bps)

// Mean duration (ms) of `reps` launches queued by `launch`, after one untimed launch.
template <typename F>
float time_launches(Ctx& c, int reps, F&& launch) {
    launch();
    cudaEvent_t a = take_event(c), b = take_event(c);
    cudaEventRecord(a, c.stream);
    for (int k = 0; k < reps; ++k) launch();
    cudaEventRecord(b, c.stream);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    c.ev_pool.push_back(a);
    c.ev_pool.push_back(b);
    return ms / reps;
}

}  // namespace

extern "C" {

pic_status pic_autotune(pic_ctx* ctx, int32_t* push_blocks_per_sm, int32_t* push32_blocks_per_sm) {
    if (!ctx) return PIC_ERR_ARG;
    Ctx& c = ctx->c;
    c.err.clear();
    const TuneKey key{{c.m.n[0], c.m.n[1], c.m.n[2]}, c.np >> 14, c.cfg.precision};
    bool cached = c.cfg.deterministic != 0;   // deterministic mode keeps the default grids
    if (!cached) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            c.push_bps = it->second.first;
            c.push32_bps = it->second.second;
            cached = true;
        }
    }
    if (!cached && c.np > 0) {
        // One Algorithm 1 iteration body from the extrapolated guess sets up the mesh table;
        // everything written is scratch (iterates, next current, creeping list), nothing of
        // the committed state changes.
        const int64_t N = c.m.ncell;
        cudaMemsetAsync(c.dev_status, 0, sizeof(int), c.stream);
        c.have_accepted = false;   // the timing launches overwrite vit and slide
        mesh_begin(c);
        cudaMemcpyAsync(c.F1, c.F0, sizeof(double) * 4 * N, cudaMemcpyDeviceToDevice, c.stream);
        cudaMemsetAsync(c.J[0], 0, sizeof(double) * 3 * N, c.stream);
        launch_first_scatter(c, c.J[0], nullptr);
        mesh_phase(c, c.J[0], nullptr);
        c.run.hist = false;   // scratch timing: no iterate history
        const int cand[4] = {2, 4, 8, 16};
        float best = INFINITY;
        int best_bps = c.push_bps;
        for (int bps : cand) {
            c.push_bps = bps;
            const float ms = time_launches(c, 2, [&] {
                launch_push(c, c.vit, c.vnew, c.J[1], false, false);
                if (c.cfg.picard_accel) launch_local(c, c.vit, c.vnew, c.J[1]);
            });
            if (ms < best) {
                best = ms;
                best_bps = bps;
            }
        }
        c.push_bps = best_bps;
        if (c.cfg.precision == PIC_MIXED) {
            launch_to32(c);
            launch_table32(c);
            const int cand32[3] = {4, 8, 16};
            float best32 = INFINITY;
            int best32_bps = c.push32_bps;
            for (int bps : cand32) {
                c.push32_bps = bps;
                const float ms = time_launches(c, 2, [&] {
                    cudaMemsetAsync(c.J[1], 0, sizeof(double) * 3 * N, c.stream);
                    launch_push32(c, c.J[1]);
                });
                if (ms < best32) {
                    best32 = ms;
                    best32_bps = bps;
                }
            }
            c.push32_bps = best32_bps;
        }
        pic_status s = sync_results(ctx, "pic_autotune");
        if (s != PIC_OK) return s;
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = {c.push_bps, c.push32_bps};
    }
    if (push_blocks_per_sm) *push_blocks_per_sm = c.push_bps;
    if (push32_blocks_per_sm) *push32_blocks_per_sm = c.push32_bps;
    return check_cuda(ctx, "pic_autotune");
}

// ---- ensembles -----------------------------------------------------------------------------

}  // extern "C"

struct pic_ensemble {
    std::vector<pic_ctx*> runs;
    std::vector<cudaStream_t> streams;
    std::string err;
};

extern "C" {

pic_status pic_ensemble_init(int32_t nruns, const pic_config* cfgs, const pic_particles* particles,
                             const pic_allocator* alloc, pic_ensemble** out) {
    if (!out || nruns < 1 || !cfgs || !particles) return PIC_ERR_ARG;
    *out = nullptr;
    pic_ensemble* e = new (std::nothrow) pic_ensemble;
    if (!e) return PIC_ERR_OOM;
    for (int32_t i = 0; i < nruns; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            pic_ensemble_destroy(e);
            return PIC_ERR_CUDA;
        }
        e->streams.push_back(st);
        pic_ctx* c = nullptr;
        pic_status s = pic_init(&cfgs[i], &particles[i], alloc, (void*)st, &c);
        if (s != PIC_OK) {
            pic_ensemble_destroy(e);
            return s;
        }
        e->runs.push_back(c);
    }
    *out = e;
    return PIC_OK;
}

int32_t pic_ensemble_size(const pic_ensemble* e) { return e ? (int32_t)e->runs.size() : -1; }

pic_ctx* pic_ensemble_run(pic_ensemble* e, int32_t i) {
    if (!e || i < 0 || i >= (int32_t)e->runs.size()) return nullptr;
    return e->runs[i];
}

pic_status pic_ensemble_step(pic_ensemble* e, int32_t nsteps, pic_step_info* infos, pic_status* statuses) {
    if (!e || nsteps < 0) return PIC_ERR_ARG;
    const int R = (int)e->runs.size();
    std::vector<pic_step_info> acc(R), last(R);
    std::vector<pic_status> st(R, PIC_OK);
    std::vector<int> pending, finals;
    for (int k = 0; k < nsteps; ++k) {
        pending.clear();
        finals.clear();
        for (int r = 0; r < R; ++r) {
            if (st[r] != PIC_OK) continue;   // a failed run stays at its last committed step
            Ctx& c = e->runs[r]->c;
            c.err.clear();
            step_begin(c);
            iter_issue(c);
            pending.push_back(r);
        }
        // Poll the runs' streams; a run whose iteration has completed is evaluated and its
        // next iteration (or its final sweep) is queued at once, while the others compute.
        while (!pending.empty()) {
            bool progressed = false;
            for (size_t j = 0; j < pending.size();) {
                const int r = pending[j];
                pic_ctx* ctx = e->runs[r];
                const cudaError_t q = cudaStreamQuery(ctx->c.stream);
                if (q == cudaErrorNotReady) {
                    ++j;
                    continue;
                }
                progressed = true;
                pic_status s = wait_results(ctx, "pic_ensemble_step");
                if (s == PIC_OK) s = iter_finish(ctx);
                if (s == PIC_OK && ctx->c.run.iterating) {
                    iter_issue(ctx->c);
                    ++j;
                    continue;
                }
                if (s == PIC_OK) s = iter_close(ctx, &last[r]);
                if (s == PIC_OK) {
                    final_issue(ctx->c);
                    finals.push_back(r);
                } else {
                    st[r] = s;
                }
                pending.erase(pending.begin() + (long)j);
            }
            if (!progressed) std::this_thread::yield();
        }
        for (int r : finals) {
            pic_ctx* ctx = e->runs[r];
            pic_status s = wait_results(ctx, "pic_ensemble_step final sweep");
            if (s != PIC_OK) {
                st[r] = s;
                continue;
            }
            final_finish(ctx->c);
            acc[r].steps_done += 1;
            acc[r].total_iterations += last[r].iterations;
            acc[r].total_iterations_fp32 += last[r].iterations_fp32;
            acc[r].total_iterations_pair += last[r].iterations_pair;
        }
    }
    pic_status first = PIC_OK;
    e->err.clear();
    for (int r = 0; r < R; ++r) {
        acc[r].iterations = last[r].iterations;
        acc[r].iterations_fp32 = last[r].iterations_fp32;
        acc[r].iterations_pair = last[r].iterations_pair;
        acc[r].converged = last[r].converged;
        acc[r].e_v = last[r].e_v;
        acc[r].e_J = last[r].e_J;
        if (infos) infos[r] = acc[r];
        if (statuses) statuses[r] = st[r];
        if (st[r] != PIC_OK && first == PIC_OK) {
            first = st[r];
            e->err = "run " + std::to_string(r) + ": " + e->runs[r]->c.err;
        }
    }
    return first;
}

const char* pic_ensemble_last_error(const pic_ensemble* e) {
    if (!e) return "null ensemble";
    return e->err.c_str();
}

void pic_ensemble_destroy(pic_ensemble* e) {
    if (!e) return;
    for (pic_ctx* c : e->runs) pic_destroy(c);
    for (cudaStream_t st : e->streams) cudaStreamDestroy(st);
    delete e;
}

const char* pic_last_error(const pic_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->c.err.c_str();
}

void pic_destroy(pic_ctx* ctx) {
    if (!ctx) return;
    cudaStreamSynchronize(ctx->c.stream);
    prof_resolve(ctx->c);
    for (cudaEvent_t e : ctx->c.ev_pool) cudaEventDestroy(e);
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
