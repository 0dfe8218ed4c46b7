// C entry points, context management and the host-side orchestration of one
// OC iteration (paper Section 2.5).  Every arithmetic step of the path runs
// in this library's CUDA kernels; the host only sequences launches, reads a
// few device scalars per solve chunk and fills the iteration record.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace to3d;

namespace to3d {

const char* status_name(to3d_status s) {
    switch (s) {
        case TO3D_OK: return "ok";
        case TO3D_EINVAL: return "invalid argument";
        case TO3D_ENOMEM: return "out of memory";
        case TO3D_ECUDA: return "CUDA error";
        case TO3D_ENOCONV: return "no convergence within the iteration limit";
        case TO3D_ENUMERIC: return "numerical breakdown (NaN/Inf or non-positive curvature)";
        case TO3D_ETIMEOUT: return "device-side wait timed out";
        case TO3D_ESTATE: return "invalid state";
    }
    return "unknown status";
}

to3d_status set_err(to3d_ctx* c, to3d_status s, const std::string& msg) {
    if (c) c->err = std::string(status_name(s)) + ": " + msg;
    return s;
}
to3d_status cuda_check(to3d_ctx* c, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TO3D_OK;
    return set_err(c, e == cudaErrorMemoryAllocation ? TO3D_ENOMEM : TO3D_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}
to3d_status launch_check(to3d_ctx* c, const char* what) {
    return cuda_check(c, cudaGetLastError(), what);
}

// ------------------------------------------------------------------ KE
// Unit-modulus hex8 stiffness from the tensor-product closed form.  With
// linear 1D shape functions N_0 = 1 - t, N_1 = t on [0, 1]:
//   M = int N_a N_b = [[1/3, 1/6], [1/6, 1/3]],   S = int N_a' N_b' = [[1, -1], [-1, 1]],
//   C = int N_a' N_b = [[-1/2, -1/2], [1/2, 1/2]].
// G_pq[a][b] = int d_p N_a d_q N_b dV is a product of one 1D factor per
// axis (S on an axis carrying both derivatives, C or C^T on an axis carrying
// one, M otherwise), and isotropic elasticity gives
//   KE[(a,i),(b,j)] = lam G_ij[a][b] + mu (delta_ij sum_k G_kk[a][b] + G_ji[a][b]).
// 72 G is integer, which gives the exact integer split used by the tensor cores.
static void hex8_split(double A_lam[576], double A_mu[576]) {
    const double M[2][2] = {{1.0 / 3, 1.0 / 6}, {1.0 / 6, 1.0 / 3}};
    const double S[2][2] = {{1.0, -1.0}, {-1.0, 1.0}};
    const double C[2][2] = {{-0.5, -0.5}, {0.5, 0.5}};
    auto G = [&](int p, int q, int a, int b) {
        double v = 1.0;
        for (int d = 0; d < 3; ++d) {
            const int ad = (a >> d) & 1, bd = (b >> d) & 1;
            if (d == p && d == q) v *= S[ad][bd];
            else if (d == p) v *= C[ad][bd];
            else if (d == q) v *= C[bd][ad];
            else v *= M[ad][bd];
        }
        return v;
    };
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b)
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    const int r = 3 * a + i, c = 3 * b + j;
                    A_lam[r * 24 + c] = 72.0 * G(i, j, a, b);
                    double m = G(j, i, a, b);
                    if (i == j) m += G(0, 0, a, b) + G(1, 1, a, b) + G(2, 2, a, b);
                    A_mu[r * 24 + c] = 72.0 * m;
                }
}

static bool build_ke(to3d_ctx* c) {
    double Al[576], Am[576];
    hex8_split(Al, Am);
    const double nu = c->prm.nu;
    const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
    for (int k = 0; k < 576; ++k) {
        const double rl = std::nearbyint(Al[k]), rm = std::nearbyint(Am[k]);
        if (std::fabs(rl - Al[k]) > 1e-9 || std::fabs(rm - Am[k]) > 1e-9) return false;
        c->kes.a_lam[k] = (float)rl;
        c->kes.a_mu[k] = (float)rm;
        c->ke.v[k] = lam / 72.0 * rl + mu / 72.0 * rm;
    }
    c->kes.c_lam = lam / 72.0;
    c->kes.c_mu = mu / 72.0;
    return true;
}

// Unit-modulus KE for Poisson ratio nu (same derivation as build_ke).
bool unit_ke(double nu, KE64* out) {
    double Al[576], Am[576];
    hex8_split(Al, Am);
    const double lam = nu / ((1 + nu) * (1 - 2 * nu)), mu = 1.0 / (2 * (1 + nu));
    for (int k = 0; k < 576; ++k) {
        const double rl = std::nearbyint(Al[k]), rm = std::nearbyint(Am[k]);
        if (std::fabs(rl - Al[k]) > 1e-9 || std::fabs(rm - Am[k]) > 1e-9) return false;
        out->v[k] = lam / 72.0 * rl + mu / 72.0 * rm;
    }
    return true;
}

static bool build_stencil(to3d_ctx* c) {
    const double rmin = c->prm.rmin;
    const int R = (int)std::ceil(rmin);
    if (R > 15) return false;
    Stencil* st = c->st;
    st->n = 0;
    st->radius = R;
    for (int dk = -R; dk <= R; ++dk)
        for (int dj = -R; dj <= R; ++dj)
            for (int di = -R; di <= R; ++di) {
                const double w = rmin - std::sqrt((double)(di * di + dj * dj + dk * dk));
                if (w > 0.0) {
                    if (st->n >= kMaxStencil) return false;
                    st->off[st->n] = (di + 16) | ((dj + 16) << 8) | ((dk + 16) << 16);
                    st->w[st->n] = w;
                    st->n++;
                }
            }
    return st->n > 0;
}

}  // namespace to3d

// ------------------------------------------------------------------ helpers
#define CK(call)                                                         \
    do {                                                                 \
        to3d_status _s = cuda_check(c, (call), #call);                   \
        if (_s != TO3D_OK) return _s;                                    \
    } while (0)
#define LK(what)                                                         \
    do {                                                                 \
        to3d_status _s = launch_check(c, what);                          \
        if (_s != TO3D_OK) return _s;                                    \
    } while (0)

template <typename T>
static cudaError_t dalloc(T** p, size_t n) {
    return cudaMalloc((void**)p, (n ? n : 1) * sizeof(T));
}

static void free_all(to3d_ctx* c) {
    destroy_mg(c);
    if (c->xphys) cudaFree(c->xphys);
    void* ptrs[] = {c->x, c->xnew, c->E, c->E32, c->ce, c->dc, c->dcf, c->Hs, c->ocq, c->oclo,
                    c->ochi, c->ocs, c->passive, c->nodemask, c->dinv, c->dinv32, c->f, c->ftmp, c->u,
                    c->r, c->p, c->q, c->tmp, c->d32, c->r32, c->p32a, c->p32b, c->q32,
                    c->stage, c->red.partials, c->red.counter, c->ss, c->os, c->misc,
                    c->dev_err, c->tcB, c->maskp};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->ss_h) cudaFreeHost(c->ss_h);
    if (c->os_h) cudaFreeHost(c->os_h);
    if (c->misc_h) cudaFreeHost(c->misc_h);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    for (auto& row : c->kev)
        for (auto& e : row)
            if (e) cudaEventDestroy(e);
    if (c->g_pcg64) cudaGraphExecDestroy(c->g_pcg64);
    if (c->g_pcg32) cudaGraphExecDestroy(c->g_pcg32);
    if (c->g_iter) cudaGraphExecDestroy(c->g_iter);
    if (c->cap_stream2) cudaStreamDestroy(c->cap_stream2);
    if (c->cap_stream3) cudaStreamDestroy(c->cap_stream3);
    if (c->dcctl) cudaFree(c->dcctl);
    if (c->dcctl_h) cudaFreeHost(c->dcctl_h);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c->st;
    destroy_cnn(c);
}

// Device pointer for an input: the caller's pointer, or a staged copy.
static to3d_status stage_in(to3d_ctx* c, const void* src, size_t bytes, int on_device,
                            size_t slot, const void** out) {
    if (on_device) {
        *out = src;
        return TO3D_OK;
    }
    if ((slot + 1) * c->stage_slot > c->stage_bytes || bytes > c->stage_slot)
        return set_err(c, TO3D_EINVAL, "staging buffer too small");
    char* dst = (char*)c->stage + slot * c->stage_slot;
    CK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, c->stream));
    *out = dst;
    return TO3D_OK;
}

static double* stage_out(to3d_ctx* c, void* dst, int on_device, size_t slot) {
    return on_device ? (double*)dst : (double*)((char*)c->stage + slot * c->stage_slot);
}

static to3d_status finish_out(to3d_ctx* c, void* dst, const void* dev, size_t bytes,
                              int on_device) {
    if (!on_device) {
        CK(cudaMemcpyAsync(dst, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return TO3D_OK;
}

static to3d_status sync_scalars(to3d_ctx* c) {
    CK(cudaMemcpyAsync(c->ss_h, c->ss, sizeof(SolverScalars), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TO3D_OK;
}

// ------------------------------------------------------------------ solvers
static constexpr int kSampleEvery = 4;

// After a captured chunk that started at solver iteration it0 has completed,
// add the sampled matvec durations of the iterations that did work.
static void accumulate_kernel_times(to3d_ctx* c, int which, int it0, int it1) {
    for (int sl = 0; sl < c->kslots[which]; ++sl) {
        if (it0 + c->kslot_iter[which][sl] >= it1) continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->kev[which][2 * sl], c->kev[which][2 * sl + 1]) ==
            cudaSuccess) {
            c->kt_ms[which] += ms;
            c->kt_n[which] += 1;
        }
    }
    cudaGetLastError();
}

// ------------------------------------------------------------------
// Launch `n` iterations of the FP64 PCG, through a captured graph when the
// chunk matches the captured length.
static to3d_status pcg64_chunk(to3d_ctx* c, int n) {
    if (n == c->chunk) {
        if (!c->g_pcg64) {
            cudaGraph_t gr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            c->kslots[1] = 0;
            for (int i = 0; i < n; ++i) {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (i % kSampleEvery == 0 && c->kslots[1] < to3d_ctx::kTimedSlots) {
                    const int sl = c->kslots[1]++;
                    e0 = c->kev[1][2 * sl];
                    e1 = c->kev[1][2 * sl + 1];
                    c->kslot_iter[1][sl] = i;
                }
                launch_pcg64_iter(c, c->cap_stream, e0, e1);
            }
            CK(cudaStreamEndCapture(c->cap_stream, &gr));
            CK(cudaGraphInstantiate(&c->g_pcg64, gr, 0));
            cudaGraphDestroy(gr);
            c->launches -= 3 * n;
        }
        CK(cudaGraphLaunch(c->g_pcg64, c->stream));
        c->launches += 3 * n;
    } else {
        for (int i = 0; i < n; ++i) launch_pcg64_iter(c, c->stream);
    }
    LK("pcg64 chunk");
    return TO3D_OK;
}

static to3d_status pcg32_chunk(to3d_ctx* c, int prec, int n) {
    // n is even so the direction ping-pong stays in phase across chunks
    if (n == c->chunk) {
        if (!c->g_pcg32 || c->g_pcg32_prec != prec) {
            if (c->g_pcg32) cudaGraphExecDestroy(c->g_pcg32);
            c->g_pcg32 = nullptr;
            cudaGraph_t gr;
            CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            c->kslots[0] = 0;
            for (int i = 0; i < n; ++i) {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (i % kSampleEvery == 0 && c->kslots[0] < to3d_ctx::kTimedSlots) {
                    const int sl = c->kslots[0]++;
                    e0 = c->kev[0][2 * sl];
                    e1 = c->kev[0][2 * sl + 1];
                    c->kslot_iter[0][sl] = i;
                }
                launch_pcg32_iter(c, c->cap_stream, prec, i & 1, e0, e1);
            }
            CK(cudaStreamEndCapture(c->cap_stream, &gr));
            CK(cudaGraphInstantiate(&c->g_pcg32, gr, 0));
            cudaGraphDestroy(gr);
            c->g_pcg32_prec = prec;
            c->launches -= 2 * n;
        }
        CK(cudaGraphLaunch(c->g_pcg32, c->stream));
        c->launches += 2 * n;
    } else {
        for (int i = 0; i < n; ++i) launch_pcg32_iter(c, c->stream, prec, i & 1);
    }
    LK("pcg32 chunk");
    return TO3D_OK;
}

// r = f - K u (FP64) and rr_true = |r|^2 into ss; returns |r| / |f| on host.
static to3d_status true_residual(to3d_ctx* c, const double* f, double fnorm, double* relres) {
    launch_matvec64(c, c->stream, c->E, c->u, c->q, false);
    launch_residual64(c, c->stream, f, c->q, c->r, true);
    LK("residual");
    to3d_status s = sync_scalars(c);
    if (s) return s;
    *relres = fnorm > 0 ? std::sqrt(c->ss_h->rr_true) / fnorm : 0.0;
    return TO3D_OK;
}

static to3d_status solve_f64(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    const double tol = c->prm.cg_rtol;
    const double tol2 = tol * tol * fnorm * fnorm;
    int total = 0, restarts = 0;
    double relres = 0.0;
    to3d_status st = true_residual(c, f, fnorm, &relres);
    if (st) return st;
    int status = TO3D_OK;
    while (relres > tol && fnorm > 0) {
        launch_ss_reset(c, c->stream, tol2, c->prm.cg_maxit - total);
        launch_pcg64_init(c, c->stream);
        LK("pcg64 init");
        int n = 16, it0 = 0;
        for (;;) {
            const int chunk_n = n < c->chunk ? n : c->chunk;
            if ((st = pcg64_chunk(c, chunk_n))) return st;
            if ((st = sync_scalars(c))) return st;
            if (chunk_n == c->chunk) accumulate_kernel_times(c, 1, it0, c->ss_h->it);
            it0 = c->ss_h->it;
            if (c->ss_h->done) break;
            if (n < c->chunk) n *= 2;
        }
        total += c->ss_h->it;
        status = c->ss_h->status;
        if ((st = true_residual(c, f, fnorm, &relres))) return st;
        if (status != TO3D_OK || relres <= tol || ++restarts > 4 || total >= c->prm.cg_maxit) break;
    }
    if (status == TO3D_OK && relres > tol) status = TO3D_ENOCONV;
    if (status == TO3D_OK && total > 0) c->pcg_its_est = total;
    if (info) {
        info->iters = total;
        info->outer = restarts + 1;
        info->status = status;
        info->relres = relres;
    }
    return TO3D_OK;
}

// FP64 defect correction around one FP32 inner PCG with the tensor-core
// matvec.  The inner CG is not restarted: whenever its recurrence residual
// has dropped by the factor delta (= inner_rtol) since the last replacement,
// u absorbs the correction d in FP64, the true residual f - K u is formed in
// FP64 and replaces the FP32 residual, and the CG continues from its last
// search direction, re-orthogonalised against the new residual.  When the
// true residual does not halve over a segment the inner CG restarts from it;
// after 8 such stalls a single-slice operand form switches to its two-slice
// form for the rest of the solve.  The solve ends when the true relative
// residual is <= cg_rtol.
constexpr int kEscalateAfterStalls = 8;

static to3d_status solve_dc(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    const double tol = c->prm.cg_rtol;
    const double delta = c->prm.inner_rtol;
    int prec = c->prm.precision;
    const long long ndof = 3 * c->g.nnode;
    int total = 0, outer = 0, status = TO3D_OK, stalls = 0;
    double relres = 0.0;
    to3d_status st;
    if ((st = true_residual(c, f, fnorm, &relres))) return st;
    if (relres > tol && fnorm > 0.0) {
        // unit-RMS scaling of the inner system, fixed for the whole solve
        const double scale = 1.0 / std::sqrt(c->ss_h->rr_true / (double)ndof);
        const double relres0 = relres;
        const double t = 0.5 * tol * fnorm * scale;
        const double target2 = t * t;
        launch_ss_reset(c, c->stream, std::fmax(delta * delta * (double)ndof, target2), c->prm.cg_maxit);
        launch_pcg32_init(c, c->stream, c->r, scale);
        LK("pcg32 init");
        for (;;) {
            int n = 16, it0 = 0;
            for (;;) {
                const int chunk_n = n < c->chunk ? n : c->chunk;
                if ((st = pcg32_chunk(c, prec, chunk_n))) return st;
                if ((st = sync_scalars(c))) return st;
                if (chunk_n == c->chunk) accumulate_kernel_times(c, 0, it0, c->ss_h->it);
                it0 = c->ss_h->it;
                if (c->ss_h->done) break;
                if (n < c->chunk) n *= 2;
            }
            const int its = c->ss_h->it;
            total += its;
            if (c->ss_h->status == TO3D_ETIMEOUT || c->ss_h->status == TO3D_ENUMERIC) {
                status = c->ss_h->status;
                break;
            }
            launch_axpy_d32(c, c->stream, 1.0 / scale);
            LK("axpy");
            const double prev = relres;
            if ((st = true_residual(c, f, fnorm, &relres))) return st;
            if (c->trace)
                std::fprintf(stderr, "to3d: segment %d: %d inner its (total %d), relres %.3e -> %.3e\n",
                             outer, its, total, prev, relres);
            if (relres <= tol) break;
            if (total >= c->prm.cg_maxit || outer >= 1000) {
                status = TO3D_ENOCONV;
                break;
            }
            outer++;
            if (relres > 0.5 * prev) {
                // the recurrence residual ran away from the true one (too
                // coarse an operand): restart the inner CG from the true
                // residual instead of keeping its direction
                if (++stalls > 50) {
                    status = TO3D_ENOCONV;
                    break;
                }
                // a single-slice operand that keeps stalling the outer
                // iteration is too coarse for this system: finish the solve
                // with the two-slice form of the same format
                if (stalls == kEscalateAfterStalls && (prec == TO3D_BF16_DC || prec == TO3D_FP16_DC)) {
                    prec += 1;
                    if (c->trace)
                        std::fprintf(stderr, "to3d: %d stalls, inner operand now form %d\n", stalls, prec);
                }
                launch_ss_reset(c, c->stream,
                                std::fmax(delta * delta * (double)ndof * (relres / relres0) *
                                              (relres / relres0),
                                          target2),
                                c->prm.cg_maxit - total);
                launch_pcg32_init(c, c->stream, c->r, scale);
                LK("pcg32 restart");
                continue;
            }
            // the last direction is in p32a after an odd number of fused
            // iterations; the captured chunks read p_old from p32b first
            if (its & 1)
                CK(cudaMemcpyAsync(c->p32b, c->p32a, sizeof(float) * 3 * c->vol,
                                   cudaMemcpyDeviceToDevice, c->stream));
            launch_ss_segment(c, c->stream, target2, c->prm.cg_maxit - total);
            launch_pcg32_replace(c, c->stream, c->r, scale, c->p32b, delta * delta, target2);
            LK("residual replacement");
        }
    }
    if (info) {
        info->iters = total;
        info->outer = outer + 1;
        info->status = status;
        info->relres = relres;
    }
    return TO3D_OK;
}

static to3d_status prepare_operator(to3d_ctx* c, const double* x) {
    c->xop = x;
    launch_simp(c, c->stream, x);
    launch_diag(c, c->stream, c->E);
    mg_operator_changed(c);
    LK("simp/diag");
    return TO3D_OK;
}

namespace to3d {
to3d_status prepare_op(to3d_ctx* c, const double* x) { return prepare_operator(c, x); }

to3d_status stage_input(to3d_ctx* c, const void* src, size_t bytes, int on_device, size_t slot,
                        const void** out) {
    return stage_in(c, src, bytes, on_device, slot, out);
}

// FP64 Jacobi-PCG from u = 0 for exactly `iters` iterations (rhs f, masked)
to3d_status run_pcg64_iters(to3d_ctx* c, const double* f, int iters) {
    launch_fill_zero(c, c->stream, c->u, sizeof(double) * 3 * c->g.nnode);
    launch_ss_reset(c, c->stream, 0.0, iters);
    launch_mask_copy(c, c->stream, f, c->r);
    launch_pcg64_init(c, c->stream);
    for (int i = 0; i < iters; ++i) launch_pcg64_iter(c, c->stream);
    return launch_check(c, "pcg64 iterations");
}

// FP64 Jacobi-PCG of K u = f to relative residual rtol (u starts at 0)
to3d_status solve64_rtol(to3d_ctx* c, const double* f, double fnorm, double rtol,
                         to3d_solve_info* info) {
    const double keep = c->prm.cg_rtol;
    c->prm.cg_rtol = rtol;
    launch_fill_zero(c, c->stream, c->u, sizeof(double) * 3 * c->g.nnode);
    to3d_status st = solve_f64(c, f, fnorm, info);
    c->prm.cg_rtol = keep;
    return st;
}

to3d_status solve_fcg(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info);
}  // namespace to3d

static to3d_status solve_current(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    if (!c->prm.warm_start || !c->have_u)
        launch_fill_zero(c, c->stream, c->u, sizeof(double) * 3 * c->g.nnode);
    to3d_status st;
    if (c->prm.precond == TO3D_CNN_FCG) st = solve_fcg(c, f, fnorm, info);
    else if (c->prm.precond == TO3D_LMG && c->prm.precision == TO3D_F64) st = solve_fcg(c, f, fnorm, info);
    else if (c->prm.precond == TO3D_LMG) st = solve_dc_mg(c, f, fnorm, info);
    else if (c->prm.precision == TO3D_F64) st = solve_f64(c, f, fnorm, info);
    else st = solve_dc(c, f, fnorm, info);
    c->have_u = true;
    return st;
}

namespace to3d {
to3d_status true_residual64(to3d_ctx* c, const double* f, double fnorm, double* relres) {
    return true_residual(c, f, fnorm, relres);
}
to3d_status sync_solver_scalars(to3d_ctx* c) { return sync_scalars(c); }
void accumulate_tc_times(to3d_ctx* c, int it0, int it1) { accumulate_kernel_times(c, 0, it0, it1); }

// FP64 Jacobi-PCG continuing from the current u (fallback of flexible CG)
to3d_status solve64_from_u(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    return solve_f64(c, f, fnorm, info);
}
}  // namespace to3d

// ------------------------------------------------------------------ C API
extern "C" {

to3d_status to3d_default_params(to3d_params* p) {
    if (!p) return TO3D_EINVAL;
    std::memset(p, 0, sizeof(*p));
    p->volfrac = 0.3;
    p->penal = 3.0;
    p->rmin = 1.5;
    p->E0 = 1.0;
    p->Emin = 1e-9;
    p->nu = 0.3;
    p->move = 0.2;
    p->bisect_tol = 1e-3;
    p->cg_rtol = 1e-8;
    p->inner_rtol = 0.3;
    p->cg_maxit = 200000;
    p->filter = TO3D_FILTER_SENS;
    p->precision = TO3D_F64;
    p->precond = TO3D_JACOBI;
    p->oc_levels = 3;
    p->warm_start = 1;
    return TO3D_OK;
}

const char* to3d_status_string(to3d_status s) { return status_name(s); }

const char* to3d_last_error(const to3d_ctx* c) { return c ? c->err.c_str() : "null context"; }

int64_t to3d_launch_count(const to3d_ctx* c) { return c ? c->launches : 0; }

to3d_status to3d_kernel_stats(to3d_ctx* c, int32_t which, double* ms_total, int64_t* samples,
                              int32_t reset) {
    if (!c || which < 0 || which > 1) return TO3D_EINVAL;
    if (ms_total) *ms_total = c->kt_ms[which];
    if (samples) *samples = c->kt_n[which];
    if (reset) {
        c->kt_ms[which] = 0.0;
        c->kt_n[which] = 0;
    }
    return TO3D_OK;
}

to3d_status to3d_create(const to3d_params* prm, const uint8_t* fixed, const double* load,
                        const uint8_t* passive, void* stream, to3d_ctx** out) {
    if (!out) return TO3D_EINVAL;
    *out = nullptr;
    if (!prm || !fixed || !load) return TO3D_EINVAL;
    if (prm->nelx < 1 || prm->nely < 1 || prm->nelz < 1) return TO3D_EINVAL;
    if ((long long)(prm->nelx + 1) * (prm->nely + 1) * (prm->nelz + 1) > (1LL << 29))
        return TO3D_EINVAL;
    if (!(prm->volfrac > 0 && prm->volfrac <= 1) || !(prm->penal >= 1) || !(prm->rmin > 0) ||
        !(prm->E0 > 0) || !(prm->Emin > 0) || !(prm->Emin < prm->E0) || !(prm->nu > -1) ||
        !(prm->nu < 0.5) || !(prm->move > 0) || !(prm->bisect_tol > 0) || !(prm->cg_rtol > 0) ||
        prm->cg_maxit < 1 || prm->oc_levels < 1 || prm->oc_levels > 5 || prm->precision < 0 ||
        prm->precision > 4 || prm->filter < 0 || prm->filter > 1 || prm->fcg_ref_iters < 0)
        return TO3D_EINVAL;
    if (prm->precond != TO3D_JACOBI && prm->precond != TO3D_CNN_FCG && prm->precond != TO3D_LMG)
        return TO3D_EINVAL;
    if (prm->mg_sweeps < 0 || prm->mg_sweeps > 1000 || prm->mg_nu < 0 || prm->mg_nu > 8)
        return TO3D_EINVAL;
    {
        // a NaN or Inf load would make every residual test false and end the
        // solves "converged": reject it here
        const long long ndof = 3LL * (prm->nelx + 1) * (prm->nely + 1) * (prm->nelz + 1);
        for (long long d = 0; d < ndof; ++d)
            if (!std::isfinite(load[d])) return TO3D_EINVAL;
    }

    to3d_ctx* c = new (std::nothrow) to3d_ctx();
    if (!c) return TO3D_ENOMEM;
    c->prm = *prm;
    c->trace = std::getenv("TO3D_TRACE") != nullptr;   // per-segment solver log on stderr
    if (!(c->prm.inner_rtol > 0 && c->prm.inner_rtol < 1)) c->prm.inner_rtol = 0.3;
    c->stream = (cudaStream_t)stream;
    Grid& g = c->g;
    g.nelx = prm->nelx; g.nely = prm->nely; g.nelz = prm->nelz;
    g.nx = g.nelx + 1; g.ny = g.nely + 1; g.nz = g.nelz + 1;
    g.nel = (long long)g.nelx * g.nely * g.nelz;
    g.nnode = (long long)g.nx * g.ny * g.nz;
    const long long N = g.nnode, ndof = 3 * N, nel = g.nel;

    c->st = new (std::nothrow) Stencil();
    auto fail = [&](to3d_status s) {
        free_all(c);
        delete c;
        return s;
    };
    if (!c->st) return fail(TO3D_ENOMEM);
    if (!build_ke(c) || !build_stencil(c)) return fail(TO3D_EINVAL);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) return fail(TO3D_ECUDA);
    init_tc_attributes();

#define AL(ptr, n)                                        \
    if (dalloc(&(ptr), (size_t)(n)) != cudaSuccess) return fail(TO3D_ENOMEM);
    c->pex = (g.nelx + 3) / 4 * 4;
    const long long nel32 = (long long)c->pex * g.nely * g.nelz;
    AL(c->x, nel); AL(c->xnew, nel); AL(c->E, nel); AL(c->E32, nel32);
    AL(c->ce, nel); AL(c->dc, nel); AL(c->dcf, nel); AL(c->Hs, nel);
    AL(c->ocq, nel); AL(c->oclo, nel); AL(c->ochi, nel); AL(c->ocs, 6 * nel); AL(c->passive, nel);
    c->px = (g.nx + 3) / 4 * 4;
    c->vol = (long long)c->px * g.ny * g.nz;
    const long long vol = c->vol;
    AL(c->nodemask, N); AL(c->dinv, N); AL(c->dinv32, vol); AL(c->maskp, vol);
    AL(c->f, ndof); AL(c->ftmp, ndof); AL(c->u, ndof); AL(c->r, ndof); AL(c->p, ndof);
    AL(c->q, ndof); AL(c->tmp, ndof);
    AL(c->d32, 3 * vol); AL(c->r32, 3 * vol); AL(c->p32a, 3 * vol); AL(c->p32b, 3 * vol);
    AL(c->q32, 3 * vol);
    c->stage_slot = (size_t)(ndof > nel ? ndof : nel) * sizeof(double);
    if ((size_t)(3 * vol) * sizeof(float) > c->stage_slot) c->stage_slot = (size_t)(3 * vol) * sizeof(float);
    c->stage_bytes = 4 * c->stage_slot;
    if (cudaMalloc(&c->stage, c->stage_bytes) != cudaSuccess) return fail(TO3D_ENOMEM);
    AL(c->red.partials, (size_t)kMaxReduceVals * kMaxBlocks);
    AL(c->red.counter, 1);
    AL(c->ss, 1); AL(c->os, 1); AL(c->misc, 8); AL(c->dev_err, 1);
#undef AL
    if (cudaMallocHost(&c->ss_h, sizeof(SolverScalars)) != cudaSuccess ||
        cudaMallocHost(&c->os_h, sizeof(OCScalars)) != cudaSuccess ||
        cudaMallocHost(&c->misc_h, 8 * sizeof(double)) != cudaSuccess)
        return fail(TO3D_ENOMEM);
    for (auto& ev : c->ev)
        if (cudaEventCreate(&ev) != cudaSuccess) return fail(TO3D_ECUDA);
    for (auto& row : c->kev)
        for (auto& ev : row)
            if (cudaEventCreate(&ev) != cudaSuccess) return fail(TO3D_ECUDA);
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return fail(TO3D_ECUDA);
    if (!prepare_tc_operands(c)) return fail(TO3D_ECUDA);

    // host-side setup of inputs (copies; masks and initial design)
    std::vector<uint8_t> nm(N, 0);
    std::vector<double> fm(ndof, 0.0);
    double f2 = 0.0;
    for (long long n = 0; n < N; ++n)
        for (int k = 0; k < 3; ++k) {
            if (fixed[3 * n + k]) nm[n] |= (uint8_t)(1u << k);
            else {
                fm[3 * n + k] = load[3 * n + k];
                f2 += load[3 * n + k] * load[3 * n + k];
            }
        }
    c->fnorm = std::sqrt(f2);
    std::vector<uint8_t> pas(nel, 0);
    std::vector<double> x0(nel, prm->volfrac);
    long long ndesign = 0;
    for (long long i = 0; i < nel; ++i) {
        pas[i] = passive ? passive[i] : 0;
        if (pas[i] > 2) return fail(TO3D_EINVAL);
        if (pas[i] == 1) x0[i] = 0.0;
        else if (pas[i] == 2) x0[i] = 1.0;
        else ndesign++;
    }
    c->ndesign = ndesign;
    std::vector<uint8_t> mp(vol, 0xff);
    for (long long n = 0; n < N; ++n) mp[(n % g.nx) + (long long)c->px * (n / g.nx)] = nm[n];
    cudaStream_t s = c->stream;
    if (cudaMemcpyAsync(c->nodemask, nm.data(), N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->f, fm.data(), ndof * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->passive, pas.data(), nel, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(c->x, x0.data(), nel * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->red.counter, 0, sizeof(unsigned), s) != cudaSuccess ||
        cudaMemsetAsync(c->dev_err, 0, sizeof(int), s) != cudaSuccess ||
        cudaMemsetAsync(c->u, 0, ndof * 8, s) != cudaSuccess ||
        cudaMemcpyAsync(c->maskp, mp.data(), vol, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(c->dinv32, 0, vol * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->E32, 0, nel32 * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->d32, 0, 3 * vol * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->r32, 0, 3 * vol * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->q32, 0, 3 * vol * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->p32a, 0, 3 * vol * 4, s) != cudaSuccess ||
        cudaMemsetAsync(c->p32b, 0, 3 * vol * 4, s) != cudaSuccess)
        return fail(TO3D_ECUDA);
    launch_hs(c, s);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(TO3D_ECUDA);
    *out = c;
    return TO3D_OK;
}

void to3d_destroy(to3d_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_all(c);
    delete c;
}

to3d_status to3d_get_density(to3d_ctx* c, double* x, int32_t on_device) {
    if (!c || !x) return TO3D_EINVAL;
    const size_t b = c->g.nel * sizeof(double);
    if (on_device) {
        CK(cudaMemcpyAsync(x, c->x, b, cudaMemcpyDeviceToDevice, c->stream));
        return TO3D_OK;
    }
    CK(cudaMemcpyAsync(x, c->x, b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TO3D_OK;
}

to3d_status to3d_set_density(to3d_ctx* c, const double* x, int32_t on_device) {
    if (!c || !x) return TO3D_EINVAL;
    const size_t b = c->g.nel * sizeof(double);
    if (on_device) {
        CK(cudaMemcpyAsync(c->x, x, b, cudaMemcpyDeviceToDevice, c->stream));
        return TO3D_OK;
    }
    // host input: staged in the OC output buffer (free between iterations)
    // and range-checked there on the GPU, so a rejected design leaves x as it was
    int* bad = reinterpret_cast<int*>(c->misc + 7);
    int bad_h = 0;
    CK(cudaMemcpyAsync(c->xnew, x, b, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    launch_check_unit(c, c->stream, c->xnew, bad);
    CK(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (bad_h) return set_err(c, TO3D_EINVAL, "densities must lie in [0, 1]");
    CK(cudaMemcpyAsync(c->x, c->xnew, b, cudaMemcpyDeviceToDevice, c->stream));
    return TO3D_OK;
}

to3d_status to3d_set_displacement(to3d_ctx* c, const double* u, int32_t on_device) {
    if (!c || !u) return TO3D_EINVAL;
    const size_t b = 3 * c->g.nnode * sizeof(double);
    CK(cudaMemcpyAsync(c->u, u, b, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    c->have_u = true;
    return TO3D_OK;
}

to3d_status to3d_get_iteration(const to3d_ctx* c, int32_t* iter) {
    if (!c || !iter) return TO3D_EINVAL;
    *iter = c->iter;
    return TO3D_OK;
}

to3d_status to3d_set_iteration(to3d_ctx* c, int32_t iter) {
    if (!c || iter < 0) return TO3D_EINVAL;
    c->iter = iter;
    return TO3D_OK;
}

to3d_status to3d_get_displacement(to3d_ctx* c, double* u, int32_t on_device) {
    if (!c || !u) return TO3D_EINVAL;
    const size_t b = 3 * c->g.nnode * sizeof(double);
    if (on_device) {
        CK(cudaMemcpyAsync(u, c->u, b, cudaMemcpyDeviceToDevice, c->stream));
        return TO3D_OK;
    }
    CK(cudaMemcpyAsync(u, c->u, b, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return TO3D_OK;
}

to3d_status to3d_matvec(to3d_ctx* c, const double* x, const double* p, double* y,
                        int32_t on_device) {
    if (!c || !x || !p || !y) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 8;
    const void *dx, *dp;
    to3d_status st;
    if ((st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_in(c, p, db, on_device, 1, &dp))) return st;
    if ((st = prepare_operator(c, (const double*)dx))) return st;
    double* dy = stage_out(c, y, on_device, 2);
    launch_matvec64(c, c->stream, c->E, (const double*)dp, dy, false);
    LK("matvec64");
    return finish_out(c, y, dy, db, on_device);
}

to3d_status to3d_matvec_lowp(to3d_ctx* c, const double* x, const float* p, float* y, int32_t prec,
                             int32_t on_device) {
    if (!c || !x || !p || !y) return TO3D_EINVAL;
    if (prec != TO3D_BF16_DC && prec != TO3D_BF16X2_DC && prec != TO3D_FP16_DC &&
        prec != TO3D_FP16X2_DC)
        return set_err(c, TO3D_EINVAL, "matvec_lowp: precision must be a tensor-core form");
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 4;
    const void *dx, *dp;
    to3d_status st;
    if ((st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_in(c, p, db, on_device, 1, &dp))) return st;
    if ((st = prepare_operator(c, (const double*)dx))) return st;
    float* dy = on_device ? y : (float*)((char*)c->stage + 2 * c->stage_slot);
    CK(cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream));
    launch_aos_to_soa(c, c->stream, (const float*)dp, c->p32a);
    launch_matvec_tc(c, c->stream, prec, false, 0);
    launch_soa_to_aos(c, c->stream, c->q32, (const float*)dp, dy);
    LK("matvec_tc");
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    st = finish_out(c, y, dy, db, on_device);
    if (st) return st;
    CK(cudaStreamSynchronize(c->stream));
    if (herr) return set_err(c, (to3d_status)herr, "tensor-core matvec wait timed out");
    return TO3D_OK;
}

to3d_status to3d_solve(to3d_ctx* c, const double* x, const double* f, double* u, int32_t on_device,
                       to3d_solve_info* info) {
    if (!c || !x || !u) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 8;
    const void *dx, *df = nullptr, *du0;
    to3d_status st;
    if ((st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = prepare_operator(c, (const double*)dx))) return st;
    const double* fuse = c->f;
    double fnorm = c->fnorm;
    if (f) {
        if ((st = stage_in(c, f, db, on_device, 1, &df))) return st;
        launch_mask_copy(c, c->stream, (const double*)df, c->ftmp);
        launch_norm2(c, c->stream, c->ftmp, 3 * c->g.nnode, c->misc + 4);
        LK("mask f");
        CK(cudaMemcpyAsync(c->misc_h, c->misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        fnorm = std::sqrt(c->misc_h[4]);
        fuse = c->ftmp;
    }
    if (c->prm.warm_start) {
        if ((st = stage_in(c, u, db, on_device, 2, &du0))) return st;
        CK(cudaMemcpyAsync(c->u, du0, db, cudaMemcpyDeviceToDevice, c->stream));
        c->have_u = true;
    }
    to3d_solve_info inf{};
    if ((st = solve_current(c, fuse, fnorm, &inf))) return st;
    if (info) *info = inf;
    if (on_device) {
        CK(cudaMemcpyAsync(u, c->u, db, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        CK(cudaMemcpyAsync(u, c->u, db, cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    return inf.status == TO3D_OK ? TO3D_OK
                                 : set_err(c, (to3d_status)inf.status, "solve did not converge");
}

to3d_status to3d_sensitivity(to3d_ctx* c, const double* x, const double* u, double* ce, double* dc,
                             double* compliance, int32_t on_device) {
    if (!c || !x || !u || !ce || !dc) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 8;
    const void *dx, *du;
    to3d_status st;
    if ((st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_in(c, u, db, on_device, 1, &du))) return st;
    double* dce = stage_out(c, ce, on_device, 2);
    double* ddc = stage_out(c, dc, on_device, 3);
    launch_sensitivity(c, c->stream, (const double*)dx, (const double*)du, dce, ddc);
    LK("sensitivity");
    CK(cudaMemcpyAsync(c->misc_h, c->misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((st = finish_out(c, ce, dce, nb, on_device))) return st;
    if ((st = finish_out(c, dc, ddc, nb, on_device))) return st;
    CK(cudaStreamSynchronize(c->stream));
    if (compliance) *compliance = c->misc_h[0];
    return TO3D_OK;
}

to3d_status to3d_filter_apply(to3d_ctx* c, int32_t kind, const double* x, const double* v,
                              double* out, int32_t transpose, int32_t on_device) {
    if (!c || !v || !out) return TO3D_EINVAL;
    if (kind == TO3D_FILTER_SENS && !x) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8;
    const void *dx = nullptr, *dv;
    to3d_status st;
    if (kind == TO3D_FILTER_SENS && (st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_in(c, v, nb, on_device, 1, &dv))) return st;
    double* dout = stage_out(c, out, on_device, 2);
    if (kind == TO3D_FILTER_SENS)
        launch_filter(c, c->stream, 0, (const double*)dx, (const double*)dv, dout);
    else
        launch_filter(c, c->stream, transpose ? 2 : 1, (const double*)dv, nullptr, dout);
    LK("filter");
    return finish_out(c, out, dout, nb, on_device);
}

to3d_status to3d_oc_update(to3d_ctx* c, const double* x, const double* dcf, double* xnew,
                           double* lambda, double* volume, int32_t* halvings, int32_t on_device) {
    if (!c || !x || !dcf || !xnew) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8;
    const void *dx, *dd;
    to3d_status st;
    if ((st = stage_in(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_in(c, dcf, nb, on_device, 1, &dd))) return st;
    double* dxn = stage_out(c, xnew, on_device, 2);
    const double target = c->prm.volfrac * (double)c->ndesign;
    launch_oc_begin(c, c->stream, (const double*)dx, (const double*)dd, target);
    int passes = 0;
    for (;;) {
        const int np = (64 + c->prm.oc_levels - 1) / c->prm.oc_levels;
        launch_oc_passes(c, c->stream, np);
        passes += np;
        LK("oc passes");
        CK(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        if (c->os_h->done || passes > 1000) break;
    }
    launch_oc_apply(c, c->stream, (const double*)dx, dxn);
    LK("oc apply");
    CK(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, c->stream));
    if ((st = finish_out(c, xnew, dxn, nb, on_device))) return st;
    CK(cudaStreamSynchronize(c->stream));
    if (lambda) *lambda = c->os_h->lmid;
    if (volume) *volume = c->os_h->volume;
    if (halvings) *halvings = c->os_h->halvings;
    if (c->os_h->status) return set_err(c, (to3d_status)c->os_h->status, "bisection did not finish");
    return TO3D_OK;
}

to3d_status to3d_step(to3d_ctx* c, to3d_iter_info* info) {
    if (!c) return TO3D_EINVAL;
    cudaStream_t s = c->stream;
    to3d_status st;
    // density filter (Section 2.4): the analysis runs on the filtered field
    // xphys = H x / Hs (passive elements pinned), and the chain rule carries
    // its sensitivities back, dc_x = H^T (dc / Hs) over the unpinned
    // elements; the OC update and its volume act on x
    const bool dens = c->prm.filter == TO3D_FILTER_DENS;
    if (dens && !c->xphys && cudaMalloc(&c->xphys, sizeof(double) * c->g.nel) != cudaSuccess)
        return set_err(c, TO3D_ENOMEM, "filtered densities");
    const double* xa = dens ? c->xphys : c->x;
    CK(cudaEventRecord(c->ev[0], s));
    if (dens) {
        launch_filter(c, s, 1, c->x, nullptr, c->xphys);
        launch_pin_passive(c, s, c->xphys);
        LK("density filter");
    }
    if ((st = prepare_operator(c, xa))) return st;
    to3d_solve_info si{};
    if ((st = solve_current(c, c->f, c->fnorm, &si))) return st;
    CK(cudaEventRecord(c->ev[1], s));
    launch_sensitivity(c, s, xa, c->u, c->ce, c->dc);
    LK("sensitivity");
    CK(cudaEventRecord(c->ev[2], s));
    if (dens) {
        launch_zero_passive(c, s, c->dc);
        launch_filter(c, s, 2, c->dc, nullptr, c->dcf);
    } else {
        launch_filter(c, s, 0, c->x, c->dc, c->dcf);
    }
    LK("filter");
    CK(cudaEventRecord(c->ev[3], s));
    const double target = c->prm.volfrac * (double)c->ndesign;
    launch_oc_begin(c, s, c->x, c->dcf, target);
    // enough passes for ~48 halvings; more are added below if the bracket is not done
    launch_oc_passes(c, s, (48 + c->prm.oc_levels - 1) / c->prm.oc_levels);
    LK("oc passes");
    CK(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    int extra = 0;
    while (!c->os_h->done && extra < 1000) {
        const int np = (32 + c->prm.oc_levels - 1) / c->prm.oc_levels;
        launch_oc_passes(c, s, np);
        extra += np;
        LK("oc passes");
        CK(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    launch_oc_apply(c, s, c->x, c->xnew);
    LK("oc apply");
    CK(cudaEventRecord(c->ev[4], s));
    CK(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(c->misc_h, c->misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double* t = c->x;
    c->x = c->xnew;
    c->xnew = t;
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->iter = c->iter;
        info->status = si.status != TO3D_OK ? si.status : c->os_h->status;
        info->compliance = c->misc_h[0];
        info->volume = c->ndesign ? c->os_h->volume / (double)c->ndesign : 0.0;
        info->change = c->os_h->change;
        info->lambda = c->os_h->lmid;
        info->relres = si.relres;
        info->cg_iters = si.iters;
        info->outer_iters = si.outer;
        info->halvings = c->os_h->halvings;
        float ms;
        cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]); info->ms_solve = ms;
        cudaEventElapsedTime(&ms, c->ev[1], c->ev[2]); info->ms_sens = ms;
        cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]); info->ms_filter = ms;
        cudaEventElapsedTime(&ms, c->ev[3], c->ev[4]); info->ms_oc = ms;
    }
    c->iter++;
    if (si.status != TO3D_OK)
        return set_err(c, (to3d_status)si.status, "solve did not reach the tolerance");
    return TO3D_OK;
}

to3d_status to3d_run(to3d_ctx* c, int32_t iters, to3d_iter_info* hist) {
    if (!c || iters < 0) return TO3D_EINVAL;
    for (int i = 0; i < iters; ++i) {
        to3d_status st = to3d_step(c, hist ? hist + i : nullptr);
        if (st) return st;
    }
    return TO3D_OK;
}

}  // extern "C"
