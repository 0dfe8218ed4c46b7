// Many independent problems: one CUDA graph per problem and OC iteration.
//
// For a batch, every OC iteration of a problem (Section 2.5) is captured
// once as a single CUDA graph whose loops are decided on the device through
// conditional WHILE nodes:
//   outer loop   defect correction: inner solve, u += d in FP64, true FP64
//                residual, then residual replacement or restart (decided by
//                k_dc_decide from the true residual);
//   inner loop   chunks of fused tensor-core matvec + update iterations
//                until the inner residual target is met;
//   OC loop      bisection passes until the bracket is resolved.
// A step of the batch launches all problems' graphs on a pool of streams,
// so the small problems' kernels run side by side, and waits once.  No host
// round trip happens inside an OC iteration.  Every loop body always sets
// its loop condition and every loop has an iteration cap, so a graph cannot
// spin forever.
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "internal.cuh"
#include "reduce.cuh"

namespace to3d {

struct DcCtl {
    double tol, fnorm, delta2, target2, scale, relres0, relres, prev;
    int mode;            // next inner start: 1 = (re)start from the true residual, 0 = replacement
    int outer, stalls, total, maxit, status, done, guard;
};

constexpr int kInnerChunk = 8;            // fused iterations per inner-loop body (even)
constexpr int kGuardChunks = 1 << 20;     // cap on inner-loop bodies per OC iteration

// First true residual: solve at all?  Fixes the inner scaling for the solve.
__global__ void k_dc_start(DcCtl* ctl, SolverScalars* ss, long long ndof,
                           cudaGraphConditionalHandle outer) {
    const double relres = ctl->fnorm > 0.0 ? sqrt(ss->rr_true) / ctl->fnorm : 0.0;
    ctl->relres = ctl->relres0 = ctl->prev = relres;
    ctl->outer = ctl->stalls = ctl->total = ctl->status = ctl->guard = 0;
    ctl->mode = 1;
    ctl->done = (relres <= ctl->tol || ctl->fnorm == 0.0) ? 1 : 0;
    if (!ctl->done) {
        ctl->scale = 1.0 / sqrt(ss->rr_true / (double)ndof);
        const double t = 0.5 * ctl->tol * ctl->fnorm * ctl->scale;
        ctl->target2 = t * t;
        ss->maxit = ctl->maxit;
        ss->status = 0;
    }
    cudaGraphSetConditional(outer, ctl->done ? 0u : 1u);
}

// Start or continue the inner CG from the true residual r64 (see
// k_pcg32_replace for the replacement rule); sets the inner loop condition.
__global__ void k_dc_prepare(const Grid g, int px, long long vol, const double* __restrict__ r64,
                             const float* __restrict__ dinv, float* __restrict__ p32a,
                             float* __restrict__ p32b, float* __restrict__ r32,
                             float* __restrict__ d32, const Reducer red, SolverScalars* ss,
                             DcCtl* ctl, cudaGraphConditionalHandle inner) {
    __shared__ double sh[96];
    __shared__ double out[3];
    const int mode = ctl->mode;
    const double scale = ctl->scale;
    const bool odd = (ss->it & 1) != 0;       // last direction sits in p32a
    double rzd = 0.0, rrd = 0.0, rpd = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
        const float di = dinv[pp];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = c * vol + pp;
            const float rv = (float)(r64[3 * n + c] * scale);
            r32[d] = rv;
            d32[d] = 0.f;
            float pl = 0.f;
            if (mode) {
                p32b[d] = 0.f;
            } else {
                pl = odd ? p32a[d] : p32b[d];
                if (odd) p32b[d] = pl;
            }
            rzd += (double)(di * rv * rv);
            rrd += (double)(rv * rv);
            rpd += (double)(rv * pl);
        }
    }
    double v[3] = {rzd, rrd, rpd};
    if (grid_sum<3>(red, v, sh, out) && threadIdx.x == 0) {
        const double rz = out[0], rr = out[1], rp = out[2];
        if (mode) {
            const double q = ctl->relres / ctl->relres0;
            ss->beta = 0.0;
            ss->zcoef = 1.0;
            ss->tol2 = fmax(ctl->delta2 * (double)(3 * g.nnode) * q * q, ctl->target2);
        } else {
            const double beta = rz / ss->rz;
            ss->beta = beta;
            ss->zcoef = 1.0 - beta * (rz > 0.0 ? rp / rz : 0.0);
            ss->tol2 = fmax(ctl->delta2 * rr, ctl->target2);
        }
        ss->rz = rz;
        ss->rr = rr;
        ss->it = 0;
        ss->done = 0;
        if (!isfinite(rz) || !isfinite(rr) || !isfinite(rp)) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (rr <= ss->tol2) {
            ss->done = 1;
        }
        cudaGraphSetConditional(inner, ss->done ? 0u : 1u);
    }
}

// Learned-multigrid form: every segment restarts the inner CG from the true
// residual (r32 = scale r64, d = 0, p_old = 0, q = 0, first-step flag),
// stopping it once |r32| has dropped by inner_rtol or the target is met.
__global__ void k_dc_prepare_mg(const Grid g, int px, long long vol, const double* __restrict__ r64,
                                const uint8_t* __restrict__ nodemask, float* __restrict__ p32b,
                                float* __restrict__ r32, float* __restrict__ d32,
                                float* __restrict__ q32, const Reducer red, SolverScalars* ss,
                                DcCtl* ctl, cudaGraphConditionalHandle inner) {
    __shared__ double sh[32];
    __shared__ double out[1];
    const double scale = ctl->scale;
    double rrd = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
        const uint8_t m = nodemask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = c * vol + pp;
            const float rv = ((m >> c) & 1) ? 0.f : (float)(r64[3 * n + c] * scale);
            r32[d] = rv;
            d32[d] = 0.f;
            p32b[d] = 0.f;
            q32[d] = 0.f;
            rrd += (double)(rv * rv);
        }
    }
    double v[1] = {rrd};
    if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) {
        const double rr = out[0];
        ss->beta = 0.0;
        ss->zcoef = 1.0;
        ss->pad0 = 1;
        ss->tol2 = fmax(ctl->delta2 * rr, ctl->target2);
        ss->rr = rr;
        ss->it = 0;
        ss->done = 0;
        if (!isfinite(rr)) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (rr <= ss->tol2) {
            ss->done = 1;
        }
        cudaGraphSetConditional(inner, ss->done ? 0u : 1u);
    }
}

__global__ void k_inner_cond(const SolverScalars* ss, DcCtl* ctl, cudaGraphConditionalHandle inner) {
    const bool more = !ss->done && ++ctl->guard < kGuardChunks;
    cudaGraphSetConditional(inner, more ? 1u : 0u);
}

// u += d / scale with the scale held on the device
__global__ void k_axpy_ctl(const Grid g, int px, long long vol, double* __restrict__ u,
                           const float* __restrict__ d32, const DcCtl* ctl) {
    const double inv = 1.0 / ctl->scale;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) u[3 * n + c] = fma((double)d32[c * vol + pp], inv, u[3 * n + c]);
    }
}

// After a segment: converged, replace, restart or give up.
__global__ void k_dc_decide(DcCtl* ctl, SolverScalars* ss, cudaGraphConditionalHandle outer) {
    ctl->total += ss->it;
    const double relres = ctl->fnorm > 0.0 ? sqrt(ss->rr_true) / ctl->fnorm : 0.0;
    unsigned more = 0u;
    if (ss->status == TO3D_ETIMEOUT || ss->status == TO3D_ENUMERIC) {
        ctl->status = ss->status;
    } else if (relres <= ctl->tol) {
        ctl->status = TO3D_OK;
    } else if (ctl->total >= ctl->maxit || ctl->outer >= 1000) {
        ctl->status = TO3D_ENOCONV;
    } else {
        ctl->outer += 1;
        if (relres > 0.5 * ctl->prev) {
            ctl->mode = 1;
            if (++ctl->stalls > 50) ctl->status = TO3D_ENOCONV;
            else more = 1u;
        } else {
            ctl->mode = 0;
            more = 1u;
        }
        ss->maxit = ctl->maxit - ctl->total;
        ss->status = 0;
    }
    ctl->prev = relres;
    ctl->relres = relres;
    ctl->done = more ? 0 : 1;
    cudaGraphSetConditional(outer, more);
}

// ------------------------------------------------------------------ capture helpers
static cudaError_t new_handle(cudaStream_t s, cudaGraphConditionalHandle* h, unsigned dflt) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    return cudaGraphConditionalHandleCreate(h, g, dflt, cudaGraphCondAssignDefault);
}

// Append a WHILE node on handle h to the capture on s; its body is captured on `body`.
static cudaError_t begin_while(cudaStream_t s, cudaStream_t body, cudaGraphConditionalHandle h) {
    cudaStreamCaptureStatus st;
    cudaGraph_t g;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
    if (e != cudaSuccess) return e;
    cudaGraphNodeParams p = {cudaGraphNodeTypeConditional};
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if ((e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p)) != cudaSuccess) return e;
    if ((e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1,
                                                 cudaStreamSetCaptureDependencies)) != cudaSuccess)
        return e;
    return cudaStreamBeginCaptureToGraph(body, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
}

static cudaError_t end_while(cudaStream_t body) {
    cudaGraph_t g;
    return cudaStreamEndCapture(body, &g);
}

#define CE(call)                                          \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return _e;                 \
    } while (0)

// Capture one whole OC iteration of context c (defect-correction forms).
static cudaError_t build_iter_graph(to3d_ctx* c) {
    const Grid& g = c->g;
    const long long ndof = 3 * g.nnode;
    cudaStream_t s0 = c->cap_stream, s1 = c->cap_stream2, s2 = c->cap_stream3;
    DcCtl* ctl = (DcCtl*)c->dcctl;
    const int prec = c->prm.precision;
    const double target = c->prm.volfrac * (double)c->ndesign;
    // density filter: analysis on xphys = H x / Hs (passive pinned), chain
    // rule back to x over the unpinned elements; the OC update acts on x (as
    // the single-context step)
    const bool dens = c->prm.filter == TO3D_FILTER_DENS;
    const double* xa = dens ? c->xphys : c->x;
    cudaGraph_t graph;
    CE(cudaStreamBeginCapture(s0, cudaStreamCaptureModeThreadLocal));
    if (dens) {
        launch_filter(c, s0, 1, c->x, nullptr, c->xphys);
        launch_pin_passive(c, s0, c->xphys);
    }
    const bool lmg = c->prm.precond == TO3D_LMG;
    launch_simp(c, s0, xa);
    launch_diag(c, s0, c->E);
    if (lmg) mg_setup_launch(c, s0);
    launch_matvec64(c, s0, c->E, c->u, c->q, false);
    launch_residual64(c, s0, c->f, c->q, c->r, true);
    cudaGraphConditionalHandle h_outer, h_inner, h_oc;
    CE(new_handle(s0, &h_outer, 0));
    k_dc_start<<<1, 1, 0, s0>>>(ctl, c->ss, ndof, h_outer);
    CE(begin_while(s0, s1, h_outer));
    {
        CE(new_handle(s1, &h_inner, 0));
        if (lmg)
            k_dc_prepare_mg<<<152 * 4, 256, 0, s1>>>(g, c->px, c->vol, c->r, c->nodemask, c->p32b,
                                                     c->r32, c->d32, c->q32, c->red, c->ss, ctl,
                                                     h_inner);
        else
            k_dc_prepare<<<152 * 4, 256, 0, s1>>>(g, c->px, c->vol, c->r, c->dinv32, c->p32a,
                                                  c->p32b, c->r32, c->d32, c->red, c->ss, ctl,
                                                  h_inner);
        CE(begin_while(s1, s2, h_inner));
        for (int i = 0; i < kInnerChunk; ++i) {
            if (lmg) mg_pcg_iter_launch(c, s2, prec, i & 1);
            else launch_pcg32_iter(c, s2, prec, i & 1);
        }
        k_inner_cond<<<1, 1, 0, s2>>>(c->ss, ctl, h_inner);
        CE(end_while(s2));
        k_axpy_ctl<<<152 * 4, 256, 0, s1>>>(g, c->px, c->vol, c->u, c->d32, ctl);
        launch_matvec64(c, s1, c->E, c->u, c->q, false);
        launch_residual64(c, s1, c->f, c->q, c->r, true);
        k_dc_decide<<<1, 1, 0, s1>>>(ctl, c->ss, h_outer);
    }
    CE(end_while(s1));
    launch_sensitivity(c, s0, xa, c->u, c->ce, c->dc);
    if (dens) {
        launch_zero_passive(c, s0, c->dc);
        launch_filter(c, s0, 2, c->dc, nullptr, c->dcf);
    } else {
        launch_filter(c, s0, 0, c->x, c->dc, c->dcf);
    }
    launch_oc_begin(c, s0, c->x, c->dcf, target);
    CE(new_handle(s0, &h_oc, 1));
    CE(begin_while(s0, s1, h_oc));
    launch_oc_passes(c, s1, 1, h_oc, 1);
    CE(end_while(s1));
    launch_oc_apply(c, s0, c->x, c->xnew);
    CE(cudaMemcpyAsync(c->x, c->xnew, sizeof(double) * g.nel, cudaMemcpyDeviceToDevice, s0));
    CE(cudaMemcpyAsync(c->os_h, c->os, sizeof(OCScalars), cudaMemcpyDeviceToHost, s0));
    CE(cudaMemcpyAsync(c->misc_h, c->misc, 8 * sizeof(double), cudaMemcpyDeviceToHost, s0));
    CE(cudaMemcpyAsync(c->dcctl_h, c->dcctl, sizeof(DcCtl), cudaMemcpyDeviceToHost, s0));
    CE(cudaStreamEndCapture(s0, &graph));
    cudaError_t e = cudaGraphInstantiate(&c->g_iter, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

}  // namespace to3d

using namespace to3d;

struct to3d_batch {
    std::vector<to3d_ctx*> ctx;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> done;
    cudaEvent_t start = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
};

static void batch_free(to3d_batch* b) {
    if (!b) return;
    for (to3d_ctx* c : b->ctx)
        if (c) to3d_destroy(c);
    for (cudaStream_t s : b->pool)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->done)
        if (e) cudaEventDestroy(e);
    if (b->start) cudaEventDestroy(b->start);
    delete b;
}

extern "C" {

to3d_status to3d_batch_create(int32_t nprob, const to3d_params* params, const uint8_t* const* fixed,
                              const double* const* load, const uint8_t* const* passive,
                              void* stream, to3d_batch** out) {
    if (!out) return TO3D_EINVAL;
    *out = nullptr;
    if (nprob < 1 || !params || !fixed || !load) return TO3D_EINVAL;
    for (int i = 0; i < nprob; ++i) {
        if (params[i].precision == TO3D_F64) return TO3D_EINVAL;   // tensor-core forms only
    }
    to3d_batch* b = new (std::nothrow) to3d_batch();
    if (!b) return TO3D_ENOMEM;
    b->stream = (cudaStream_t)stream;
    const int npool = nprob < 16 ? nprob : 16;
    b->pool.resize(npool, nullptr);
    b->done.resize(npool, nullptr);
    for (int i = 0; i < npool; ++i)
        if (cudaStreamCreateWithFlags(&b->pool[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->done[i], cudaEventDisableTiming) != cudaSuccess) {
            batch_free(b);
            return TO3D_ECUDA;
        }
    if (cudaEventCreateWithFlags(&b->start, cudaEventDisableTiming) != cudaSuccess) {
        batch_free(b);
        return TO3D_ECUDA;
    }
    b->ctx.resize(nprob, nullptr);
    for (int i = 0; i < nprob; ++i) {
        to3d_status st = to3d_create(&params[i], fixed[i], load[i], passive ? passive[i] : nullptr,
                                     b->pool[i % npool], &b->ctx[i]);
        if (st != TO3D_OK) {
            batch_free(b);
            return st;
        }
        to3d_ctx* c = b->ctx[i];
        DcCtl h;
        std::memset(&h, 0, sizeof(h));
        h.tol = c->prm.cg_rtol;
        h.fnorm = c->fnorm;
        h.delta2 = c->prm.inner_rtol * c->prm.inner_rtol;
        h.maxit = c->prm.cg_maxit;
        if (cudaStreamCreateWithFlags(&c->cap_stream2, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&c->cap_stream3, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMalloc(&c->dcctl, sizeof(DcCtl)) != cudaSuccess ||
            cudaMallocHost(&c->dcctl_h, sizeof(DcCtl)) != cudaSuccess ||
            cudaMemcpy(c->dcctl, &h, sizeof(DcCtl), cudaMemcpyHostToDevice) != cudaSuccess ||
            (c->prm.filter == TO3D_FILTER_DENS &&
             cudaMalloc(&c->xphys, sizeof(double) * c->g.nel) != cudaSuccess) ||
            tune_tc_lz(c, c->prm.precision, c->tm_pa, c->q32, true) != cudaSuccess ||
            (c->prm.precond == TO3D_LMG && mg_capture_ready(c) != TO3D_OK) ||
            build_iter_graph(c) != cudaSuccess) {
            batch_free(b);
            return TO3D_ECUDA;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        batch_free(b);
        return TO3D_ECUDA;
    }
    *out = b;
    return TO3D_OK;
}

to3d_status to3d_batch_set_mg_params(to3d_batch* b, const double* theta, int64_t n) {
    if (!b || !theta) return TO3D_EINVAL;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TO3D_ECUDA;
    for (to3d_ctx* c : b->ctx) {
        if (c->prm.precond != TO3D_LMG) return TO3D_ESTATE;
        to3d_status st = to3d_mg_set_params(c, theta, n);
        if (st != TO3D_OK) return st;
        // the parameters are kernel arguments of the captured set-up: capture again
        if (c->g_iter) cudaGraphExecDestroy(c->g_iter);
        c->g_iter = nullptr;
        if (build_iter_graph(c) != cudaSuccess) return TO3D_ECUDA;
    }
    return TO3D_OK;
}

to3d_status to3d_batch_step(to3d_batch* b, to3d_iter_info* info) {
    if (!b) return TO3D_EINVAL;
    const int npool = (int)b->pool.size();
    if (cudaEventRecord(b->start, b->stream) != cudaSuccess) return TO3D_ECUDA;
    for (int i = 0; i < npool; ++i)
        if (cudaStreamWaitEvent(b->pool[i], b->start, 0) != cudaSuccess) return TO3D_ECUDA;
    for (size_t i = 0; i < b->ctx.size(); ++i)
        if (cudaGraphLaunch(b->ctx[i]->g_iter, b->pool[i % npool]) != cudaSuccess) return TO3D_ECUDA;
    for (int i = 0; i < npool; ++i) {
        if (cudaEventRecord(b->done[i], b->pool[i]) != cudaSuccess) return TO3D_ECUDA;
        if (cudaStreamWaitEvent(b->stream, b->done[i], 0) != cudaSuccess) return TO3D_ECUDA;
    }
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return TO3D_ECUDA;
    to3d_status worst = TO3D_OK;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        to3d_ctx* c = b->ctx[i];
        const DcCtl* h = (const DcCtl*)c->dcctl_h;
        const int status = h->status != TO3D_OK ? h->status : c->os_h->status;
        if (status != TO3D_OK) worst = (to3d_status)status;
        if (info) {
            to3d_iter_info& r = info[i];
            std::memset(&r, 0, sizeof(r));
            r.iter = c->iter;
            r.status = status;
            r.compliance = c->misc_h[0];
            r.volume = c->ndesign ? c->os_h->volume / (double)c->ndesign : 0.0;
            r.change = c->os_h->change;
            r.lambda = c->os_h->lmid;
            r.relres = h->relres;
            r.cg_iters = h->total;
            r.outer_iters = h->outer + 1;
            r.halvings = c->os_h->halvings;
        }
        c->iter++;
    }
    return worst;
}

to3d_status to3d_batch_get_density(to3d_batch* b, int32_t i, double* x, int32_t on_device) {
    if (!b || i < 0 || i >= (int)b->ctx.size()) return TO3D_EINVAL;
    return to3d_get_density(b->ctx[i], x, on_device);
}

int32_t to3d_batch_size(const to3d_batch* b) { return b ? (int32_t)b->ctx.size() : 0; }

void to3d_batch_destroy(to3d_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    cudaDeviceSynchronize();
    batch_free(b);
}

}  // extern "C"
