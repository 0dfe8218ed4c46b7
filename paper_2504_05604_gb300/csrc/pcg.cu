// Jacobi-preconditioned conjugate gradients on the device.
//
// The paper solves K U = F directly (Section 2.2).  Here the solve is the
// textbook PCG with M = diag(K); all scalars (rz, pq, alpha, beta, the
// convergence flag) live in device memory and are produced by the last
// block of each reduction, so a run of iterations needs no host round trip
// and can be captured once as a CUDA graph.  Kernels return at once when the
// device flag says the solve is finished.
//
// FP64 form: matvec64 (q = K p, p.q, alpha) -> update (u, r, rz, |r|^2,
// beta, flag) -> direction (p = M^-1 r + beta p).
// Inner FP32 form of the defect-correction solve: the tensor-core matvec
// fuses the direction update (p_new = M^-1 r + beta p_old, ping-pong
// buffers) with q = K p_new and p_new.q; the update kernel then does
// d += alpha p_new, r -= alpha q and the two dot products.  Vectors are FP32;
// per-thread partial sums of positive terms are FP32, block and grid sums
// FP64.
#include "internal.cuh"
#include "reduce.cuh"

namespace to3d {

constexpr int PCG_THREADS = 256;

__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }
__device__ __forceinline__ long long gtid() {
    return blockIdx.x * (long long)blockDim.x + threadIdx.x;
}

__global__ void k_ss_segment(SolverScalars* ss, double tol2, int maxit) {
    ss->tol2 = tol2;
    ss->it = 0;
    ss->done = 0;
    ss->maxit = maxit;
}

__global__ void k_ss_reset(SolverScalars* ss, double tol2, int maxit) {
    ss->rz = ss->rz_new = ss->pq = ss->rr = ss->alpha = ss->beta = 0.0;
    ss->zcoef = 1.0;
    ss->tol2 = tol2;
    ss->it = 0;
    ss->done = 0;
    ss->status = 0;
    ss->maxit = maxit;
}

// ---------------------------------------------------------------- FP64 form
// z = M^-1 r, p = z, rz = r.z, rr = r.r
__global__ void k_pcg64_init(long long nnode, const double* __restrict__ r,
                             const double* __restrict__ dinv, double* __restrict__ p,
                             const Reducer red, SolverScalars* ss) {
    __shared__ double sh[64];
    __shared__ double out[2];
    double rz = 0.0, rr = 0.0;
    for (long long n = gtid(); n < nnode; n += gstride()) {
        const double di = dinv[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double rv = r[3 * n + c];
            p[3 * n + c] = di * rv;
            rz += di * rv * rv;
            rr += rv * rv;
        }
    }
    double v[2] = {rz, rr};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) {
        ss->rz = out[0];
        ss->rr = out[1];
        if (!isfinite(out[0]) || !isfinite(out[1])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[1] <= ss->tol2) {
            ss->done = 1;
        }
    }
}

// u += alpha p, r -= alpha q, rz_new = r.M^-1 r, rr = r.r, beta, flags
__global__ void k_pcg64_update(long long nnode, double* __restrict__ u, double* __restrict__ r,
                               const double* __restrict__ p, const double* __restrict__ q,
                               const double* __restrict__ dinv, const Reducer red,
                               SolverScalars* ss) {
    if (ss->done) return;
    __shared__ double sh[64];
    __shared__ double out[2];
    const double alpha = ss->alpha;
    double rz = 0.0, rr = 0.0;
    for (long long n = gtid(); n < nnode; n += gstride()) {
        const double di = dinv[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = 3 * n + c;
            u[d] = fma(alpha, p[d], u[d]);
            const double rv = fma(-alpha, q[d], r[d]);
            r[d] = rv;
            rz += di * rv * rv;
            rr += rv * rv;
        }
    }
    double v[2] = {rz, rr};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) {
        const double rzn = out[0];
        ss->beta = rzn / ss->rz;
        ss->rz = rzn;
        ss->rr = out[1];
        ss->it += 1;
        if (!isfinite(rzn) || !isfinite(out[1])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[1] <= ss->tol2) {
            ss->done = 1;
        } else if (ss->it >= ss->maxit) {
            ss->status = TO3D_ENOCONV;
            ss->done = 1;
        }
    }
}

// p = M^-1 r + beta p
__global__ void k_pcg64_dir(long long nnode, const double* __restrict__ r,
                            const double* __restrict__ dinv, double* __restrict__ p,
                            const SolverScalars* ss) {
    if (ss->done) return;
    const double beta = ss->beta;
    for (long long n = gtid(); n < nnode; n += gstride()) {
        const double di = dinv[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long d = 3 * n + c;
            p[d] = fma(di, r[d], beta * p[d]);
        }
    }
}

// ---------------------------------------------------------------- FP32 inner form
// Vectors on the padded structure-of-arrays node grid (component c of padded
// node p at c*vol + p; pad nodes stay zero).
// r32 = r64 * scale (the host picks scale = 1/RMS(r64)), d = 0, p_old = 0;
// the first fused matvec then builds p = M^-1 r.  rz and rr of the scaled r.
__global__ void k_pcg32_init(const Grid g, int px, long long vol, const double* __restrict__ r64,
                             double scale, const float* __restrict__ dinv, float* __restrict__ r32,
                             float* __restrict__ d32, float* __restrict__ p_old,
                             const Reducer red, SolverScalars* ss) {
    __shared__ double sh[64];
    __shared__ double out[2];
    float rz = 0.f, rr = 0.f;
    double rzd = 0.0, rrd = 0.0;
    int cnt = 0;
    for (long long n = gtid(); n < g.nnode; n += gstride()) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
        const float di = dinv[pp];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float rv = (float)(r64[3 * n + c] * scale);
            r32[c * vol + pp] = rv;
            d32[c * vol + pp] = 0.f;
            p_old[c * vol + pp] = 0.f;
            rz = fmaf(di * rv, rv, rz);
            rr = fmaf(rv, rv, rr);
        }
        if (++cnt == 16) { rzd += rz; rrd += rr; rz = rr = 0.f; cnt = 0; }
    }
    rzd += rz;
    rrd += rr;
    double v[2] = {rzd, rrd};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) {
        ss->rz = out[0];
        ss->rr = out[1];
        ss->beta = 0.0;
        ss->zcoef = 1.0;
        if (!isfinite(out[0]) || !isfinite(out[1])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[1] <= ss->tol2) {
            ss->done = 1;
        }
    }
}

// d += alpha p, r -= alpha q (clamped dofs and pads kept at 0), rz_new, rr,
// beta, flags.  Four consecutive nodes per step (vol is a multiple of 4), so
// every thread keeps 14 independent 16-byte loads in flight.  Without the
// Jacobi beta (JB = 0: the caller forms beta) M^-1 is neither read nor used.
template <int JB>
__global__ void __launch_bounds__(256)
    k_pcg32_update(long long vol, float* __restrict__ d32, float* __restrict__ r32,
                   const float* __restrict__ p, const float* __restrict__ q,
                   const float* __restrict__ dinv, const uint8_t* __restrict__ maskp,
                   const Reducer red, SolverScalars* ss) {
    constexpr int jacobi_beta = JB;
    if (ss->done) return;
    __shared__ double sh[64];
    __shared__ double out[2];
    const float alpha = (float)ss->alpha;
    const long long v4 = vol >> 2;
    float4* d4 = reinterpret_cast<float4*>(d32);
    float4* r4 = reinterpret_cast<float4*>(r32);
    const float4* p4 = reinterpret_cast<const float4*>(p);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    const float4* di4 = reinterpret_cast<const float4*>(dinv);
    const uchar4* m4 = reinterpret_cast<const uchar4*>(maskp);
    double rzd = 0.0, rrd = 0.0;
    for (long long n = gtid(); n < v4; n += gstride()) {
        const float4 di = JB ? __ldg(di4 + n) : make_float4(0.f, 0.f, 0.f, 0.f);
        const uchar4 mk = __ldg(m4 + n);
        float4 dd[3], pp[3], qq[3], rr[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dd[c] = d4[c * v4 + n];
            pp[c] = __ldg(p4 + c * v4 + n);
            qq[c] = __ldg(q4 + c * v4 + n);
            rr[c] = r4[c * v4 + n];
        }
        float rz = 0.f, rs = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dd[c].x = fmaf(alpha, pp[c].x, dd[c].x);
            dd[c].y = fmaf(alpha, pp[c].y, dd[c].y);
            dd[c].z = fmaf(alpha, pp[c].z, dd[c].z);
            dd[c].w = fmaf(alpha, pp[c].w, dd[c].w);
            float4 rv;
            rv.x = ((mk.x >> c) & 1) ? 0.f : fmaf(-alpha, qq[c].x, rr[c].x);
            rv.y = ((mk.y >> c) & 1) ? 0.f : fmaf(-alpha, qq[c].y, rr[c].y);
            rv.z = ((mk.z >> c) & 1) ? 0.f : fmaf(-alpha, qq[c].z, rr[c].z);
            rv.w = ((mk.w >> c) & 1) ? 0.f : fmaf(-alpha, qq[c].w, rr[c].w);
            d4[c * v4 + n] = dd[c];
            r4[c * v4 + n] = rv;
            if (JB) {
                rz = fmaf(di.x * rv.x, rv.x, rz);
                rz = fmaf(di.y * rv.y, rv.y, rz);
                rz = fmaf(di.z * rv.z, rv.z, rz);
                rz = fmaf(di.w * rv.w, rv.w, rz);
            }
            rs = fmaf(rv.x, rv.x, fmaf(rv.y, rv.y, fmaf(rv.z, rv.z, fmaf(rv.w, rv.w, rs))));
        }
        if (JB) rzd += rz;
        rrd += rs;
    }
    double v[2] = {rzd, rrd};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) {
        const double rzn = out[0];
        if (jacobi_beta) {
            ss->beta = rzn / ss->rz;
            ss->zcoef = 1.0;
            ss->rz = rzn;
        }
        ss->rr = out[1];
        ss->it += 1;
        if ((jacobi_beta && !isfinite(rzn)) || !isfinite(out[1])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[1] <= ss->tol2) {
            ss->done = 1;
        } else if (ss->it >= ss->maxit) {
            ss->status = TO3D_ENOCONV;
            ss->done = 1;
        }
    }
}

// out[0] = a.b, out[1] = cc.d (cc may be null)
__global__ void k_dots64(long long n, const double* __restrict__ a, const double* __restrict__ b,
                         const double* __restrict__ cc, const double* __restrict__ d,
                         const Reducer red, double* out_dev) {
    __shared__ double sh[64];
    __shared__ double o2[2];
    double s0 = 0.0, s1 = 0.0;
    for (long long i = gtid(); i < n; i += gstride()) {
        s0 = fma(a[i], b[i], s0);
        if (cc) s1 = fma(cc[i], d[i], s1);
    }
    double v[2] = {s0, s1};
    if (grid_sum<2>(red, v, sh, o2) && threadIdx.x == 0) {
        out_dev[0] = o2[0];
        out_dev[1] = o2[1];
    }
}

// Residual replacement ("reliable update") of the inner solve: the FP32
// recurrence residual is replaced by the true FP64 residual r' (scaled),
// the correction d restarts at 0 (u has absorbed it), and the last search
// direction p is kept.  To keep r'^T p = 0 the next direction is built from
// p - gamma z' with z' = M^-1 r' and gamma = r'^T p / r'^T z', i.e.
//   p_new = (1 - beta gamma) z' + beta p,   beta = r'^T z' / rz_old,
// which the fused matvec forms through the coefficient zcoef.
__global__ void k_pcg32_replace(const Grid g, int px, long long vol, const double* __restrict__ r64,
                                double scale, const float* __restrict__ dinv,
                                const float* __restrict__ p, float* __restrict__ r32,
                                float* __restrict__ d32, const Reducer red, SolverScalars* ss,
                                double delta2, double target2) {
    __shared__ double sh[96];
    __shared__ double out[3];
    double rzd = 0.0, rrd = 0.0, rpd = 0.0;
    for (long long n = gtid(); n < g.nnode; n += gstride()) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
        const float di = dinv[pp];
        float rz = 0.f, rr = 0.f, rp = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float rv = (float)(r64[3 * n + c] * scale);
            r32[c * vol + pp] = rv;
            d32[c * vol + pp] = 0.f;
            rz = fmaf(di * rv, rv, rz);
            rr = fmaf(rv, rv, rr);
            rp = fmaf(rv, p[c * vol + pp], rp);
        }
        rzd += rz;
        rrd += rr;
        rpd += rp;
    }
    double v[3] = {rzd, rrd, rpd};
    if (grid_sum<3>(red, v, sh, out) && threadIdx.x == 0) {
        const double rz = out[0], rr = out[1], rp = out[2];
        const double beta = rz / ss->rz;
        const double gamma = rz > 0.0 ? rp / rz : 0.0;
        ss->beta = beta;
        ss->zcoef = 1.0 - beta * gamma;
        ss->rz = rz;
        ss->rr = rr;
        ss->done = 0;
        ss->tol2 = fmax(delta2 * rr, target2);     // next replacement after a drop by delta
        if (!isfinite(rz) || !isfinite(rr) || !isfinite(rp)) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (rr <= ss->tol2) {
            ss->done = 1;
        }
    }
}

// u64 += d32 / scale (FP64 accumulation of the correction)
__global__ void k_axpy_d32(const Grid g, int px, long long vol, double* __restrict__ u,
                           const float* __restrict__ d32, double inv_scale) {
    for (long long n = gtid(); n < g.nnode; n += gstride()) {
        const long long pp = (n % g.nx) + (long long)px * (n / g.nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) u[3 * n + c] = fma((double)d32[c * vol + pp], inv_scale, u[3 * n + c]);
    }
}

__global__ void k_norm2(long long n, const double* __restrict__ v, const Reducer red,
                        double* out_dev) {
    __shared__ double sh[32];
    __shared__ double out[1];
    double acc = 0.0;
    for (long long i = gtid(); i < n; i += gstride()) acc += v[i] * v[i];
    double a[1] = {acc};
    if (grid_sum<1>(red, a, sh, out) && threadIdx.x == 0) *out_dev = out[0];
}

static unsigned vec_blocks(long long n) {
    long long nb = (n + PCG_THREADS - 1) / PCG_THREADS;
    if (nb > 152 * 8) nb = 152 * 8;
    if (nb < 1) nb = 1;
    return (unsigned)nb;
}

void launch_pcg64_init(to3d_ctx* c, cudaStream_t s) {
    k_pcg64_init<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(c->g.nnode, c->r, c->dinv, c->p,
                                                                 c->red, c->ss);
    c->launches++;
}

void launch_pcg64_iter(to3d_ctx* c, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
    if (ev0) cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal);
    launch_matvec64(c, s, c->E, c->p, c->q, true);
    if (ev1) cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal);
    k_pcg64_update<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(c->g.nnode, c->u, c->r, c->p,
                                                                   c->q, c->dinv, c->red, c->ss);
    k_pcg64_dir<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(c->g.nnode, c->r, c->dinv, c->p,
                                                                c->ss);
    c->launches += 2;
}

void launch_pcg32_init(to3d_ctx* c, cudaStream_t s, const double* r64, double scale) {
    k_pcg32_init<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(
        c->g, c->px, c->vol, r64, scale, c->dinv32, c->r32, c->d32, c->p32b, c->red, c->ss);
    c->launches++;
}

// parity 0: p_old = p32b -> p_new = p32a; parity 1: the reverse.
// ev0/ev1 (may be null): external events recorded around the matvec launch.
void launch_pcg32_iter(to3d_ctx* c, cudaStream_t s, int prec, int parity, cudaEvent_t ev0,
                       cudaEvent_t ev1) {
    float* p_new = parity ? c->p32b : c->p32a;
    if (ev0) cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal);
    launch_matvec_tc(c, s, prec, true, parity);
    if (ev1) cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal);
    launch_pcg32_update_mode(c, s, p_new, 1);
}

// d += alpha p_new, r -= alpha q, |r|^2; with jacobi_beta also r.M^-1 r and
// beta = rz_new / rz (Jacobi PCG); without, the caller forms beta itself.
void launch_pcg32_update_mode(to3d_ctx* c, cudaStream_t s, const float* p_new, int jacobi_beta) {
    if (jacobi_beta)
        k_pcg32_update<1><<<vec_blocks(c->vol / 4), PCG_THREADS, 0, s>>>(
            c->vol, c->d32, c->r32, p_new, c->q32, c->dinv32, c->maskp, c->red, c->ss);
    else
        k_pcg32_update<0><<<vec_blocks(c->vol / 4), PCG_THREADS, 0, s>>>(
            c->vol, c->d32, c->r32, p_new, c->q32, c->dinv32, c->maskp, c->red, c->ss);
    c->launches++;
}

void launch_dots64(to3d_ctx* c, cudaStream_t s, long long n, const double* a, const double* b,
                   const double* cc, const double* d, double* out_dev) {
    k_dots64<<<vec_blocks(n), PCG_THREADS, 0, s>>>(n, a, b, cc, d, c->red, out_dev);
    c->launches++;
}

void launch_pcg32_replace(to3d_ctx* c, cudaStream_t s, const double* r64, double scale,
                          const float* p_latest, double delta2, double target2) {
    k_pcg32_replace<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(
        c->g, c->px, c->vol, r64, scale, c->dinv32, p_latest, c->r32, c->d32, c->red, c->ss,
        delta2, target2);
    c->launches++;
}

void launch_axpy_d32(to3d_ctx* c, cudaStream_t s, double inv_scale) {
    k_axpy_d32<<<vec_blocks(c->g.nnode), PCG_THREADS, 0, s>>>(c->g, c->px, c->vol, c->u, c->d32,
                                                               inv_scale);
    c->launches++;
}

void launch_norm2(to3d_ctx* c, cudaStream_t s, const double* v, long long n, double* out) {
    k_norm2<<<vec_blocks(n), PCG_THREADS, 0, s>>>(n, v, c->red, out);
    c->launches++;
}

void launch_ss_segment(to3d_ctx* c, cudaStream_t s, double tol2, int maxit) {
    k_ss_segment<<<1, 1, 0, s>>>(c->ss, tol2, maxit);
    c->launches++;
}

void launch_ss_reset(to3d_ctx* c, cudaStream_t s, double tol2, int maxit) {
    k_ss_reset<<<1, 1, 0, s>>>(c->ss, tol2, maxit);
    c->launches++;
}

}  // namespace to3d
