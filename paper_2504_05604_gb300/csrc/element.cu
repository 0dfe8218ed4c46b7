// Element-wise steps of one OC iteration: energies and sensitivities
// (Section 2.3), the rmin filter (Section 2.4) and the OC update with
// bisection on the volume multiplier (Section 2.3).
#include "internal.cuh"
#include "reduce.cuh"

namespace to3d {

constexpr int EL_THREADS = 256;

// ---------------------------------------------------------------- energies
// ce_e = u_e^T KE u_e, dc_e = -p x^(p-1) (E0-Emin) ce_e, c = sum E_e ce_e.
__global__ void __launch_bounds__(EL_THREADS)
    k_sensitivity(const __grid_constant__ KE64 ke, const Grid g, const double* __restrict__ x,
                  const double* __restrict__ u, double penal, double E0, double Emin,
                  double* __restrict__ ce_out, double* __restrict__ dc_out, const Reducer red,
                  double* comp_out) {
    __shared__ double sh[32];
    __shared__ double out[1];
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (e < g.nel) {
        const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / ((long long)g.nelx * g.nely);
        double ue[24];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const long long n = node_id(g, i + (b & 1), j + ((b >> 1) & 1), k + (b >> 2));
#pragma unroll
            for (int c = 0; c < 3; ++c) ue[3 * b + c] = u[3 * n + c];
        }
        double ce = 0.0;
#pragma unroll
        for (int r = 0; r < 24; ++r) {
            double s = 0.5 * ke.v[r * 24 + r] * ue[r];
#pragma unroll
            for (int q = r + 1; q < 24; ++q) s = fma(ke.v[r * 24 + q], ue[q], s);
            ce = fma(2.0 * ue[r], s, ce);
        }
        const double xe = x[e];
        const double xp1 = (penal == 3.0) ? xe * xe : pow(xe, penal - 1.0);
        const double Ee = Emin + xp1 * xe * (E0 - Emin);
        ce_out[e] = ce;
        dc_out[e] = -penal * xp1 * (E0 - Emin) * ce;
        contrib = Ee * ce;
    }
    double v[1] = {contrib};
    if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) *comp_out = out[0];
}

// dc_e = -p x^(p-1) (E0-Emin) ce_e and c = sum E_e ce_e from energies
// computed elsewhere (the sliced tensor-core path), same formulas as above.
__global__ void __launch_bounds__(EL_THREADS)
    k_sens_from_ce(long long nel, const double* __restrict__ x, const double* __restrict__ ce,
                   double penal, double E0, double Emin, double* __restrict__ dc_out,
                   const Reducer red, double* comp_out) {
    __shared__ double sh[32];
    __shared__ double out[1];
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double contrib = 0.0;
    if (e < nel) {
        const double xe = x[e], c = ce[e];
        const double xp1 = (penal == 3.0) ? xe * xe : pow(xe, penal - 1.0);
        const double Ee = Emin + xp1 * xe * (E0 - Emin);
        dc_out[e] = -penal * xp1 * (E0 - Emin) * c;
        contrib = Ee * c;
    }
    double v[1] = {contrib};
    if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) *comp_out = out[0];
}

// ---------------------------------------------------------------- filter
__device__ __forceinline__ void unpack_off(int o, int& di, int& dj, int& dk) {
    di = (o & 0xff) - 16;
    dj = ((o >> 8) & 0xff) - 16;
    dk = ((o >> 16) & 0xff) - 16;
}

// Hs_e = sum of the stencil weights that land inside the grid.
__global__ void k_hs(const __grid_constant__ Stencil st, const Grid g, double* __restrict__ Hs) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= g.nel) return;
    const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / ((long long)g.nelx * g.nely);
    double s = 0.0;
    for (int o = 0; o < st.n; ++o) {
        int di, dj, dk;
        unpack_off(st.off[o], di, dj, dk);
        const int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii >= 0 && ii < g.nelx && jj >= 0 && jj < g.nely && kk >= 0 && kk < g.nelz)
            s += st.w[o];
    }
    Hs[e] = s;
}

// mode 0 (sensitivity): out = H(a.b) / (Hs max(1e-3, a))     a = x, b = dc
// mode 1 (density):     out = H a / Hs
// mode 2 (density^T):   out = H (a / Hs)      (H is symmetric)
__global__ void __launch_bounds__(EL_THREADS)
    k_filter(const __grid_constant__ Stencil st, const Grid g, int mode,
             const double* __restrict__ a, const double* __restrict__ b,
             const double* __restrict__ Hs, double* __restrict__ outv) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= g.nel) return;
    const int i = e % g.nelx, j = (e / g.nelx) % g.nely, k = e / ((long long)g.nelx * g.nely);
    double s = 0.0;
    for (int o = 0; o < st.n; ++o) {
        int di, dj, dk;
        unpack_off(st.off[o], di, dj, dk);
        const int ii = i + di, jj = j + dj, kk = k + dk;
        if (ii >= 0 && ii < g.nelx && jj >= 0 && jj < g.nely && kk >= 0 && kk < g.nelz) {
            const long long n = elem_id(g, ii, jj, kk);
            double v = a[n];
            if (mode == 0) v *= b[n];
            else if (mode == 2) v /= Hs[n];
            s = fma(st.w[o], v, s);
        }
    }
    if (mode == 0) s /= Hs[e] * fmax(1e-3, a[e]);
    else if (mode == 1) s /= Hs[e];
    outv[e] = s;
}

// ---------------------------------------------------------------- OC update
// Candidate tree of `levels` bisection levels from bracket [l1, l2], in
// level order: node m has children 2m+1 (bracket [lo, mid]) and 2m+2
// ([mid, hi]); every midpoint is 0.5*(lo+hi) of its own bracket, which is
// exactly the value the scalar bisection would compute on that path.
__device__ void oc_build_tree(OCScalars* os) {
    double blo[63], bhi[63];
    const int nc = (1 << os->levels) - 1;
    blo[0] = os->l1;
    bhi[0] = os->l2;
    os->cand[0] = 0.5 * (os->l1 + os->l2);
    for (int m = 0; 2 * m + 2 < nc; ++m) {
        blo[2 * m + 1] = blo[m];
        bhi[2 * m + 1] = os->cand[m];
        os->cand[2 * m + 1] = 0.5 * (blo[m] + os->cand[m]);
        blo[2 * m + 2] = os->cand[m];
        bhi[2 * m + 2] = bhi[m];
        os->cand[2 * m + 2] = 0.5 * (os->cand[m] + bhi[m]);
    }
    os->ncand = nc;
}

__global__ void k_oc_init(OCScalars* os, int levels, double tol, double target, int maxhalv) {
    os->l1 = 0.0;
    os->l2 = 1e9;
    os->lmid = 0.5e9;
    os->tol = tol;
    os->target = target;
    os->levels = levels;
    os->halvings = 0;
    os->done = 0;
    os->status = 0;
    os->maxhalv = maxhalv;
    os->volume = 0.0;
    os->change = 0.0;
    if (!((os->l2 - os->l1) / (os->l1 + os->l2) > tol)) os->done = 1;
    oc_build_tree(os);
}

// Double-single numbers: v = hi + lo with two floats, |lo| <= ulp(hi) / 2,
// about 48 significant bits.  The bisection passes evaluate the design
// volume at 2^L - 1 candidates per element and pass; in FP64 that is four
// FP64 operations per candidate and element, and this GPU's FP64 pipe is
// narrow, so the passes work on double-single copies of q, lo and hi on the
// FP32 pipe.  A term clamp(q t, lo, hi) is then correct to about 2^-46 of
// its size and a pass's volume to about 1e-13 relative: a bisection decision
// could differ from the FP64 one only if the volume at a midpoint were that
// close to the target.
struct DS {
    float h, l;
};
__device__ __forceinline__ DS ds_from(double v) {
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ DS ds_mul(DS a, DS b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);          // exact error of the leading product
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    const float s = p + e;
    return {s, e - (s - p)};
}
__device__ __forceinline__ bool ds_lt(DS a, DS b) { return a.h < b.h || (a.h == b.h && a.l < b.l); }
// acc += v (two-sum of the leading parts, the rest into the low part)
__device__ __forceinline__ void ds_acc(DS& acc, DS v) {
    const float s = acc.h + v.h;
    const float bb = s - acc.h;
    const float err = (acc.h - (s - bb)) + (v.h - bb);
    const float l = acc.l + err + v.l;
    const float h2 = s + l;
    acc.l = l - (h2 - s);
    acc.h = h2;
}

// q = x sqrt(max(0,-dcf)), lo = max(0, x-move), hi = min(1, x+move); passive
// elements get q = lo = hi = 0 so they add nothing to the design volume.
// FP64 for the final update, double-single copies for the passes.
__global__ void k_oc_prep(long long nel, const double* __restrict__ x,
                          const double* __restrict__ dcf, const uint8_t* __restrict__ passive,
                          double move, double* __restrict__ q, double* __restrict__ lo,
                          double* __restrict__ hi, float* __restrict__ qs) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nel) return;
    const double xe = x[e];
    double qe = 0.0, le = 0.0, he = 0.0;
    if (!passive[e]) {
        qe = xe * sqrt(fmax(0.0, -dcf[e]));
        le = fmax(0.0, xe - move);
        he = fmin(1.0, xe + move);
    }
    q[e] = qe;
    lo[e] = le;
    hi[e] = he;
    const DS a = ds_from(qe), b = ds_from(le), c = ds_from(he);
    float2* o = reinterpret_cast<float2*>(qs + 6 * e);
    o[0] = make_float2(a.h, a.l);
    o[1] = make_float2(b.h, b.l);
    o[2] = make_float2(c.h, c.l);
}

// One pass: design volume at every candidate of the tree, then the last
// block walks the tree exactly as the scalar bisection would.
template <int LEV>
__global__ void __launch_bounds__(EL_THREADS)
    k_oc_pass(long long nel, const float* __restrict__ qs, const Reducer red, OCScalars* os,
              cudaGraphConditionalHandle loop, int use_loop) {
    if (os->done) {
        // inside a graph loop the body must always decide the loop condition
        if (use_loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(loop, 0u);
        return;
    }
    constexpr int NC = (1 << LEV) - 1;
    __shared__ double sh[32 * NC];
    __shared__ double out[NC];
    __shared__ float2 st[NC];
    if (threadIdx.x < NC) {
        // capped so that it stays finite in FP32 (q t then clamps at hi, or
        // is 0 for q = 0, as in FP64)
        const DS t = ds_from(fmin(1.0 / sqrt(os->cand[threadIdx.x]), 1e30));
        st[threadIdx.x] = make_float2(t.h, t.l);
    }
    __syncthreads();
    DS t[NC], acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        t[c] = {st[c].x, st[c].y};
        acc[c] = {0.f, 0.f};
    }
    const float2* q2 = reinterpret_cast<const float2*>(qs);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nel;
         e += (long long)gridDim.x * blockDim.x) {
        const float2 a = __ldg(q2 + 3 * e), b = __ldg(q2 + 3 * e + 1), d = __ldg(q2 + 3 * e + 2);
        const DS qe{a.x, a.y}, le{b.x, b.y}, he{d.x, d.y};
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            // clamp(q t, lo, hi) with lo <= hi
            const DS v = ds_mul(qe, t[c]);
            ds_acc(acc[c], ds_lt(v, le) ? le : (ds_lt(he, v) ? he : v));
        }
    }
    double v[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = (double)acc[c].h + (double)acc[c].l;
    if (grid_sum<NC>(red, v, sh, out) && threadIdx.x == 0) {
        int node = 0;
        for (int lev = 0; lev < LEV; ++lev) {
            if (!((os->l2 - os->l1) / (os->l1 + os->l2) > os->tol)) {
                os->done = 1;
                break;
            }
            const double lm = os->cand[node];
            os->lmid = lm;
            os->halvings += 1;
            if (out[node] > os->target) {
                os->l1 = lm;
                node = 2 * node + 2;
            } else {
                os->l2 = lm;
                node = 2 * node + 1;
            }
            if (os->halvings >= os->maxhalv) {
                os->status = TO3D_ENOCONV;
                os->done = 1;
                break;
            }
        }
        if (!os->done && !((os->l2 - os->l1) / (os->l1 + os->l2) > os->tol)) os->done = 1;
        if (!os->done) oc_build_tree(os);
        if (use_loop) cudaGraphSetConditional(loop, os->done ? 0u : 1u);
    }
}

// x_new at the last midpoint; passive pinned; change and design volume.
__global__ void __launch_bounds__(EL_THREADS)
    k_oc_apply(long long nel, const double* __restrict__ x, const double* __restrict__ q,
               const double* __restrict__ lo, const double* __restrict__ hi,
               const uint8_t* __restrict__ passive, double* __restrict__ xnew, const Reducer red,
               OCScalars* os) {
    __shared__ double sh[64];
    __shared__ double out[2];
    const double t = 1.0 / sqrt(os->lmid);
    double vol = 0.0, chg = 0.0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < nel;
         e += (long long)gridDim.x * blockDim.x) {
        const uint8_t pe = passive[e];
        double xn;
        if (pe == 1) xn = 0.0;
        else if (pe == 2) xn = 1.0;
        else {
            xn = fmax(lo[e], fmin(hi[e], q[e] * t));
            vol += xn;
        }
        chg = fmax(chg, fabs(xn - x[e]));
        xnew[e] = xn;
    }
    double v[2] = {vol, chg};
    if (grid_sum<2>(red, v, sh, out, 2u) && threadIdx.x == 0) {
        os->volume = out[0];
        os->change = out[1];
    }
}

// ---------------------------------------------------------------- input check
// *bad = 1 if any x_e lies outside [0, 1] (or is NaN); the flag is cleared
// by the caller
__global__ void k_check_unit(long long n, const double* __restrict__ x, int* bad) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x)
        if (!(x[e] >= 0.0 && x[e] <= 1.0)) *bad = 1;
}

// ---------------------------------------------------------------- launchers
static unsigned el_blocks(long long n) { return (unsigned)((n + EL_THREADS - 1) / EL_THREADS); }
static unsigned el_blocks_capped(long long n) {
    long long nb = (n + EL_THREADS - 1) / EL_THREADS;
    if (nb > 152 * 8) nb = 152 * 8;
    return (unsigned)(nb < 1 ? 1 : nb);
}

void launch_sensitivity(to3d_ctx* c, cudaStream_t s, const double* x, const double* u,
                        double* ce, double* dc) {
    if (c->prm.fp64_tc && matvec_x64_available(c)) {
        // energies on the tensor cores by exact slicing, then dc and c
        launch_energies_x64(c, s, u, ce);
        k_sens_from_ce<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(
            c->g.nel, x, ce, c->prm.penal, c->prm.E0, c->prm.Emin, dc, c->red, c->misc + 0);
        c->launches++;
        return;
    }
    k_sensitivity<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(
        c->ke, c->g, x, u, c->prm.penal, c->prm.E0, c->prm.Emin, ce, dc, c->red, c->misc + 0);
    c->launches++;
}

void launch_sensitivity_raw(const KE64& ke, const Grid& g, cudaStream_t s, const double* x,
                            const double* u, double penal, double E0, double Emin, double* ce,
                            double* dc, const Reducer& red, double* comp_out) {
    k_sensitivity<<<el_blocks(g.nel), EL_THREADS, 0, s>>>(ke, g, x, u, penal, E0, Emin, ce, dc, red,
                                                          comp_out);
}

// passive elements keep their pinned density: void 0, solid 1
// v_e = void_val on void and solid_val on solid passive elements
__global__ void k_pin_passive(long long nel, const uint8_t* __restrict__ passive,
                              double* __restrict__ x, double void_val, double solid_val) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nel) return;
    const uint8_t t = passive[e];
    if (t == 1) x[e] = void_val;
    else if (t == 2) x[e] = solid_val;
}

void launch_check_unit(to3d_ctx* c, cudaStream_t s, const double* x, int* bad) {
    k_check_unit<<<el_blocks_capped(c->g.nel), EL_THREADS, 0, s>>>(c->g.nel, x, bad);
    c->launches++;
}

void launch_pin_passive(to3d_ctx* c, cudaStream_t s, double* x) {
    if (!c->passive) return;
    k_pin_passive<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(c->g.nel, c->passive, x, 0.0, 1.0);
    c->launches++;
}

// The filtered densities of passive elements are pinned, so they do not
// depend on x: their sensitivities carry nothing back through the density
// filter's chain rule.
void launch_zero_passive(to3d_ctx* c, cudaStream_t s, double* v) {
    if (!c->passive) return;
    k_pin_passive<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(c->g.nel, c->passive, v, 0.0, 0.0);
    c->launches++;
}

void launch_hs(to3d_ctx* c, cudaStream_t s) {
    k_hs<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(*c->st, c->g, c->Hs);
    c->launches++;
}

void launch_filter(to3d_ctx* c, cudaStream_t s, int mode, const double* a, const double* b,
                   double* outv) {
    k_filter<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(*c->st, c->g, mode, a, b, c->Hs, outv);
    c->launches++;
}

void launch_oc_begin(to3d_ctx* c, cudaStream_t s, const double* x, const double* dcf,
                     double target) {
    k_oc_prep<<<el_blocks(c->g.nel), EL_THREADS, 0, s>>>(c->g.nel, x, dcf, c->passive,
                                                        c->prm.move, c->ocq, c->oclo, c->ochi, c->ocs);
    k_oc_init<<<1, 1, 0, s>>>(c->os, c->prm.oc_levels, c->prm.bisect_tol, target, 400);
    c->launches += 2;
}

void launch_oc_passes(to3d_ctx* c, cudaStream_t s, int npass, cudaGraphConditionalHandle loop,
                      int use_loop) {
    const unsigned nb = el_blocks_capped(c->g.nel);
    for (int i = 0; i < npass; ++i) {
        switch (c->prm.oc_levels) {
            case 1: k_oc_pass<1><<<nb, EL_THREADS, 0, s>>>(c->g.nel, c->ocs, c->red, c->os, loop, use_loop); break;
            case 2: k_oc_pass<2><<<nb, EL_THREADS, 0, s>>>(c->g.nel, c->ocs, c->red, c->os, loop, use_loop); break;
            case 3: k_oc_pass<3><<<nb, EL_THREADS, 0, s>>>(c->g.nel, c->ocs, c->red, c->os, loop, use_loop); break;
            case 4: k_oc_pass<4><<<nb, EL_THREADS, 0, s>>>(c->g.nel, c->ocs, c->red, c->os, loop, use_loop); break;
            default: k_oc_pass<5><<<nb, EL_THREADS, 0, s>>>(c->g.nel, c->ocs, c->red, c->os, loop, use_loop); break;
        }
        c->launches++;
    }
}

void launch_oc_apply(to3d_ctx* c, cudaStream_t s, const double* x, double* xnew) {
    k_oc_apply<<<el_blocks_capped(c->g.nel), EL_THREADS, 0, s>>>(
        c->g.nel, x, c->ocq, c->oclo, c->ochi, c->passive, xnew, c->red, c->os);
    c->launches++;
}

}  // namespace to3d
