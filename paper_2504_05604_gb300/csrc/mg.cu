// Learned multigrid preconditioner for the state equation K u = f.
//
// The paper solves K U = F with a sparse direct solver (Section 2.2); the
// library solves it iteratively, and Jacobi-preconditioned CG needs thousands
// of iterations on fine SIMP grids.  This file builds a geometric multigrid
// V-cycle on the same operator K = sum_e E_e KE whose free parameters are
// learned from the method's own residuals:
//
//   hierarchy   level l+1 halves every element count of level l, rounding
//               up; coarse node C sits on fine node 2C; a coarse dof is
//               clamped when the fine dof at 2C is.  Each coarse level is a
//               full context of its own (same element, same tensor-core
//               kernel), created once per design grid.
//   coarse K    rediscretised: coarse element modulus s_l (mean over the 8
//               child slots of E^q_l)^(1/q_l), missing children 0 (s = 2 and
//               any q give the Galerkin operator for a uniform modulus).
//   transfer    trilinear prolongation, restriction its transpose.
//   smoother    damped Jacobi, one sweep before and one after the coarse
//               correction, `sweeps` sweeps on the coarsest level; damping
//               om_l = w_l * 2 / lam_l with lam_l = min(1.2 rq_l, l1), rq_l
//               the Rayleigh quotient of D^-1 K after 16 power steps from a
//               fixed hashed start vector, l1 = max_a sum_b |KE_ab| / KE_aa
//               (no modulus field exceeds it): every sweep with 0 < w < 1
//               converges, also on nodes bounded by void elements.
//   learned     theta = (w_g for g = 0..3, q_g and s_g for g = 1..3), group g
//               = min(level, 3), so parameters learned on one grid size apply
//               to any other.  Training minimises the energy-norm error that
//               one application leaves, ||e - V r||_K^2 / ||e||_K^2 with
//               e = K^-1 r, over residual snapshots of the context's own
//               design, by Adam on central-difference gradients.
//
// The cycle runs in FP32 on the padded structure-of-arrays vectors of each
// level, every operator application on the tensor cores (the context's
// operand form).  It is linear in its input and symmetric up to that
// rounding, so it serves flexible CG in FP64 (TO3D_F64) and an FP32 inner
// CG inside the FP64 defect correction (the *_DC forms).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "reduce.cuh"

#define MG_CK(call)                                             \
    do {                                                        \
        cudaError_t _e = (call);                                \
        if (_e != cudaSuccess) return cuda_check(c, _e, #call); \
    } while (0)

namespace to3d {
namespace mg {

constexpr int kGroups = 4;                          // level 0, 1, 2, >= 3
constexpr int kParams = kGroups + 2 * (kGroups - 1);
constexpr int kMaxLevels = 12;
constexpr int kThreads = 256;

struct Level {
    to3d_ctx* ctx = nullptr;     // level 0: the owning context (not owned here)
    float* z = nullptr;          // cycle solution (padded SoA, 3 vol)
    float* t = nullptr;          // operator output
    CUtensorMap tm_z;
};

struct Snap {
    double* r = nullptr;         // residual (AoS FP64, dofs)
    double rn = 0.0;             // |r|
    double rte = 0.0;            // r^T K^-1 r for the operator of its design
    int design = 0;              // index into Mg::designs
};

constexpr int kBottomMaxLevels = 8;
constexpr int kBottomThreads = 1024;
constexpr int kBottomSmem = 200 * 1024;

struct BottomLevel {
    Grid g;
    int px, pex;
    long long vol;
    const float* E32;
    const float* dinv32;
    const uint8_t* maskp;
    int ob, oz, ot, od, oE;      // float offsets in shared memory
    int om;                      // byte offset of the clamp bits
};

struct BottomArgs {
    int nb, lb, sweeps, nu;
    BottomLevel L[kBottomMaxLevels];
    const float* b_in;           // right-hand side of level lb (padded SoA)
    float* z_out;                // solution of level lb (padded SoA)
    const float* KE;             // unit KE, FP32
    const float* wdev;
};

struct Mg {
    std::vector<Level> lv;
    double theta[kParams];
    float* wdev = nullptr;            // damping per level (device)
    double* lamdev = nullptr;         // eigenvalue bound per level (device)
    double l1 = 59.0 / 11.0;          // max_a sum_b |KE_ab| / KE_aa
    int sweeps = 6;
    int nu = 1;                       // smoothing sweeps before and after the coarse correction
    int lb = 1 << 30;                 // first level of the one-CTA bottom cycle
    BottomArgs bottom;                // its level table (b_in, z_out set per launch)
    int bottom_smem = 0;
    int prec = TO3D_BF16_DC;
    cudaGraphExec_t cycle = nullptr;  // ctx->r32 -> lv[0].z, captured
    long long cycle_launches = 0;     // kernels in one cycle
    bool params_dirty = true;         // coarse moduli / weights not set up for the current operator
    double* z64 = nullptr;            // FP64 flexible-CG buffers
    double* rprev = nullptr;
    double* dots = nullptr;
    double* dots_h = nullptr;
    float* ones = nullptr;            // per-node scaling 1 (fused direction p = z + beta p)
    float* ke32 = nullptr;            // unit KE in FP32 (the one-CTA bottom cycle)
    CUtensorMap tm_ones;
    cudaGraphExec_t pcg = nullptr;    // chunk of inner MG-PCG iterations
    int pcg_prec = -1, pcg_n = 0;
    std::vector<Snap> snaps;
    std::vector<double*> designs;     // densities the snapshots belong to (device)
    bool trained = false;
};

static int group(int l) { return l < kGroups - 1 ? l : kGroups - 1; }
static double w_of(const Mg* m, int l) { return m->theta[group(l)]; }
static double q_of(const Mg* m, int l) { return m->theta[kGroups + group(l) - 1]; }
static double s_of(const Mg* m, int l) { return m->theta[2 * kGroups - 1 + group(l) - 1]; }

constexpr int kPowerSteps = 16;
constexpr double kPowerMargin = 1.2;

static void default_theta(double* th) {
    for (int g = 0; g < kGroups; ++g) th[g] = 2.0 / 3.0;
    for (int g = 1; g < kGroups; ++g) {
        th[kGroups + g - 1] = 1.0;
        th[2 * kGroups - 1 + g - 1] = 2.0;
    }
}

static bool theta_valid(const double* th) {
    for (int g = 0; g < kGroups; ++g)
        if (!(th[g] > 0.0 && th[g] < 1.0)) return false;   // fraction of the stability limit
    for (int g = 1; g < kGroups; ++g) {
        const double q = th[kGroups + g - 1], s = th[2 * kGroups - 1 + g - 1];
        if (!(q >= 0.125 && q <= 8.0) || !(s > 0.0 && s <= 64.0)) return false;
    }
    return true;
}

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ bool skip(const SolverScalars* ss) { return ss && ss->done; }

// z = w D^-1 b (first smoothing sweep, from z = 0); clamped dofs and pads 0
__global__ void k_jacobi0(long long vol, const float* __restrict__ b, const float* __restrict__ dinv,
                          const uint8_t* __restrict__ maskp, const float* __restrict__ wdev, int l,
                          float* __restrict__ z, const SolverScalars* ss) {
    if (skip(ss)) return;
    const float w = wdev[l];
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < vol;
         n += (long long)gridDim.x * blockDim.x) {
        const float d = w * dinv[n];
        const uint8_t m = maskp[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[c * vol + n] = ((m >> c) & 1) ? 0.f : d * b[c * vol + n];
    }
}

// z += w D^-1 (b - t), t = K z
__global__ void k_jacobi(long long vol, const float* __restrict__ b, const float* __restrict__ t,
                         const float* __restrict__ dinv, const uint8_t* __restrict__ maskp,
                         const float* __restrict__ wdev, int l, float* __restrict__ z,
                         const SolverScalars* ss) {
    if (skip(ss)) return;
    const float w = wdev[l];
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < vol;
         n += (long long)gridDim.x * blockDim.x) {
        const float d = w * dinv[n];
        const uint8_t m = maskp[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long i = c * vol + n;
            z[i] = ((m >> c) & 1) ? 0.f : fmaf(d, b[i] - t[i], z[i]);
        }
    }
}

// Restriction: b_c = R (b_f - t_f), each coarse node gathering the 27 fine
// nodes 2C + d with weights prod (1 - |d| / 2); clamped dofs of either grid
// contribute 0.  The 27 points are unrolled (bounds as predicates), so all
// their loads are in flight together.
__global__ void k_restrict(const Grid gf, int pxf, long long volf, const float* __restrict__ bf,
                           const float* __restrict__ tf, const uint8_t* __restrict__ maskf,
                           const Grid gc, int pxc, long long volc, const uint8_t* __restrict__ maskc,
                           float* __restrict__ bc, const SolverScalars* ss) {
    if (skip(ss)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= gc.nx) return;
    const long long planef = (long long)pxf * gf.ny;
    const long long base = 2 * i + (long long)pxf * (2 * j) + planef * (2 * k);
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int dk = -1; dk <= 1; ++dk) {
        const bool okk = 2 * k + dk >= 0 && 2 * k + dk < gf.nz;
#pragma unroll
        for (int dj = -1; dj <= 1; ++dj) {
            const bool okj = okk && 2 * j + dj >= 0 && 2 * j + dj < gf.ny;
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
                if (!(okj && 2 * i + di >= 0 && 2 * i + di < gf.nx)) continue;
                const float wt = (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * (dk ? 0.5f : 1.f);
                const long long p = base + di + (long long)pxf * dj + planef * dk;
                const uint8_t m = maskf[p];
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    if (!((m >> c) & 1)) acc[c] = fmaf(wt, bf[c * volf + p] - tf[c * volf + p], acc[c]);
            }
        }
    }
    const long long pc = i + (long long)pxc * (j + (long long)gc.ny * k);
    const uint8_t mc = maskc[pc];
#pragma unroll
    for (int c = 0; c < 3; ++c) bc[c * volc + pc] = ((mc >> c) & 1) ? 0.f : acc[c];
}

// Prolongation z_f += P z_c (trilinear), clamped fine dofs untouched (they
// stay 0), in two forms with the same arithmetic.
//
// k_prolong: one thread per fine node (2C + d gathers the coarse nodes C..C+1
// along the odd axes, weight 1/2 per odd axis); the eight candidates are
// unrolled with predicates.  Used on the small grids, where latency rules.
__global__ void k_prolong(const Grid gf, int pxf, long long volf, const uint8_t* __restrict__ maskf,
                          float* __restrict__ zf, const Grid gc, int pxc, long long volc,
                          const float* __restrict__ zc, const SolverScalars* ss) {
    if (skip(ss)) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y, k = blockIdx.z;
    if (i >= gf.nx) return;
    const bool ox = i & 1, oy = j & 1, oz = k & 1;
    const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f) * (oz ? 0.5f : 1.f);
    const long long planec = (long long)pxc * gc.ny;
    const long long base = (i >> 1) + (long long)pxc * (j >> 1) + planec * (k >> 1);
    float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                if ((cc && !ox) || (bb && !oy) || (a && !oz)) continue;
                const long long p = base + cc + (long long)pxc * bb + planec * a;
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[c] = fmaf(w, zc[c * volc + p], acc[c]);
            }
    const long long pf = i + (long long)pxf * (j + (long long)gf.ny * k);
    const uint8_t m = maskf[pf];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        if (!((m >> c) & 1)) zf[c * volf + pf] += acc[c];
}

// k_prolong_col: one thread per coarse node (i, j, k), 32 consecutive i per
// warp, adding to the fine nodes (2i + a, 2j + b, 2k + c), a, b, c in {0, 1},
// from the coarse nodes (i..i+1, j..j+1, k..k+1) with the trilinear weights
// applied axis by axis; the i + 1 neighbour comes from the next lane by
// warp shuffle.  Each coarse value is loaded once per thread instead of
// once per fine node: used on the large grids, where instructions rule.
constexpr int kColX = 32, kColY = 4;
__global__ void __launch_bounds__(kColX * kColY)
    k_prolong_col(const Grid gf, int pxf, long long volf, const uint8_t* __restrict__ maskf,
                  float* __restrict__ zf, const Grid gc, int pxc, long long volc,
                  const float* __restrict__ zc, const SolverScalars* ss) {
    if (skip(ss)) return;
    const int lane = threadIdx.x;
    const int i = blockIdx.x * kColX + lane, j = blockIdx.y * kColY + threadIdx.y, k = blockIdx.z;
    // no early return below: the shuffles need every lane of the warp
    const bool col = i < gc.nx && j < gc.ny;
    const long long planec = (long long)pxc * gc.ny, planef = (long long)pxf * gf.ny;
    const bool okj1 = j + 1 < gc.ny;
    // X[b][a][c]: the x-interpolated coarse values of row j + b at fine x
    // offset a, for one coarse layer
    auto load = [&](int kl, float (&X)[2][2][3]) {
        const bool kok = col && kl < gc.nz;
        const long long p = kok ? i + (long long)pxc * j + planec * kl : 0;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const bool ok = kok && (b == 0 || okj1);
            const long long pb = p + (b ? pxc : 0);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float z0 = ok ? zc[c * volc + pb] : 0.f;
                float z1 = __shfl_down_sync(0xffffffffu, z0, 1);
                if (lane == kColX - 1) z1 = (ok && i + 1 < gc.nx) ? zc[c * volc + pb + 1] : 0.f;
                X[b][0][c] = z0;
                X[b][1][c] = 0.5f * (z0 + z1);
            }
        }
    };
    float Xk[2][2][3], Xn[2][2][3];
    load(k, Xk);
    load(k + 1, Xn);
    if (!col) return;
#pragma unroll
    for (int cz = 0; cz < 2; ++cz) {
        const int fk = 2 * k + cz;
        if (fk >= gf.nz) continue;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int fj = 2 * j + b;
            if (fj >= gf.ny) continue;
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int fi = 2 * i + a;
                if (fi >= gf.nx) continue;
                const long long pf = fi + (long long)pxf * fj + planef * fk;
                const uint8_t m = maskf[pf];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    // y then z interpolation of the x-interpolated values
                    const float lo = b ? 0.5f * (Xk[0][a][c] + Xk[1][a][c]) : Xk[0][a][c];
                    const float hi = b ? 0.5f * (Xn[0][a][c] + Xn[1][a][c]) : Xn[0][a][c];
                    const float v = cz ? 0.5f * (lo + hi) : lo;
                    if (!((m >> c) & 1)) zf[c * volf + pf] += v;
                }
            }
        }
    }
}

// coarse moduli: s (sum over the 8 child slots of E^q / 8)^(1/q), missing 0
__global__ void k_coarsen(const Grid gf, const double* __restrict__ Ef, const Grid gc, double q,
                          double s, double* __restrict__ Ec, float* __restrict__ E32c, int pexc) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= gc.nel) return;
    const int i = e % gc.nelx, j = (e / gc.nelx) % gc.nely, k = e / ((long long)gc.nelx * gc.nely);
    // powers in FP32 (the coarse operator needs no more than that) of the
    // children relative to the largest one, so that no power underflows:
    // (mean E^q)^(1/q) = E_max (mean (E / E_max)^q)^(1/q)
    double ch[8];
    double vmax = 0.0;
    for (int c = 0; c < 2; ++c)
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int fi = 2 * i + a, fj = 2 * j + b, fk = 2 * k + c;
                const double v = (fi < gf.nelx && fj < gf.nely && fk < gf.nelz)
                                     ? Ef[elem_id(gf, fi, fj, fk)] : 0.0;
                ch[a + 2 * b + 4 * c] = v;
                vmax = fmax(vmax, v);
            }
    double v = 0.0;
    if (vmax > 0.0) {
        if (q == 1.0) {
            double acc = 0.0;
            for (int t = 0; t < 8; ++t) acc += ch[t];
            v = s * acc / 8.0;
        } else {
            const float qf = (float)q;
            float acc = 0.f;
            for (int t = 0; t < 8; ++t) acc += powf((float)(ch[t] / vmax), qf);
            v = s * vmax * (double)powf(acc / 8.f, 1.f / qf);
        }
    }
    Ec[e] = v;
    E32c[i + (long long)pexc * (j + (long long)gc.nely * k)] = (float)v;
}

// b = scale r64 (AoS FP64 -> padded SoA FP32), clamped dofs 0
__global__ void k_in(const Grid g, int px, long long vol, const double* __restrict__ r64, double scale,
                     const uint8_t* __restrict__ nodemask, float* __restrict__ b) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long p = (n % g.nx) + (long long)px * (n / g.nx);
        const uint8_t m = nodemask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) b[c * vol + p] = ((m >> c) & 1) ? 0.f : (float)(r64[3 * n + c] * scale);
    }
}

// z64 = z / scale (padded SoA FP32 -> AoS FP64)
__global__ void k_out(const Grid g, int px, long long vol, const float* __restrict__ z, double inv_scale,
                      double* __restrict__ z64) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long p = (n % g.nx) + (long long)px * (n / g.nx);
#pragma unroll
        for (int c = 0; c < 3; ++c) z64[3 * n + c] = (double)z[c * vol + p] * inv_scale;
    }
}

__global__ void k_fill(long long n, float v, float* __restrict__ a) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        a[i] = v;
}

// beta of the inner MG-PCG from rz = r.z and zq = z.q_old (see below)
__device__ __forceinline__ void set_beta(SolverScalars* ss, double rzn, double zq) {
    const bool first = ss->pad0 != 0;
    // right after a residual replacement the recurrence r_new - r_old =
    // -alpha q_old no longer holds: Fletcher-Reeves beta once
    const bool fr = ss->pad1 != 0;
    const double beta = first ? 0.0 : (fr ? rzn / ss->rz : -ss->alpha * zq / ss->rz);
    ss->pad0 = 0;
    ss->pad1 = 0;
    ss->beta = beta;
    ss->zcoef = 1.0;
    ss->rz = rzn;
    if (!(rzn > 0.0) || !isfinite(rzn) || !isfinite(beta)) {
        ss->status = TO3D_ENUMERIC;
        ss->done = 1;
    }
}

// Inner MG-PCG, after the cycle z = V r: rz = r.z and z.q_old give the
// Polak-Ribiere coefficient beta = z_new.(r_new - r_old) / rz_old
// = -alpha z_new.q_old / rz_old (0 on the first step of a segment).
__global__ void k_pcg_dots(long long vol, const float* __restrict__ r, const float* __restrict__ z,
                           const float* __restrict__ q, const Reducer red, SolverScalars* ss) {
    if (ss->done) return;
    __shared__ double sh[64];
    __shared__ double out[2];
    // 3 vol is a multiple of 4: float4 loads; FP32 partial sums of 4 x 8
    // products per thread and step, FP64 across steps, blocks and the grid
    const long long n4 = (3 * vol) >> 2;
    const float4* r4 = reinterpret_cast<const float4*>(r);
    const float4* z4 = reinterpret_cast<const float4*>(z);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    double rz = 0.0, zq = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n4;
         i += (long long)gridDim.x * blockDim.x) {
        const float4 a = r4[i], b = z4[i], c4 = q4[i];
        rz += (double)fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
        zq += (double)fmaf(b.x, c4.x, fmaf(b.y, c4.y, fmaf(b.z, c4.z, b.w * c4.w)));
    }
    double v[2] = {rz, zq};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) set_beta(ss, out[0], out[1]);
}

// The level-0 cycle's last smoothing sweep, z += w D^-1 (b - t) with b = r,
// fused with the two dots of k_pcg_dots (r.z and z.q_old) and its beta.
// Four consecutive nodes per step (vol is a multiple of 4: 16-byte loads,
// 14 of them in flight per thread); FP32 partial sums of the 12 products of
// a step, FP64 across steps, blocks and the grid (one FP64 add per node
// would load this GPU's narrow FP64 pipe).
__global__ void __launch_bounds__(256)
    k_jacobi_dots(long long vol, const float* __restrict__ b, const float* __restrict__ t,
                  const float* __restrict__ dinv, const uint8_t* __restrict__ maskp,
                  const float* __restrict__ wdev, float* __restrict__ z, const float* __restrict__ q,
                  const Reducer red, SolverScalars* ss) {
    if (ss->done) return;
    __shared__ double sh[64];
    __shared__ double out[2];
    const float w = wdev[0];
    const long long v4 = vol >> 2;
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4* t4 = reinterpret_cast<const float4*>(t);
    const float4* q4 = reinterpret_cast<const float4*>(q);
    const float4* di4 = reinterpret_cast<const float4*>(dinv);
    const uchar4* m4 = reinterpret_cast<const uchar4*>(maskp);
    float4* z4 = reinterpret_cast<float4*>(z);
    double rz = 0.0, zq = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < v4;
         n += (long long)gridDim.x * blockDim.x) {
        const float4 di = __ldg(di4 + n);
        const uchar4 mk = __ldg(m4 + n);
        float4 bb[3], tt[3], zz[3], qq[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            bb[c] = __ldg(b4 + c * v4 + n);
            tt[c] = __ldg(t4 + c * v4 + n);
            zz[c] = z4[c * v4 + n];
            qq[c] = __ldg(q4 + c * v4 + n);
        }
        float prz = 0.f, pzq = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float4 zv;
            zv.x = ((mk.x >> c) & 1) ? 0.f : fmaf(w * di.x, bb[c].x - tt[c].x, zz[c].x);
            zv.y = ((mk.y >> c) & 1) ? 0.f : fmaf(w * di.y, bb[c].y - tt[c].y, zz[c].y);
            zv.z = ((mk.z >> c) & 1) ? 0.f : fmaf(w * di.z, bb[c].z - tt[c].z, zz[c].z);
            zv.w = ((mk.w >> c) & 1) ? 0.f : fmaf(w * di.w, bb[c].w - tt[c].w, zz[c].w);
            z4[c * v4 + n] = zv;
            prz = fmaf(bb[c].x, zv.x, fmaf(bb[c].y, zv.y, fmaf(bb[c].z, zv.z, fmaf(bb[c].w, zv.w, prz))));
            pzq = fmaf(zv.x, qq[c].x, fmaf(zv.y, qq[c].y, fmaf(zv.z, qq[c].z, fmaf(zv.w, qq[c].w, pzq))));
        }
        rz += (double)prz;
        zq += (double)pzq;
    }
    double v[2] = {rz, zq};
    if (grid_sum<2>(red, v, sh, out) && threadIdx.x == 0) set_beta(ss, out[0], out[1]);
}

// Segment start: r32 = scale r64 (masked), d = 0, p_old = 0, q = 0; |r32|^2
__global__ void k_pcg_init(const Grid g, int px, long long vol, const double* __restrict__ r64, double scale,
                           const uint8_t* __restrict__ nodemask, float* __restrict__ r32,
                           float* __restrict__ d32, float* __restrict__ p_old, float* __restrict__ q,
                           const Reducer red, SolverScalars* ss) {
    __shared__ double sh[32];
    __shared__ double out[1];
    double rr = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long p = (n % g.nx) + (long long)px * (n / g.nx);
        const uint8_t m = nodemask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = ((m >> c) & 1) ? 0.f : (float)(r64[3 * n + c] * scale);
            r32[c * vol + p] = v;
            d32[c * vol + p] = 0.f;
            p_old[c * vol + p] = 0.f;
            q[c * vol + p] = 0.f;
            rr = fma((double)v, (double)v, rr);
        }
    }
    double v[1] = {rr};
    if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) {
        ss->rr = out[0];
        ss->beta = 0.0;
        ss->zcoef = 1.0;
        ss->pad0 = 1;        // the next k_pcg_dots starts a new direction sequence
        if (!isfinite(out[0])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[0] <= ss->tol2) {
            ss->done = 1;
        }
    }
}

// Power iteration for lam_max(D^-1 K).  Start: entry of dof d = 3 node + c
// is frac(d * 2654435761 / 2^32) - 1/2 (Knuth's multiplicative hash), 0 on
// clamped dofs, nodes with D = 0 and pads.
__global__ void k_pow_start(const Grid g, int px, long long vol, const float* __restrict__ dinv,
                            const uint8_t* __restrict__ maskp, float* __restrict__ z) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < vol;
         p += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(p % px);
        const long long jk = p / px;
        const long long node = i + (long long)g.nx * jk;
        const uint8_t m = maskp[p];
        const bool ok = i < g.nx && dinv[p] > 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const uint32_t h = (uint32_t)(3 * node + c) * 2654435761u;
            z[c * vol + p] = (ok && !((m >> c) & 1)) ? (float)((double)h * 0x1p-32 - 0.5) : 0.f;
        }
    }
}

// out[0] = z.t, out[1] = z.D z (D = 1 / dinv on dofs with dinv > 0)
// Four consecutive nodes per step (vol is a multiple of 4: 16-byte loads);
// FP32 products and partial sums of a step (a Rayleigh quotient needs no
// more), FP64 across steps, blocks and the grid.
__global__ void __launch_bounds__(256)
    k_pow_dots(long long vol, const float* __restrict__ z, const float* __restrict__ t,
               const float* __restrict__ dinv, const uint8_t* __restrict__ maskp, const Reducer red,
               double* out_dev) {
    __shared__ double sh[64];
    __shared__ double o2[2];
    const long long v4 = vol >> 2;
    const float4* z4 = reinterpret_cast<const float4*>(z);
    const float4* t4 = reinterpret_cast<const float4*>(t);
    const float4* di4 = reinterpret_cast<const float4*>(dinv);
    const uchar4* m4 = reinterpret_cast<const uchar4*>(maskp);
    double a = 0.0, b = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < v4;
         n += (long long)gridDim.x * blockDim.x) {
        const float4 di = __ldg(di4 + n);
        const uchar4 mk = __ldg(m4 + n);
        float4 zz[3], tt[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            zz[c] = __ldg(z4 + c * v4 + n);
            tt[c] = __ldg(t4 + c * v4 + n);
        }
        const float dv[4] = {di.x, di.y, di.z, di.w};
        const uint8_t mv[4] = {mk.x, mk.y, mk.z, mk.w};
        float pa = 0.f, pb = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!(dv[k] > 0.f)) continue;
            const float dn = 1.f / dv[k];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                if ((mv[k] >> c) & 1) continue;
                const float zv = k == 0 ? zz[c].x : k == 1 ? zz[c].y : k == 2 ? zz[c].z : zz[c].w;
                const float tv = k == 0 ? tt[c].x : k == 1 ? tt[c].y : k == 2 ? tt[c].z : tt[c].w;
                pa = fmaf(zv, tv, pa);
                pb = fmaf(zv * zv, dn, pb);
            }
        }
        a += (double)pa;
        b += (double)pb;
    }
    double v[2] = {a, b};
    if (grid_sum<2>(red, v, sh, o2) && threadIdx.x == 0) {
        out_dev[0] = o2[0];
        out_dev[1] = o2[1];
    }
}

// z = D^-1 t / rq, rq = out[0] / out[1]
__global__ void k_pow_next(long long vol, const float* __restrict__ t, const float* __restrict__ dinv,
                           const uint8_t* __restrict__ maskp, const double* __restrict__ out,
                           float* __restrict__ z) {
    const double rq = out[1] > 0.0 ? out[0] / out[1] : 1.0;
    const float inv = (float)(rq > 0.0 ? 1.0 / rq : 1.0);
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < vol;
         n += (long long)gridDim.x * blockDim.x) {
        const float di = dinv[n] * inv;
        const uint8_t m = maskp[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) z[c * vol + n] = ((m >> c) & 1) ? 0.f : di * t[c * vol + n];
    }
}

// wdev[l] = w * 2 / min(margin rq, l1)
__global__ void k_pow_final(const double* __restrict__ out, double w, double margin, double l1,
                            float* __restrict__ wdev, int l, double* __restrict__ lam_out) {
    const double rq = out[1] > 0.0 ? out[0] / out[1] : l1;
    const double lam = fmin(margin * rq, l1);
    const double lam_ok = lam > 0.0 ? lam : l1;
    wdev[l] = (float)(w * 2.0 / lam_ok);
    lam_out[l] = lam_ok;
}

// t += K z over the elements of one bottom level, TPE threads per element:
// each thread gathers its element's 24 values of z and forms the rows of
// 8 / TPE local nodes (row by row from float4 reads of the unit KE in shared
// memory), scaled by E_e and added into t with shared-memory atomics.  More
// threads per element shorten the dependent chains on the small levels.
template <int TPE>
__device__ __forceinline__ void bottom_op_items(const Grid& g, const float* __restrict__ Ks,
                                                const float* z, float* t, const float* Es, int tid,
                                                int nt) {
    constexpr int NQ = 8 / TPE;
    const int nel = (int)g.nel, nelx = g.nelx, nely = g.nely, nx = g.nx, ny = g.ny;
    for (int w = tid; w < TPE * nel; w += nt) {
        const int e = w / TPE, part = w - e * TPE;
        const int ei = e % nelx, ej = (e / nelx) % nely, ek = e / (nelx * nely);
        const int n0 = ei + nx * (ej + ny * ek);
        float ze[24];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int nd = n0 + (q & 1) + nx * (((q >> 1) & 1) + ny * (q >> 2));
#pragma unroll
            for (int c = 0; c < 3; ++c) ze[3 * q + c] = z[3 * nd + c];
        }
        const float Ee = Es[e];
#pragma unroll
        for (int qq = 0; qq < NQ; ++qq) {
            const int q = part * NQ + qq;
            const int nd = n0 + (q & 1) + nx * (((q >> 1) & 1) + ny * (q >> 2));
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float4* row = reinterpret_cast<const float4*>(Ks + (3 * q + c) * 24);
                float acc = 0.f;
#pragma unroll
                for (int k4 = 0; k4 < 6; ++k4) {
                    const float4 kv = row[k4];
                    acc = fmaf(kv.x, ze[4 * k4 + 0], acc);
                    acc = fmaf(kv.y, ze[4 * k4 + 1], acc);
                    acc = fmaf(kv.z, ze[4 * k4 + 2], acc);
                    acc = fmaf(kv.w, ze[4 * k4 + 3], acc);
                }
                atomicAdd(&t[3 * nd + c], Ee * acc);
            }
        }
    }
}

// The V-cycle over the bottom levels in one CTA.  Levels lb..L whose
// vectors, damping, clamp bits and moduli fit in shared memory together
// (kBottomSmem) run inside one kernel: every operator application element by
// element in FP32 on the CUDA cores (24 x 24 products, shared-memory atomics
// into the nodes; bottom_op_items), restriction, prolongation and the damped-Jacobi sweeps
// as in the per-level kernels, __syncthreads between the steps.  On the
// largest grids that is the last four levels, whose per-level launches were
// bound by launch latency.
__global__ void __launch_bounds__(kBottomThreads, 1)
    k_cycle_bottom(const __grid_constant__ BottomArgs a, const SolverScalars* ss) {
    if (skip(ss)) return;
    extern __shared__ float bsm[];
    uint8_t* bytes = reinterpret_cast<uint8_t*>(bsm);
    float* Ks = bsm;                                  // 576 floats at offset 0
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < 576; i += nt) Ks[i] = a.KE[i];
    for (int li = 0; li < a.nb; ++li) {
        const BottomLevel& L = a.L[li];
        const float w = a.wdev[a.lb + li];
        const int nn = (int)L.g.nnode;
        for (int n = tid; n < nn; n += nt) {
            const int i = n % L.g.nx, jk = n / L.g.nx;
            const long long p = i + (long long)L.px * jk;
            bsm[L.od + n] = w * L.dinv32[p];
            bytes[L.om + n] = L.maskp[p];
            if (li == 0)
                for (int c = 0; c < 3; ++c) bsm[L.ob + 3 * n + c] = a.b_in[c * L.vol + p];
        }
        for (int e = tid; e < (int)L.g.nel; e += nt) {
            const int ei = e % L.g.nelx, ej = (e / L.g.nelx) % L.g.nely, ek = e / (L.g.nelx * L.g.nely);
            bsm[L.oE + e] = L.E32[ei + (long long)L.pex * (ej + (long long)L.g.nely * ek)];
        }
    }
    __syncthreads();

    // t = K z on level li
    auto op = [&](int li) {
        const BottomLevel& L = a.L[li];
        const int nn = (int)L.g.nnode, nel = (int)L.g.nel;
        const float* z = bsm + L.oz;
        float* t = bsm + L.ot;
        for (int i = tid; i < 3 * nn; i += nt) t[i] = 0.f;
        __syncthreads();
        if (8 * nel <= nt) bottom_op_items<8>(L.g, Ks, z, t, bsm + L.oE, tid, nt);
        else if (4 * nel <= nt) bottom_op_items<4>(L.g, Ks, z, t, bsm + L.oE, tid, nt);
        else if (2 * nel <= nt) bottom_op_items<2>(L.g, Ks, z, t, bsm + L.oE, tid, nt);
        else bottom_op_items<1>(L.g, Ks, z, t, bsm + L.oE, tid, nt);
        __syncthreads();
    };
    // z = d b (first sweep from 0) or z += d (b - t)
    auto smooth = [&](int li, bool first) {
        const BottomLevel& L = a.L[li];
        const int nn = (int)L.g.nnode;
        const float* d = bsm + L.od;
        const float* b = bsm + L.ob;
        const float* t = bsm + L.ot;
        float* z = bsm + L.oz;
        for (int i = tid; i < 3 * nn; i += nt) {
            const int n = i / 3, c = i - 3 * n;
            if ((bytes[L.om + n] >> c) & 1) z[i] = 0.f;
            else z[i] = first ? d[n] * b[i] : fmaf(d[n], b[i] - t[i], z[i]);
        }
        __syncthreads();
    };
    // b_{li+1} = R (b_li - t_li); the 27 points unrolled (bounds as predicates)
    auto restrict_to = [&](int li) {
        const BottomLevel& F = a.L[li];
        const BottomLevel& C = a.L[li + 1];
        const int nc = (int)C.g.nnode;
        for (int n = tid; n < nc; n += nt) {
            const int i = n % C.g.nx, j = (n / C.g.nx) % C.g.ny, k = n / (C.g.nx * C.g.ny);
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int dk = -1; dk <= 1; ++dk) {
                const int fk = 2 * k + dk;
                const bool okk = fk >= 0 && fk < F.g.nz;
#pragma unroll
                for (int dj = -1; dj <= 1; ++dj) {
                    const int fj = 2 * j + dj;
                    const bool okj = okk && fj >= 0 && fj < F.g.ny;
#pragma unroll
                    for (int di = -1; di <= 1; ++di) {
                        const int fi = 2 * i + di;
                        if (!(okj && fi >= 0 && fi < F.g.nx)) continue;
                        const float wt = (dk ? 0.5f : 1.f) * (dj ? 0.5f : 1.f) * (di ? 0.5f : 1.f);
                        const int f = fi + F.g.nx * (fj + F.g.ny * fk);
                        const uint8_t m = bytes[F.om + f];
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float v = bsm[F.ob + 3 * f + c] - bsm[F.ot + 3 * f + c];
                            acc[c] = fmaf(((m >> c) & 1) ? 0.f : wt, v, acc[c]);
                        }
                    }
                }
            }
            const uint8_t mc = bytes[C.om + n];
#pragma unroll
            for (int c = 0; c < 3; ++c) bsm[C.ob + 3 * n + c] = ((mc >> c) & 1) ? 0.f : acc[c];
        }
        __syncthreads();
    };
    // z_li += P z_{li+1}; the eight candidates unrolled (predicates)
    auto prolong_from = [&](int li) {
        const BottomLevel& F = a.L[li];
        const BottomLevel& C = a.L[li + 1];
        const int nf = (int)F.g.nnode;
        for (int n = tid; n < nf; n += nt) {
            const int i = n % F.g.nx, j = (n / F.g.nx) % F.g.ny, k = n / (F.g.nx * F.g.ny);
            const bool ox = i & 1, oy = j & 1, oz = k & 1;
            const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f) * (oz ? 0.5f : 1.f);
            const int c0 = (i >> 1) + C.g.nx * ((j >> 1) + C.g.ny * (k >> 1));
            float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int aa = 0; aa < 2; ++aa)
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc) {
                        if ((cc && !ox) || (bb && !oy) || (aa && !oz)) continue;
                        const int cn = c0 + cc + C.g.nx * (bb + C.g.ny * aa);
#pragma unroll
                        for (int c = 0; c < 3; ++c) acc[c] = fmaf(w, bsm[C.oz + 3 * cn + c], acc[c]);
                    }
            const uint8_t m = bytes[F.om + n];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                if (!((m >> c) & 1)) bsm[F.oz + 3 * n + c] += acc[c];
        }
        __syncthreads();
    };

    const int last = a.nb - 1;
    for (int li = 0; li < last; ++li) {
        smooth(li, true);
        for (int s = 1; s < a.nu; ++s) {
            op(li);
            smooth(li, false);
        }
        op(li);
        restrict_to(li);
    }
    smooth(last, true);
    for (int s = 1; s < a.sweeps; ++s) {
        op(last);
        smooth(last, false);
    }
    for (int li = last - 1; li >= 0; --li) {
        prolong_from(li);
        for (int s = 0; s < a.nu; ++s) {
            op(li);
            smooth(li, false);
        }
    }
    const BottomLevel& L0 = a.L[0];
    for (int n = tid; n < (int)L0.g.nnode; n += nt) {
        const int i = n % L0.g.nx, jk = n / L0.g.nx;
        const long long p = i + (long long)L0.px * jk;
#pragma unroll
        for (int c = 0; c < 3; ++c) a.z_out[c * L0.vol + p] = bsm[L0.oz + 3 * n + c];
    }
}

// Residual replacement that keeps the inner CG's direction: r32 = scale r64
// (masked), d = 0; |r32|^2 against the next segment's target; the next
// beta is Fletcher-Reeves.
__global__ void k_pcg_replace(const Grid g, int px, long long vol, const double* __restrict__ r64,
                              double scale, const uint8_t* __restrict__ nodemask, float* __restrict__ r32,
                              float* __restrict__ d32, const Reducer red, SolverScalars* ss, double delta2,
                              double target2) {
    __shared__ double sh[32];
    __shared__ double out[1];
    double rr = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < g.nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const long long p = (n % g.nx) + (long long)px * (n / g.nx);
        const uint8_t m = nodemask[n];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = ((m >> c) & 1) ? 0.f : (float)(r64[3 * n + c] * scale);
            r32[c * vol + p] = v;
            d32[c * vol + p] = 0.f;
            rr = fma((double)v, (double)v, rr);
        }
    }
    double v[1] = {rr};
    if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) {
        ss->rr = out[0];
        ss->pad1 = 1;
        ss->it = 0;
        ss->done = 0;
        ss->tol2 = fmax(delta2 * out[0], target2);
        if (!isfinite(out[0])) {
            ss->status = TO3D_ENUMERIC;
            ss->done = 1;
        } else if (out[0] <= ss->tol2) {
            ss->done = 1;
        }
    }
}

static unsigned nblocks(long long n) {
    long long b = (n + kThreads - 1) / kThreads;
    if (b > 152 * 8) b = 152 * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace mg

using namespace mg;

static Mg* mg_of(to3d_ctx* c) { return (Mg*)c->mg; }

void destroy_mg(to3d_ctx* c) {
    Mg* m = mg_of(c);
    if (!m) return;
    if (m->cycle) cudaGraphExecDestroy(m->cycle);
    if (m->pcg) cudaGraphExecDestroy(m->pcg);
    for (size_t l = 0; l < m->lv.size(); ++l) {
        cudaFree(m->lv[l].z);
        cudaFree(m->lv[l].t);
        if (l > 0) to3d_destroy(m->lv[l].ctx);
    }
    for (auto& s : m->snaps) cudaFree(s.r);
    for (double* x : m->designs) cudaFree(x);
    void* ptrs[] = {m->wdev, m->lamdev, m->z64, m->rprev, m->dots, m->ones, m->ke32};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (m->dots_h) cudaFreeHost(m->dots_h);
    delete m;
    c->mg = nullptr;
}

// Build the level hierarchy once per context (coarse contexts, buffers, maps).
static to3d_status ensure_mg(to3d_ctx* c) {
    if (c->mg) return TO3D_OK;
    if (c->g.ny > 65535 || c->g.nz > 65535)
        return set_err(c, TO3D_EINVAL, "multigrid: more than 65535 nodes along y or z");
    Mg* m = new (std::nothrow) Mg();
    if (!m) return set_err(c, TO3D_ENOMEM, "multigrid");
    c->mg = m;
    default_theta(m->theta);
    m->sweeps = c->prm.mg_sweeps > 0 ? c->prm.mg_sweeps : 6;
    m->nu = c->prm.mg_nu > 0 ? c->prm.mg_nu : 1;
    m->prec = c->prm.precision == TO3D_F64 ? TO3D_BF16_DC : c->prm.precision;
    // clamp masks on the host, level by level
    const Grid& g0 = c->g;
    std::vector<uint8_t> mask(g0.nnode);
    MG_CK(cudaMemcpy(mask.data(), c->nodemask, g0.nnode, cudaMemcpyDeviceToHost));
    Level L0;
    L0.ctx = c;
    m->lv.push_back(L0);
    int dims[3] = {g0.nelx, g0.nely, g0.nelz};
    while ((int)m->lv.size() < kMaxLevels &&
           std::max(dims[0], std::max(dims[1], dims[2])) > 4 &&
           std::min(dims[0], std::min(dims[1], dims[2])) >= 2) {
        const int fx = dims[0] + 1, fy = dims[1] + 1, fz = dims[2] + 1;
        int cd[3] = {(dims[0] + 1) / 2, (dims[1] + 1) / 2, (dims[2] + 1) / 2};
        const int cx = cd[0] + 1, cy = cd[1] + 1, cz = cd[2] + 1;
        std::vector<uint8_t> fixed(3LL * cx * cy * cz, 0), cmask((size_t)cx * cy * cz, 0);
        for (int k = 0; k < cz; ++k)
            for (int j = 0; j < cy; ++j)
                for (int i = 0; i < cx; ++i) {
                    if (2 * i >= fx || 2 * j >= fy || 2 * k >= fz) continue;
                    const uint8_t fm = mask[(size_t)(2 * i) + (size_t)fx * ((size_t)(2 * j) + (size_t)fy * (2 * k))];
                    const size_t n = i + (size_t)cx * (j + (size_t)cy * k);
                    cmask[n] = fm;
                    for (int cc = 0; cc < 3; ++cc) fixed[3 * n + cc] = (fm >> cc) & 1;
                }
        std::vector<double> load(fixed.size(), 0.0);
        to3d_params p = c->prm;
        p.nelx = cd[0];
        p.nely = cd[1];
        p.nelz = cd[2];
        p.precond = TO3D_JACOBI;
        p.filter = TO3D_FILTER_SENS;
        p.precision = m->prec;
        p.rmin = 1.5;
        Level Lc;
        to3d_status st = to3d_create(&p, fixed.data(), load.data(), nullptr, c->stream, &Lc.ctx);
        if (st) return set_err(c, st, "multigrid coarse level");
        m->lv.push_back(Lc);
        mask.swap(cmask);
        dims[0] = cd[0];
        dims[1] = cd[1];
        dims[2] = cd[2];
    }
    for (auto& L : m->lv) {
        const size_t bytes = sizeof(float) * 3 * L.ctx->vol;
        MG_CK(cudaMalloc(&L.z, bytes));
        MG_CK(cudaMalloc(&L.t, bytes));
        MG_CK(cudaMemset(L.z, 0, bytes));
        MG_CK(cudaMemset(L.t, 0, bytes));
        if (!encode_vec_map(L.ctx, &L.tm_z, L.z, 3)) return set_err(c, TO3D_ECUDA, "multigrid TMA map");
    }
    // the bottom levels that fit in one CTA's shared memory together
    {
        const int L = (int)m->lv.size();
        long long used = 576 * 4;
        int lb = L;
        for (int l = L - 1; l >= 0 && L - l <= kBottomMaxLevels; --l) {
            const Grid& g = m->lv[l].ctx->g;
            const long long need = 4 * (10 * g.nnode + g.nel) + g.nnode + 16;
            if (used + need > kBottomSmem) break;
            used += need;
            lb = l;
        }
        if (lb < L) {
            BottomArgs& ba = m->bottom;
            std::memset(&ba, 0, sizeof(ba));
            ba.nb = L - lb;
            ba.lb = lb;
            ba.sweeps = m->sweeps;
            ba.nu = m->nu;
            int off = 576;
            for (int i = 0; i < ba.nb; ++i) {
                to3d_ctx* k = m->lv[lb + i].ctx;
                BottomLevel& B = ba.L[i];
                B.g = k->g;
                B.px = k->px;
                B.pex = k->pex;
                B.vol = k->vol;
                B.E32 = k->E32;
                B.dinv32 = k->dinv32;
                B.maskp = k->maskp;
                const int n = (int)k->g.nnode;
                B.ob = off; off += 3 * n;
                B.oz = off; off += 3 * n;
                B.ot = off; off += 3 * n;
                B.od = off; off += n;
                B.oE = off; off += (int)k->g.nel;
            }
            int boff = 4 * off;
            for (int i = 0; i < ba.nb; ++i) {
                ba.L[i].om = boff;
                boff += (int)ba.L[i].g.nnode;
            }
            m->bottom_smem = (boff + 15) & ~15;
            m->lb = lb;
            MG_CK(cudaFuncSetAttribute(k_cycle_bottom, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kBottomSmem));
        }
    }
    // z-segment length of the tensor-core kernel per launched level (the
    // coarse grids are small: shorter segments give more CTAs)
    for (int l = 0; l < m->lb && l < (int)m->lv.size(); ++l)
        MG_CK(tune_tc_lz(m->lv[l].ctx, m->prec, m->lv[l].tm_z, m->lv[l].t, false));
    const long long ndof = 3 * g0.nnode;
    MG_CK(cudaMalloc(&m->wdev, sizeof(float) * kMaxLevels));
    MG_CK(cudaMalloc(&m->lamdev, sizeof(double) * kMaxLevels));
    {
        float ke[576];
        for (int i = 0; i < 576; ++i) ke[i] = (float)c->ke.v[i];
        MG_CK(cudaMalloc(&m->ke32, sizeof(ke)));
        MG_CK(cudaMemcpy(m->ke32, ke, sizeof(ke), cudaMemcpyHostToDevice));
        m->bottom.KE = m->ke32;
        m->bottom.wdev = m->wdev;
    }
    {
        double l1 = 0.0;
        for (int a = 0; a < 24; ++a) {
            double row = 0.0;
            for (int b = 0; b < 24; ++b) row += std::fabs(c->ke.v[a * 24 + b]);
            l1 = std::fmax(l1, row / c->ke.v[a * 24 + a]);
        }
        m->l1 = l1;
    }
    MG_CK(cudaMalloc(&m->z64, sizeof(double) * ndof));
    MG_CK(cudaMalloc(&m->rprev, sizeof(double) * ndof));
    MG_CK(cudaMalloc(&m->dots, sizeof(double) * 4));
    MG_CK(cudaMallocHost(&m->dots_h, sizeof(double) * 4));
    MG_CK(cudaMalloc(&m->ones, sizeof(float) * c->vol));
    k_fill<<<nblocks(c->vol), kThreads, 0, c->stream>>>(c->vol, 1.f, m->ones);
    if (!encode_vec_map(c, &m->tm_ones, m->ones, 1)) return set_err(c, TO3D_ECUDA, "multigrid TMA map");
    MG_CK(cudaStreamSynchronize(c->stream));
    m->params_dirty = true;
    return TO3D_OK;
}

// Coarse moduli, diagonals and smoothing weights for the fine moduli c->E
// (c->dinv32 must already belong to them).
// The set-up's launches on stream s (capturable: the batched engine puts
// them into its per-problem OC-iteration graph).
static void setup_levels_on(to3d_ctx* c, cudaStream_t s) {
    Mg* m = mg_of(c);
    for (size_t l = 1; l < m->lv.size(); ++l) {
        to3d_ctx* f = m->lv[l - 1].ctx;
        to3d_ctx* k = m->lv[l].ctx;
        k_coarsen<<<(unsigned)((k->g.nel + kThreads - 1) / kThreads), kThreads, 0, s>>>(
            f->g, f->E, k->g, q_of(m, (int)l), s_of(m, (int)l), k->E, k->E32, k->pex);
        launch_diag(k, s, k->E);
        c->launches += 2;
    }
    // damping of every level from its eigenvalue bound
    for (size_t l = 0; l < m->lv.size(); ++l) {
        Level& L = m->lv[l];
        to3d_ctx* k = L.ctx;
        double* out = k->misc + 4;
        k_pow_start<<<nblocks(k->vol), kThreads, 0, s>>>(k->g, k->px, k->vol, k->dinv32, k->maskp, L.z);
        for (int it = 0; it < kPowerSteps; ++it) {
            launch_matvec_tc_io(k, s, m->prec, false, k->tm_r, L.tm_z, k->tm_d, nullptr, L.t, nullptr);
            k_pow_dots<<<nblocks(k->vol / 4), 256, 0, s>>>(k->vol, L.z, L.t, k->dinv32, k->maskp, k->red, out);
            if (it + 1 < kPowerSteps)
                k_pow_next<<<nblocks(k->vol), kThreads, 0, s>>>(k->vol, L.t, k->dinv32, k->maskp, out, L.z);
        }
        k_pow_final<<<1, 1, 0, s>>>(out, w_of(m, (int)l), kPowerMargin, m->l1, m->wdev, (int)l, m->lamdev);
        c->launches += 2 + 3 * kPowerSteps;
    }
}

static to3d_status setup_levels(to3d_ctx* c) {
    Mg* m = mg_of(c);
    setup_levels_on(c, c->stream);
    m->params_dirty = false;
    return launch_check(c, "multigrid set-up");
}

// One V-cycle from level l: b (padded SoA of level l) -> lv[l].z.
// fuse_dots (level 0 of the inner MG-PCG only): the last sweep also forms
// r.z, z.q_old and beta (k_jacobi_dots), so no separate k_pcg_dots.
static void cycle_launch(to3d_ctx* c, Mg* m, cudaStream_t s, size_t l, const float* b,
                         SolverScalars* ss, bool fuse_dots = false) {
    Level& L = m->lv[l];
    to3d_ctx* k = L.ctx;
    const long long vol = k->vol;
    auto op = [&]() {
        launch_matvec_tc_io(k, s, m->prec, false, k->tm_r, L.tm_z, k->tm_d, nullptr, L.t, ss);
        if (k != c) c->launches++;
    };
    if ((int)l == m->lb) {
        // levels lb..L in one CTA
        BottomArgs ba = m->bottom;
        ba.b_in = b;
        ba.z_out = L.z;
        k_cycle_bottom<<<1, kBottomThreads, m->bottom_smem, s>>>(ba, ss);
        c->launches++;
        return;
    }
    k_jacobi0<<<nblocks(vol), kThreads, 0, s>>>(vol, b, k->dinv32, k->maskp, m->wdev, (int)l, L.z, ss);
    c->launches++;
    if (l + 1 == m->lv.size()) {
        for (int i = 1; i < m->sweeps; ++i) {
            op();
            k_jacobi<<<nblocks(vol), kThreads, 0, s>>>(vol, b, L.t, k->dinv32, k->maskp, m->wdev, (int)l,
                                                      L.z, ss);
            c->launches++;
        }
        return;
    }
    Level& C = m->lv[l + 1];
    to3d_ctx* kc = C.ctx;
    auto sweep = [&]() {
        op();
        k_jacobi<<<nblocks(vol), kThreads, 0, s>>>(vol, b, L.t, k->dinv32, k->maskp, m->wdev, (int)l,
                                                  L.z, ss);
        c->launches++;
    };
    for (int i = 1; i < m->nu; ++i) sweep();     // further pre-smoothing sweeps
    op();
    k_restrict<<<dim3((kc->g.nx + 63) / 64, kc->g.ny, kc->g.nz), 64, 0, s>>>(
        k->g, k->px, vol, b, L.t, k->maskp, kc->g, kc->px, kc->vol, kc->maskp, kc->r32, ss);
    c->launches++;
    cycle_launch(c, m, s, l + 1, kc->r32, ss);
    if (k->g.nnode >= (1LL << 22))
        k_prolong_col<<<dim3((kc->g.nx + kColX - 1) / kColX, (kc->g.ny + kColY - 1) / kColY, kc->g.nz),
                        dim3(kColX, kColY), 0, s>>>(k->g, k->px, vol, k->maskp, L.z, kc->g, kc->px,
                                                    kc->vol, C.z, ss);
    else
        k_prolong<<<dim3((k->g.nx + 127) / 128, k->g.ny, k->g.nz), 128, 0, s>>>(
            k->g, k->px, vol, k->maskp, L.z, kc->g, kc->px, kc->vol, C.z, ss);
    c->launches++;
    for (int i = 0; i < m->nu; ++i) {             // post-smoothing
        if (fuse_dots && i + 1 == m->nu) {
            op();
            k_jacobi_dots<<<nblocks(vol / 4), 256, 0, s>>>(vol, b, L.t, k->dinv32, k->maskp, m->wdev,
                                                          L.z, c->q32, c->red, ss);
            c->launches++;
        } else {
            sweep();
        }
    }
}

// Make sure the hierarchy belongs to the current fine operator.
static to3d_status ready(to3d_ctx* c) {
    to3d_status st = ensure_mg(c);
    if (st) return st;
    Mg* m = mg_of(c);
    if (m->params_dirty) return setup_levels(c);
    return TO3D_OK;
}

// Mark the hierarchy stale (the fine moduli changed).
void mg_operator_changed(to3d_ctx* c) {
    Mg* m = mg_of(c);
    if (m) m->params_dirty = true;
}

// z = V r for FP64 AoS vectors (r unscaled); uses ctx->r32 as the cycle input.
to3d_status mg_apply64(to3d_ctx* c, const double* r, double* z, double rnorm) {
    to3d_status st = ready(c);
    if (st) return st;
    Mg* m = mg_of(c);
    cudaStream_t s = c->stream;
    const double ndof = 3.0 * (double)c->g.nnode;
    const double scale = rnorm > 0.0 ? std::sqrt(ndof) / rnorm : 1.0;
    k_in<<<nblocks(c->g.nnode), kThreads, 0, s>>>(c->g, c->px, c->vol, r, scale, c->nodemask, c->r32);
    c->launches++;
    if (!m->cycle) {
        cudaGraph_t gr;
        MG_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c->launches;
        cycle_launch(c, m, c->cap_stream, 0, c->r32, nullptr);
        MG_CK(cudaStreamEndCapture(c->cap_stream, &gr));
        MG_CK(cudaGraphInstantiate(&m->cycle, gr, 0));
        cudaGraphDestroy(gr);
        m->cycle_launches = c->launches - l0;
        c->launches = l0;
    }
    MG_CK(cudaGraphLaunch(m->cycle, s));
    c->launches += m->cycle_launches;
    k_out<<<nblocks(c->g.nnode), kThreads, 0, s>>>(c->g, c->px, c->vol, m->lv[0].z, 1.0 / scale, z);
    c->launches++;
    return launch_check(c, "multigrid cycle");
}

}  // namespace to3d

// ------------------------------------------------------------------ inner MG-PCG
namespace to3d {

// One inner iteration: z = V r (cycle on ctx->r32), rz and beta, the fused
// tensor-core kernel p_new = z + beta p_old, q = K p_new, alpha = rz / p.q,
// then d += alpha p_new, r -= alpha q and |r|^2 (no Jacobi dot).
// ev0/ev1 (may be null): external events recorded around the fused kernel.
static void mgpcg_iter(to3d_ctx* c, Mg* m, cudaStream_t s, int prec, int parity,
                       cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr) {
    // with level 0 above the one-CTA bottom cycle the dots ride on its last
    // sweep; otherwise a separate pass
    const bool fused = m->lb > 0;
    cycle_launch(c, m, s, 0, c->r32, c->ss, fused);
    if (!fused) {
        k_pcg_dots<<<nblocks(3 * c->vol), kThreads, 0, s>>>(c->vol, c->r32, m->lv[0].z, c->q32,
                                                            c->red, c->ss);
        c->launches++;
    }
    float* p_new = parity ? c->p32b : c->p32a;
    const CUtensorMap& tp = parity ? c->tm_pa : c->tm_pb;
    if (ev0) cudaEventRecordWithFlags(ev0, s, cudaEventRecordExternal);
    launch_matvec_tc_io(c, s, prec, true, m->lv[0].tm_z, tp, m->tm_ones, p_new, c->q32, c->ss);
    if (ev1) cudaEventRecordWithFlags(ev1, s, cudaEventRecordExternal);
    launch_pcg32_update_mode(c, s, p_new, 0);
}

// Inner iterations per captured chunk (even, so the direction ping-pong stays
// in phase across chunks).
constexpr int kMgChunk = 8;

static to3d_status mgpcg_chunk(to3d_ctx* c, Mg* m, int prec, int n) {
    if (n == kMgChunk) {
        if (!m->pcg || m->pcg_prec != prec) {
            if (m->pcg) cudaGraphExecDestroy(m->pcg);
            m->pcg = nullptr;
            cudaGraph_t gr;
            const long long l0 = c->launches;
            MG_CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
            c->kslots[0] = 0;
            for (int i = 0; i < n; ++i) {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                if (i % 4 == 0 && c->kslots[0] < to3d_ctx::kTimedSlots) {
                    const int sl = c->kslots[0]++;
                    e0 = c->kev[0][2 * sl];
                    e1 = c->kev[0][2 * sl + 1];
                    c->kslot_iter[0][sl] = i;
                }
                mgpcg_iter(c, m, c->cap_stream, prec, i & 1, e0, e1);
            }
            MG_CK(cudaStreamEndCapture(c->cap_stream, &gr));
            MG_CK(cudaGraphInstantiate(&m->pcg, gr, 0));
            cudaGraphDestroy(gr);
            m->pcg_prec = prec;
            m->pcg_n = (int)(c->launches - l0);
            c->launches = l0;
        }
        MG_CK(cudaGraphLaunch(m->pcg, c->stream));
        c->launches += m->pcg_n;
    } else {
        for (int i = 0; i < n; ++i) mgpcg_iter(c, m, c->stream, prec, i & 1);
    }
    return launch_check(c, "multigrid PCG chunk");
}

// FP64 defect correction around an FP32 inner CG preconditioned by the
// cycle: each segment scales the true residual to unit RMS, runs the inner
// CG until its residual has dropped by inner_rtol (or the global target is
// met), adds the correction to u in FP64 and recomputes f - K u in FP64.
// The inner CG restarts at every segment (the cycle makes that cheap).
to3d_status solve_dc_mg(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    to3d_status st = ready(c);
    if (st) return st;
    Mg* m = mg_of(c);
    const double tol = c->prm.cg_rtol;
    const double delta = c->prm.inner_rtol;
    const int prec = c->prm.precision == TO3D_F64 ? TO3D_BF16_DC : c->prm.precision;
    const long long ndof = 3 * c->g.nnode;
    int total = 0, outer = 0, status = TO3D_OK, stalls = 0;
    double relres = 0.0;
    if ((st = true_residual64(c, f, fnorm, &relres))) return st;
    // keep: one inner CG across the replacements (scale fixed by the first
    // residual); else each segment restarts at unit RMS
    const bool keep = c->prm.mg_keep_dir != 0;
    double scale = 0.0;
    bool restart = true;
    int last_its = 0;
    while (relres > tol && fnorm > 0.0) {
        const double rnorm = relres * fnorm;
        if (!keep || scale == 0.0) scale = std::sqrt((double)ndof) / rnorm;
        const double t = 0.5 * tol * fnorm * scale;
        if (restart) {
            launch_ss_reset(c, c->stream, std::fmax(delta * delta * (double)ndof, t * t),
                            c->prm.cg_maxit - total);
            k_pcg_init<<<nblocks(c->g.nnode), kThreads, 0, c->stream>>>(
                c->g, c->px, c->vol, c->r, scale, c->nodemask, c->r32, c->d32, c->p32b, c->q32, c->red,
                c->ss);
        } else {
            // the captured chunks take p_old from p32b first: after an odd
            // number of iterations the last direction sits in p32a
            if (last_its & 1)
                MG_CK(cudaMemcpyAsync(c->p32b, c->p32a, sizeof(float) * 3 * c->vol,
                                      cudaMemcpyDeviceToDevice, c->stream));
            launch_ss_segment(c, c->stream, t * t, c->prm.cg_maxit - total);
            k_pcg_replace<<<nblocks(c->g.nnode), kThreads, 0, c->stream>>>(
                c->g, c->px, c->vol, c->r, scale, c->nodemask, c->r32, c->d32, c->red, c->ss,
                delta * delta, t * t);
        }
        c->launches++;
        int it0 = 0, chunks = 0;
        const auto seg_t0 = std::chrono::steady_clock::now();
        for (;;) {
            ++chunks;
            if ((st = mgpcg_chunk(c, m, prec, kMgChunk))) return st;
            if ((st = sync_solver_scalars(c))) return st;
            accumulate_tc_times(c, it0, c->ss_h->it);
            it0 = c->ss_h->it;
            if (c->ss_h->done) break;
        }
        const int its = c->ss_h->it;
        total += its;
        last_its = its;
        if (c->ss_h->status == TO3D_ETIMEOUT || c->ss_h->status == TO3D_ENUMERIC) {
            status = c->ss_h->status;
            break;
        }
        launch_axpy_d32(c, c->stream, 1.0 / scale);
        const double prev = relres;
        if ((st = true_residual64(c, f, fnorm, &relres))) return st;
        // keep the direction unless the true residual failed to halve (the
        // recurrence ran away from it): then restart from it
        restart = !keep || relres > 0.5 * prev;
        if (restart) scale = 0.0;
        if (c->trace) {
            const double seg_ms =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - seg_t0).count();
            std::fprintf(stderr,
                         "to3d: mg segment %d: %d inner its in %d chunks (total %d), relres %.3e -> %.3e, "
                         "%.2f ms wall (host, incl. the FP64 residual)\n",
                         outer, its, chunks, total, prev, relres, seg_ms);
        }
        if (relres <= tol) break;
        ++outer;
        if (total >= c->prm.cg_maxit || outer >= 1000) {
            status = TO3D_ENOCONV;
            break;
        }
        if (relres > 0.5 * prev && ++stalls > 20) {
            status = TO3D_ENOCONV;
            break;
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

// Pieces for the batched engine's captured OC-iteration graph.
to3d_status mg_capture_ready(to3d_ctx* c) { return ensure_mg(c); }
void mg_setup_launch(to3d_ctx* c, cudaStream_t s) { setup_levels_on(c, s); }
void mg_pcg_iter_launch(to3d_ctx* c, cudaStream_t s, int prec, int parity) {
    mgpcg_iter(c, mg_of(c), s, prec, parity);
}

// Buffers and preconditioner of flexible CG with the cycle.
static to3d_status mg_apply_fcg(to3d_ctx* c, const double* r, double* z, double rr) {
    return mg_apply64(c, r, z, std::sqrt(rr));
}

to3d_status mg_fcg_io(to3d_ctx* c, FcgIO* io) {
    to3d_status st = ready(c);
    if (st) return st;
    Mg* m = mg_of(c);
    io->z = m->z64;
    io->rprev = m->rprev;
    io->dots = m->dots;
    io->dots_h = m->dots_h;
    io->apply = mg_apply_fcg;
    return TO3D_OK;
}

// ------------------------------------------------------------------ training
// Loss of the current parameters over the snapshots (mean energy-norm error
// of one application, FP64 operator and dots).
static to3d_status snapshot_loss(to3d_ctx* c, double* loss) {
    Mg* m = mg_of(c);
    cudaStream_t s = c->stream;
    const long long ndof = 3 * c->g.nnode;
    to3d_status st;
    double sum = 0.0;
    int cur = -1;
    for (auto& sn : m->snaps) {      // grouped by design (appended design by design)
        if (sn.design != cur) {
            // the operator of this snapshot's design, and the hierarchy for
            // it with the current parameters
            cur = sn.design;
            if ((st = prepare_op(c, m->designs[cur]))) return st;
            if ((st = ready(c))) return st;
        }
        if ((st = mg_apply64(c, sn.r, m->z64, sn.rn))) return st;
        // z is 0 on clamped dofs, where the FP64 operator has identity rows
        launch_matvec64(c, s, c->E, m->z64, c->tmp, false);
        launch_dots64(c, s, ndof, m->z64, c->tmp, m->z64, sn.r, m->dots);
        MG_CK(cudaMemcpyAsync(m->dots_h, m->dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        MG_CK(cudaStreamSynchronize(s));
        const double zkz = m->dots_h[0], zr = m->dots_h[1];
        sum += (zkz - 2.0 * zr + sn.rte) / sn.rte;
    }
    *loss = m->snaps.empty() ? 0.0 : sum / (double)m->snaps.size();
    if (!std::isfinite(*loss)) *loss = 1e30;
    return TO3D_OK;
}

static unsigned long long splitmix(unsigned long long& x) {
    unsigned long long z = (x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// Parameters <-> unconstrained coordinates: w = 0.05 + 0.9 sigmoid(a),
// q = exp(b) in [0.125, 8], s = exp(c) in (0, 64].
static void to_free(const double* th, double* u) {
    for (int g = 0; g < kGroups; ++g) {
        const double y = (th[g] - 0.05) / 0.9;
        u[g] = std::log(y / (1.0 - y));
    }
    for (int i = kGroups; i < kParams; ++i) u[i] = std::log(th[i]);
}
static void from_free(const double* u, double* th) {
    for (int g = 0; g < kGroups; ++g) th[g] = 0.05 + 0.9 / (1.0 + std::exp(-u[g]));
    for (int i = kGroups; i < 2 * kGroups - 1; ++i) th[i] = std::fmin(8.0, std::fmax(0.125, std::exp(u[i])));
    for (int i = 2 * kGroups - 1; i < kParams; ++i) th[i] = std::fmin(64.0, std::exp(u[i]));
}

}  // namespace to3d

using namespace to3d;

extern "C" {

to3d_status to3d_mg_param_count(to3d_ctx* c, int64_t* n) {
    if (!c || !n) return TO3D_EINVAL;
    *n = kParams;
    return TO3D_OK;
}

to3d_status to3d_mg_get_params(to3d_ctx* c, double* theta, int64_t n) {
    if (!c || !theta || n != kParams) return TO3D_EINVAL;
    to3d_status st = ensure_mg(c);
    if (st) return st;
    std::memcpy(theta, mg_of(c)->theta, sizeof(double) * kParams);
    return TO3D_OK;
}

to3d_status to3d_mg_set_params(to3d_ctx* c, const double* theta, int64_t n) {
    if (!c || !theta || n != kParams) return TO3D_EINVAL;
    if (!theta_valid(theta)) return set_err(c, TO3D_EINVAL, "multigrid parameters out of range");
    to3d_status st = ensure_mg(c);
    if (st) return st;
    Mg* m = mg_of(c);
    std::memcpy(m->theta, theta, sizeof(double) * kParams);
    m->params_dirty = true;
    m->trained = true;
    return TO3D_OK;
}

to3d_status mg_set_params_ctx(to3d_ctx* c, const double* theta, int64_t n) {
    return to3d_mg_set_params(c, theta, n);
}

to3d_status to3d_mg_levels(to3d_ctx* c, int32_t* nlev) {
    if (!c || !nlev) return TO3D_EINVAL;
    to3d_status st = ensure_mg(c);
    if (st) return st;
    *nlev = (int32_t)mg_of(c)->lv.size();
    return TO3D_OK;
}

to3d_status to3d_mg_apply(to3d_ctx* c, const double* x, const double* r, double* z, int32_t on_device) {
    if (!c || !x || !r || !z) return TO3D_EINVAL;
    const long long ndof = 3 * c->g.nnode;
    const void *dx = nullptr, *dr = nullptr;
    to3d_status st;
    if ((st = stage_input(c, x, sizeof(double) * c->g.nel, on_device, 0, &dx))) return st;
    if ((st = stage_input(c, r, sizeof(double) * ndof, on_device, 1, &dr))) return st;
    if ((st = prepare_op(c, (const double*)dx))) return st;
    if ((st = ensure_mg(c))) return st;
    mg_of(c)->params_dirty = true;
    launch_norm2(c, c->stream, (const double*)dr, ndof, c->misc + 4);
    double rr = 0.0;
    MG_CK(cudaMemcpyAsync(&rr, c->misc + 4, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    MG_CK(cudaStreamSynchronize(c->stream));
    double* dz = on_device ? z : c->tmp;
    if ((st = mg_apply64(c, (const double*)dr, dz, std::sqrt(rr)))) return st;
    if (!on_device) MG_CK(cudaMemcpyAsync(z, dz, sizeof(double) * ndof, cudaMemcpyDeviceToHost, c->stream));
    MG_CK(cudaStreamSynchronize(c->stream));
    return launch_check(c, "mg apply");
}

// Snapshots from the context's current design: residuals of FP64 Jacobi-PCG
// from u = 0 after a random number (0..maxk) of iterations, with r^T K^-1 r
// from an FP64 solve of K e = r to 1e-10; then `steps` Adam steps on
// central-difference gradients of the mean loss.
to3d_status to3d_mg_train(to3d_ctx* c, int32_t nsnap, int32_t steps, double lr, uint64_t seed,
                          int32_t append, double* loss_first, double* loss_last) {
    if (!c || nsnap < 0 || nsnap > 256 || steps < 0 || !(lr > 0) || !loss_first || !loss_last)
        return TO3D_EINVAL;
    to3d_status st = ensure_mg(c);
    if (st) return st;
    Mg* m = mg_of(c);
    cudaStream_t s = c->stream;
    const long long ndof = 3 * c->g.nnode;
    if (!append) {
        for (auto& sn : m->snaps) cudaFree(sn.r);
        m->snaps.clear();
        for (double* x : m->designs) cudaFree(x);
        m->designs.clear();
    }
    if (m->snaps.size() + (size_t)nsnap > 256)
        return set_err(c, TO3D_EINVAL, "more than 256 multigrid training snapshots");
    if (m->snaps.size() + (size_t)nsnap == 0) return set_err(c, TO3D_EINVAL, "no training snapshots");
    // the snapshots of earlier designs keep their own r^T K^-1 r; the loss
    // evaluates every snapshot with the operator of the current design, so
    // the training loop below needs the current design's operator prepared
    if ((st = prepare_op(c, c->x))) return st;
    const int di = (int)m->designs.size();
    if (nsnap > 0) {
        double* xd = nullptr;
        MG_CK(cudaMalloc(&xd, sizeof(double) * c->g.nel));
        MG_CK(cudaMemcpyAsync(xd, c->x, sizeof(double) * c->g.nel, cudaMemcpyDeviceToDevice, s));
        m->designs.push_back(xd);
    }
    unsigned long long rng = seed * 0x2545F4914F6CDD1DULL + 12345u + 977u * (unsigned long long)di;
    for (int i = 0; i < nsnap; ++i) {
        const int k = (int)(splitmix(rng) % 201ULL);
        Snap sn;
        sn.design = di;
        MG_CK(cudaMalloc(&sn.r, sizeof(double) * ndof));
        m->snaps.push_back(sn);
        if ((st = run_pcg64_iters(c, c->f, k))) return st;
        MG_CK(cudaMemcpyAsync(m->snaps.back().r, c->r, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
        launch_norm2(c, s, m->snaps.back().r, ndof, c->misc + 4);
        double rr = 0.0;
        MG_CK(cudaMemcpyAsync(&rr, c->misc + 4, sizeof(double), cudaMemcpyDeviceToHost, s));
        MG_CK(cudaStreamSynchronize(s));
        m->snaps.back().rn = std::sqrt(rr);
        to3d_solve_info si{};
        if ((st = solve64_rtol(c, m->snaps.back().r, std::sqrt(rr), 1e-10, &si))) return st;
        launch_dots64(c, s, ndof, m->snaps.back().r, c->u, nullptr, nullptr, m->dots);
        MG_CK(cudaMemcpyAsync(m->dots_h, m->dots, sizeof(double), cudaMemcpyDeviceToHost, s));
        MG_CK(cudaStreamSynchronize(s));
        m->snaps.back().rte = m->dots_h[0];
        if (!(m->snaps.back().rte > 0.0)) return set_err(c, TO3D_ENUMERIC, "snapshot r^T K^-1 r <= 0");
    }
    c->have_u = false;
    double u[kParams], mo[kParams] = {}, ve[kParams] = {}, gr[kParams], th[kParams];
    to_free(m->theta, u);
    double loss = 0.0;
    if ((st = snapshot_loss(c, &loss))) return st;
    *loss_first = loss;
    double best = loss;
    double best_th[kParams];
    std::memcpy(best_th, m->theta, sizeof(best_th));
    const double h = 0.05, b1 = 0.9, b2 = 0.999;
    for (int t = 1; t <= steps; ++t) {
        for (int i = 0; i < kParams; ++i) {
            double up[kParams], lp = 0.0, lm = 0.0;
            std::memcpy(up, u, sizeof(up));
            up[i] = u[i] + h;
            from_free(up, m->theta);
            if ((st = snapshot_loss(c, &lp))) return st;
            up[i] = u[i] - h;
            from_free(up, m->theta);
            if ((st = snapshot_loss(c, &lm))) return st;
            gr[i] = (std::fmin(lp, 1e3) - std::fmin(lm, 1e3)) / (2.0 * h);
        }
        for (int i = 0; i < kParams; ++i) {
            mo[i] = b1 * mo[i] + (1 - b1) * gr[i];
            ve[i] = b2 * ve[i] + (1 - b2) * gr[i] * gr[i];
            const double mh = mo[i] / (1 - std::pow(b1, t)), vh = ve[i] / (1 - std::pow(b2, t));
            u[i] -= lr * mh / (std::sqrt(vh) + 1e-12);
        }
        from_free(u, th);
        std::memcpy(m->theta, th, sizeof(th));
        if ((st = snapshot_loss(c, &loss))) return st;
        if (c->trace) std::fprintf(stderr, "to3d: mg train step %d loss %.5f\n", t, loss);
        if (loss < best) {
            best = loss;
            std::memcpy(best_th, th, sizeof(best_th));
        }
    }
    std::memcpy(m->theta, best_th, sizeof(best_th));
    m->params_dirty = true;
    m->trained = true;
    *loss_last = best;
    if ((st = prepare_op(c, c->x))) return st;
    return launch_check(c, "mg train");
}

}  // extern "C"
