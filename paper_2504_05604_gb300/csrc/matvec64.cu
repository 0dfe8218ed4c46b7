// FP64 matrix-free stiffness operator, Jacobi diagonal and SIMP moduli.
//
// Section 2.2 of the paper assembles K = sum_e E_e P_e^T KE P_e and solves
// K U = F.  Here K is never formed: y = K p is evaluated node by node,
//   y_n = sum_{e ni n} E_e KE[rows of n in e, :] p_e,
// from a shared-memory tile of p (tile nodes plus a one-node halo) and of E
// (tile elements plus halo).  Each node reads the 8 elements around it, so
// no atomics are needed and the result is deterministic.  KE rows are
// indexed with compile-time offsets and sit in the kernel-parameter constant
// bank, which lets every DFMA take its KE operand straight from there.
#include "internal.cuh"
#include "reduce.cuh"

namespace to3d {

constexpr int MV_TX = 32, MV_TY = 4, MV_TZ = 2;
constexpr int MV_PX = MV_TX + 2, MV_PY = MV_TY + 2, MV_PZ = MV_TZ + 2;   // node tile + halo
constexpr int MV_EX = MV_TX + 1, MV_EY = MV_TY + 1, MV_EZ = MV_TZ + 1;   // element tile

// Load the node tile (clamped dofs and out-of-grid nodes as zero) and the
// element tile (out-of-grid elements as zero modulus).
template <typename T, typename ET>
__device__ __forceinline__ void load_tiles(const Grid g, const T* __restrict__ p,
                                           const uint8_t* __restrict__ nodemask,
                                           const ET* __restrict__ E, int i0, int j0, int k0,
                                           T* sP, ET* sE) {
    const int t = flat_tid(), nt = flat_nthreads();
    constexpr int ROW = 3 * MV_PX;
    for (int idx = t; idx < ROW * MV_PY * MV_PZ; idx += nt) {
        const int o = idx % ROW, rj = (idx / ROW) % MV_PY, rk = idx / (ROW * MV_PY);
        const int li = o / 3, c = o % 3;
        const int gi = i0 - 1 + li, gj = j0 - 1 + rj, gk = k0 - 1 + rk;
        T v = T(0);
        if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny && gk >= 0 && gk < g.nz) {
            const long long n = node_id(g, gi, gj, gk);
            if (!((nodemask[n] >> c) & 1)) v = p[3 * n + c];
        }
        sP[idx] = v;
    }
    for (int idx = t; idx < MV_EX * MV_EY * MV_EZ; idx += nt) {
        const int li = idx % MV_EX, lj = (idx / MV_EX) % MV_EY, lk = idx / (MV_EX * MV_EY);
        const int gi = i0 - 1 + li, gj = j0 - 1 + lj, gk = k0 - 1 + lk;
        ET v = ET(0);
        if (gi >= 0 && gi < g.nelx && gj >= 0 && gj < g.nely && gk >= 0 && gk < g.nelz)
            v = E[elem_id(g, gi, gj, gk)];
        sE[idx] = v;
    }
}

__device__ __forceinline__ int ptile(int li, int lj, int lk, int c) {
    return 3 * (li + MV_PX * (lj + MV_PY * lk)) + c;
}

// Contribution of element at tile-offset (ex,ey,ez) around the thread's node.
template <int EX, int EY, int EZ>
__device__ __forceinline__ void node_elem(const KE64& ke, const double* sP, const double* sE,
                                          int tx, int ty, int tz, double& y0, double& y1,
                                          double& y2) {
    constexpr int a = (1 - EX) + 2 * (1 - EY) + 4 * (1 - EZ);   // node's local index in e
    const double Ee = sE[(tx + EX) + MV_EX * ((ty + EY) + MV_EY * (tz + EZ))];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const int bi = b & 1, bj = (b >> 1) & 1, bk = b >> 2;
        const int base = ptile(tx + EX + bi, ty + EY + bj, tz + EZ + bk, 0);
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            const double pv = sP[base + cc];
            s0 = fma(ke.v[(3 * a + 0) * 24 + 3 * b + cc], pv, s0);
            s1 = fma(ke.v[(3 * a + 1) * 24 + 3 * b + cc], pv, s1);
            s2 = fma(ke.v[(3 * a + 2) * 24 + 3 * b + cc], pv, s2);
        }
    }
    y0 = fma(Ee, s0, y0);
    y1 = fma(Ee, s1, y1);
    y2 = fma(Ee, s2, y2);
}

// y = Kbar p; optionally the grid sum p.y into ss->pq and alpha = rz / pq.
__global__ void __launch_bounds__(MV_TX* MV_TY* MV_TZ)
    k_matvec64(const __grid_constant__ KE64 ke, const Grid g, const double* __restrict__ E,
               const double* __restrict__ p, const uint8_t* __restrict__ nodemask,
               double* __restrict__ y, const Reducer red, SolverScalars* ss, int dot_pq) {
    if (dot_pq && ss->done) return;
    __shared__ double sP[3 * MV_PX * MV_PY * MV_PZ];
    __shared__ double sE[MV_EX * MV_EY * MV_EZ];
    __shared__ double sh[32];
    __shared__ double out[1];
    const int i0 = blockIdx.x * MV_TX, j0 = blockIdx.y * MV_TY, k0 = blockIdx.z * MV_TZ;
    load_tiles<double, double>(g, p, nodemask, E, i0, j0, k0, sP, sE);
    __syncthreads();
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    double y0 = 0.0, y1 = 0.0, y2 = 0.0;
    node_elem<0, 0, 0>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<1, 0, 0>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<0, 1, 0>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<1, 1, 0>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<0, 0, 1>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<1, 0, 1>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<0, 1, 1>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    node_elem<1, 1, 1>(ke, sP, sE, tx, ty, tz, y0, y1, y2);
    const int gi = i0 + tx, gj = j0 + ty, gk = k0 + tz;
    double dot = 0.0;
    if (gi < g.nx && gj < g.ny && gk < g.nz) {
        const long long n = node_id(g, gi, gj, gk);
        const uint8_t m = nodemask[n];
        const double* pn = p + 3 * n;
        if (m & 1) y0 = pn[0];
        if (m & 2) y1 = pn[1];
        if (m & 4) y2 = pn[2];
        y[3 * n + 0] = y0;
        y[3 * n + 1] = y1;
        y[3 * n + 2] = y2;
        if (dot_pq) dot = pn[0] * y0 + pn[1] * y1 + pn[2] * y2;
    }
    if (dot_pq) {
        double v[1] = {dot};
        if (grid_sum<1>(red, v, sh, out)) {
            if (flat_tid() == 0) {
                const double pq = out[0];
                ss->pq = pq;
                if (!(pq > 0.0) || !isfinite(pq)) {
                    ss->status = TO3D_ENUMERIC;
                    ss->done = 1;
                    ss->alpha = 0.0;
                } else {
                    ss->alpha = ss->rz / pq;
                }
            }
        }
    }
}

// Jacobi diagonal: every KE diagonal entry is the same number (all nodes of
// the unit hex are equivalent), so diag(K)_n = KE_00 * sum_{e ni n} E_e for
// each of the node's three dofs.  dinv = 0 on clamped dofs keeps the
// preconditioned residual zero there.
__global__ void k_diag(const Grid g, const double* __restrict__ E, double kdd,
                       const uint8_t* __restrict__ nodemask, double* __restrict__ dinv,
                       float* __restrict__ dinv32, int px) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nnode) return;
    const int i = n % g.nx, j = (n / g.nx) % g.ny, k = n / ((long long)g.nx * g.ny);
    double s = 0.0;
#pragma unroll
    for (int dz = -1; dz <= 0; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 0; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 0; ++dx) {
                const int ei = i + dx, ej = j + dy, ek = k + dz;
                if (ei >= 0 && ei < g.nelx && ej >= 0 && ej < g.nely && ek >= 0 && ek < g.nelz)
                    s += E[elem_id(g, ei, ej, ek)];
            }
    const double d = s * kdd;
    const uint8_t m = nodemask[n];
    // a node whose three dofs are all clamped gets 0; partially clamped nodes
    // keep 1/d and the clamped components are zeroed by the residual mask
    const double di = (m == 7 || !(d > 0.0)) ? 0.0 : 1.0 / d;
    dinv[n] = di;
    dinv32[i + (long long)px * (j + (long long)g.ny * k)] = (float)di;   // padded layout
}

// E_e = Emin + x_e^p (E0 - Emin) (Section 2.3), FP64 and an FP32 copy.
__global__ void k_simp(long long nel, int nelx, int pex, const double* __restrict__ x,
                       double penal, double E0, double Emin, double* __restrict__ E,
                       float* __restrict__ E32) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= nel) return;
    const double xe = x[e];
    const double xp = (penal == 3.0) ? xe * xe * xe : pow(xe, penal);
    const double v = Emin + xp * (E0 - Emin);
    E[e] = v;
    E32[(e % nelx) + (long long)pex * (e / nelx)] = (float)v;   // padded rows
}

// r = f - Ku on free dofs (0 on clamped); optional grid sums of r.r into ss.
__global__ void k_residual64(long long ndof, const double* __restrict__ f,
                             const double* __restrict__ Ku, const uint8_t* __restrict__ nodemask,
                             double* __restrict__ r, const Reducer red, SolverScalars* ss,
                             int to_ss) {
    __shared__ double sh[32];
    __shared__ double out[1];
    double acc = 0.0;
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < ndof;
         d += (long long)gridDim.x * blockDim.x) {
        const bool fx = (nodemask[d / 3] >> (d % 3)) & 1;
        const double v = fx ? 0.0 : f[d] - Ku[d];
        r[d] = v;
        acc += v * v;
    }
    if (to_ss) {
        double v[1] = {acc};
        if (grid_sum<1>(red, v, sh, out) && threadIdx.x == 0) ss->rr_true = out[0];
    }
}

// dst = src with clamped dofs zeroed
__global__ void k_mask_copy(long long ndof, const double* __restrict__ src,
                            const uint8_t* __restrict__ nodemask, double* __restrict__ dst) {
    for (long long d = blockIdx.x * (long long)blockDim.x + threadIdx.x; d < ndof;
         d += (long long)gridDim.x * blockDim.x)
        dst[d] = ((nodemask[d / 3] >> (d % 3)) & 1) ? 0.0 : src[d];
}

void launch_mask_copy(to3d_ctx* c, cudaStream_t s, const double* src, double* dst) {
    k_mask_copy<<<152 * 8, 256, 0, s>>>(3 * c->g.nnode, src, c->nodemask, dst);
    c->launches++;
}

void launch_matvec64(to3d_ctx* c, cudaStream_t s, const double* E, const double* p, double* y,
                     bool dot_pq) {
    if (c->prm.fp64_tc && matvec_x64_available(c)) {
        launch_matvec_x64(c, s, E, p, y, dot_pq);
        return;
    }
    const Grid& g = c->g;
    dim3 blk(MV_TX, MV_TY, MV_TZ);
    dim3 grd((g.nx + MV_TX - 1) / MV_TX, (g.ny + MV_TY - 1) / MV_TY, (g.nz + MV_TZ - 1) / MV_TZ);
    k_matvec64<<<grd, blk, 0, s>>>(c->ke, g, E, p, c->nodemask, y, c->red, c->ss, dot_pq ? 1 : 0);
    c->launches++;
}

void launch_diag(to3d_ctx* c, cudaStream_t s, const double* E) {
    const Grid& g = c->g;
    k_diag<<<(unsigned)((g.nnode + 255) / 256), 256, 0, s>>>(g, E, c->ke.v[0], c->nodemask,
                                                             c->dinv, c->dinv32, c->px);
    c->launches++;
}

void launch_simp(to3d_ctx* c, cudaStream_t s, const double* x) {
    const Grid& g = c->g;
    k_simp<<<(unsigned)((g.nel + 255) / 256), 256, 0, s>>>(g.nel, g.nelx, c->pex, x, c->prm.penal,
                                                           c->prm.E0, c->prm.Emin, c->E, c->E32);
    c->launches++;
}

void launch_residual64(to3d_ctx* c, cudaStream_t s, const double* f, const double* Ku, double* r,
                       bool to_ss) {
    const long long ndof = 3 * c->g.nnode;
    long long nb = (ndof + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    k_residual64<<<(unsigned)nb, 256, 0, s>>>(ndof, f, Ku, c->nodemask, r, c->red, c->ss,
                                              to_ss ? 1 : 0);
    c->launches++;
}

}  // namespace to3d
