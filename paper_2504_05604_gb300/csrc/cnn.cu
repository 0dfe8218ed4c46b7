// Learned preconditioner: a four-level U-Net on the node grid (channels
// 16/32/64/64, 3x3x3 convolutions, 2x2x2 average pooling down, nearest x2
// up with skip concatenation, ReLU), trained on the GPU with this
// library's own forward and backward kernels from residuals that the
// method's own solves produce, and applied inside flexible CG.
//
// Input channels: the Jacobi-scaled residual rt = D^-1/2 r divided by its
// RMS s (3) and log10 of the node density (mean of the adjacent elements,
// clamped at 1e-3), padded to 16 channels; output: three correction
// channels, z = D^-1 r + s D^-1/2 out (a zero network is plain Jacobi).  The
// node grid is zero-padded to multiples of 8 in every direction.
//
// Flexible CG (Polak-Ribiere beta, FP64 vectors) takes z = D^-1 r in any
// iteration where the network's r^T z <= 0, and falls back to Jacobi-PCG
// from its current iterate on a non-positive curvature, when the smallest
// residual seen drops by less than 10 % over 200 iterations, or when it
// runs 10x behind the rate of the context's last plain Jacobi-PCG solve;
// the true FP64 residual decides convergence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cnn_kernels.cuh"
#include "internal.cuh"
#include "reduce.cuh"

#define CK_RET(call)                                         \
    do {                                                     \
        cudaError_t _e = (call);                             \
        if (_e != cudaSuccess) return cuda_check(c, _e, #call); \
    } while (0)

namespace to3d {
namespace cnn {

constexpr int IN_CHANNELS = 4, OUT_CHANNELS = 3;

struct Layer {
    int co, ci, c1;          // output, input channels; input channels taken from the first tensor
    size_t woff, boff;       // offsets in the flat parameter vector (floats)
    size_t wb_off;           // offset in the BF16 weight images (elements)
};

enum { E0A, E0B, E1A, E1B, E2A, E2B, E3A, E3B, D2A, D2B, D1A, D1B, D0A, D0B, OUT, NLAYER };

struct Work {
    int Z = 0, Y = 0, X = 0;
    bool grads = false;
    std::vector<void*> bufs;
    bf16 *in = nullptr, *e0a, *e0, *p0, *e1a, *e1, *p1, *e2a, *e2, *p2, *e3a, *e3, *u3, *d2a, *d2,
         *u2, *d1a, *d1, *u1, *d0a, *d0;
    float* out = nullptr;
    float *g_out, *g_d0, *g_d0a, *g_cat0, *g_d1, *g_d1a, *g_cat1, *g_d2, *g_d2a, *g_cat2, *g_e3,
        *g_e3a, *g_p2, *g_e2, *g_e2a, *g_p1, *g_e1, *g_e1a, *g_p0, *g_e0, *g_e0a;
};

struct Net {
    Layer L[NLAYER];
    size_t nparam = 0, nwb = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    bf16 *Wb = nullptr, *Wt = nullptr;
    int t = 0;
    Work inf, trn;
    // training snapshots: network input on the padded node grid, the
    // residual r (FP64, dofs), the design x it belongs to and r^T K^-1 r
    struct Snap {
        bf16* in = nullptr;
        double* r = nullptr;
        double* x = nullptr;
        double rte = 0.0;
    };
    std::vector<Snap> snaps;
    int Zp = 0, Yp = 0, Xp = 0;
    // flexible-CG vectors
    double *z = nullptr, *rprev = nullptr;
    double* dots = nullptr;      // device scalars
    double* dots_h = nullptr;
    bool trained = false;
};

static void free_work(Work& w) {
    for (void* p : w.bufs) cudaFree(p);
    w.bufs.clear();
    w.Z = w.Y = w.X = 0;
}

void free_net(Net* n) {
    if (!n) return;
    free_work(n->inf);
    free_work(n->trn);
    for (auto& sn : n->snaps) {
        cudaFree(sn.in);
        cudaFree(sn.r);
        cudaFree(sn.x);
    }
    void* ptrs[] = {n->P, n->G, n->M, n->V, n->Wb, n->Wt, n->z, n->rprev, n->dots};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (n->dots_h) cudaFreeHost(n->dots_h);
    delete n;
}

static bool alloc_work(Work& w, int Z, int Y, int X, bool grads) {
    if (w.Z == Z && w.Y == Y && w.X == X && w.grads == grads) return true;
    free_work(w);
    w.Z = Z; w.Y = Y; w.X = X; w.grads = grads;
    const long long v0 = (long long)Z * Y * X, v1 = v0 / 8, v2 = v1 / 8, v3 = v2 / 8;
    auto B = [&](bf16** p, long long n) {
        if (cudaMalloc((void**)p, sizeof(bf16) * n) != cudaSuccess) return false;
        w.bufs.push_back(*p);
        return true;
    };
    auto F = [&](float** p, long long n) {
        if (cudaMalloc((void**)p, sizeof(float) * n) != cudaSuccess) return false;
        w.bufs.push_back(*p);
        return true;
    };
    bool ok = B(&w.in, 16 * v0) && B(&w.e0a, 16 * v0) && B(&w.e0, 16 * v0) && B(&w.p0, 16 * v1) &&
              B(&w.e1a, 32 * v1) && B(&w.e1, 32 * v1) && B(&w.p1, 32 * v2) && B(&w.e2a, 64 * v2) &&
              B(&w.e2, 64 * v2) && B(&w.p2, 64 * v3) && B(&w.e3a, 64 * v3) && B(&w.e3, 64 * v3) &&
              B(&w.u3, 64 * v2) && B(&w.d2a, 64 * v2) && B(&w.d2, 64 * v2) && B(&w.u2, 64 * v1) &&
              B(&w.d1a, 32 * v1) && B(&w.d1, 32 * v1) && B(&w.u1, 32 * v0) && B(&w.d0a, 16 * v0) &&
              B(&w.d0, 16 * v0) && F(&w.out, 16 * v0);
    if (ok && grads)
        ok = F(&w.g_out, 16 * v0) && F(&w.g_d0, 16 * v0) && F(&w.g_d0a, 16 * v0) &&
             F(&w.g_cat0, 48 * v0) && F(&w.g_d1, 32 * v1) && F(&w.g_d1a, 32 * v1) &&
             F(&w.g_cat1, 96 * v1) && F(&w.g_d2, 64 * v2) && F(&w.g_d2a, 64 * v2) &&
             F(&w.g_cat2, 128 * v2) && F(&w.g_e3, 64 * v3) && F(&w.g_e3a, 64 * v3) &&
             F(&w.g_p2, 64 * v3) && F(&w.g_e2, 64 * v2) && F(&w.g_e2a, 64 * v2) &&
             F(&w.g_p1, 32 * v2) && F(&w.g_e1, 32 * v1) && F(&w.g_e1a, 32 * v1) &&
             F(&w.g_p0, 16 * v1) && F(&w.g_e0, 16 * v0) && F(&w.g_e0a, 16 * v0);
    if (!ok) free_work(w);
    return ok;
}

// ---- layer table (matches the network description above)
static void build_layers(Net* n) {
    const int spec[NLAYER][3] = {{16, 16, 16}, {16, 16, 16}, {32, 16, 16}, {32, 32, 32},
                                 {64, 32, 32}, {64, 64, 64}, {64, 64, 64}, {64, 64, 64},
                                 {64, 128, 64}, {64, 64, 64}, {32, 96, 64}, {32, 32, 32},
                                 {16, 48, 32}, {16, 16, 16}, {16, 16, 16}};
    size_t off = 0, wb = 0;
    for (int i = 0; i < NLAYER; ++i) {
        Layer& l = n->L[i];
        l.co = spec[i][0];
        l.ci = spec[i][1];
        l.c1 = spec[i][2];
        l.woff = off;
        off += 27ull * l.co * l.ci;
        l.boff = off;
        off += l.co;
        l.wb_off = wb;
        wb += 27ull * l.co * l.ci;
    }
    n->nparam = off;
    n->nwb = wb;
}

// deterministic He-normal initialisation (counter-based hash + Box-Muller);
// input channels 4..15 of the first layer and output channels 3..15 of the
// last one stay zero
__device__ __forceinline__ float hash_uniform(unsigned long long k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
    return ((k >> 40) + 0.5f) * (1.0f / 16777216.0f);
}

__global__ void k_init_layer(float* w, float* b, int co, int ci, int ci_used, int co_used, float std,
                             unsigned long long seed) {
    const long long n = 27LL * co * ci;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < co) b[i] = 0.f;
    if (i >= n) return;
    const int c_in = (int)(i % ci), c_out = (int)((i / ci) % co);
    float v = 0.f;
    if (c_in < ci_used && c_out < co_used) {
        const float u1 = hash_uniform(seed * 0x9E3779B97F4A7C15ULL + 2 * i + 1);
        const float u2 = hash_uniform(seed * 0x9E3779B97F4A7C15ULL + 2 * i + 2);
        v = std * sqrtf(-2.f * logf(u1)) * cosf(6.2831853f * u2);
    }
    w[i] = v;
}

static void refresh_bf16(Net* n, cudaStream_t s) {
    for (int i = 0; i < NLAYER; ++i) {
        const Layer& l = n->L[i];
        to_bf16(n->P + l.woff, n->Wb + l.wb_off, 27LL * l.co * l.ci, s);
        transpose_flip(n->Wb + l.wb_off, n->Wt + l.wb_off, l.co, l.ci, s);
    }
}

// ---- forward / backward
static void conv(Net* n, int li, const Work& w, int lev, const void* in1, const void* in2,
                 bool relu, bf16* ob, float* of, cudaStream_t s) {
    const Layer& l = n->L[li];
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Z = w.Z >> lev; a.Y = w.Y >> lev; a.X = w.X >> lev;
    a.nvox = (long long)a.Z * a.Y * a.X;
    a.C1 = l.c1;
    a.C2 = l.ci - l.c1;
    a.Cout = l.co;
    a.in1 = in1;
    a.in2 = in2;
    a.W = n->Wb + l.wb_off;
    a.bias = n->P + l.boff;
    a.out_b = ob;
    a.out_f = of;
    a.out_cstride = l.co;
    a.relu = relu ? 1 : 0;
    conv_forward(a, false, s);
}

static void forward(Net* n, const Work& w, const bf16* in, cudaStream_t s) {
    const int Z = w.Z, Y = w.Y, X = w.X;
    conv(n, E0A, w, 0, in, nullptr, true, w.e0a, nullptr, s);
    conv(n, E0B, w, 0, w.e0a, nullptr, true, w.e0, nullptr, s);
    pool2_forward(w.e0, w.p0, Z, Y, X, 16, s);
    conv(n, E1A, w, 1, w.p0, nullptr, true, w.e1a, nullptr, s);
    conv(n, E1B, w, 1, w.e1a, nullptr, true, w.e1, nullptr, s);
    pool2_forward(w.e1, w.p1, Z >> 1, Y >> 1, X >> 1, 32, s);
    conv(n, E2A, w, 2, w.p1, nullptr, true, w.e2a, nullptr, s);
    conv(n, E2B, w, 2, w.e2a, nullptr, true, w.e2, nullptr, s);
    pool2_forward(w.e2, w.p2, Z >> 2, Y >> 2, X >> 2, 64, s);
    conv(n, E3A, w, 3, w.p2, nullptr, true, w.e3a, nullptr, s);
    conv(n, E3B, w, 3, w.e3a, nullptr, true, w.e3, nullptr, s);
    up2_forward(w.e3, w.u3, Z >> 2, Y >> 2, X >> 2, 64, s);
    conv(n, D2A, w, 2, w.u3, w.e2, true, w.d2a, nullptr, s);
    conv(n, D2B, w, 2, w.d2a, nullptr, true, w.d2, nullptr, s);
    up2_forward(w.d2, w.u2, Z >> 1, Y >> 1, X >> 1, 64, s);
    conv(n, D1A, w, 1, w.u2, w.e1, true, w.d1a, nullptr, s);
    conv(n, D1B, w, 1, w.d1a, nullptr, true, w.d1, nullptr, s);
    up2_forward(w.d1, w.u1, Z, Y, X, 32, s);
    conv(n, D0A, w, 0, w.u1, w.e0, true, w.d0a, nullptr, s);
    conv(n, D0B, w, 0, w.d0a, nullptr, true, w.d0, nullptr, s);
    conv(n, OUT, w, 0, w.d0, nullptr, false, nullptr, w.out, s);
}

// gradient of layer li: weights and bias (accumulated into G) and, if gx,
// the input gradient (written, FP32, all ci channels)
static void bconv(Net* n, int li, const Work& w, int lev, const float* gy, const bf16* act,
                  const void* x1, const void* x2, float* gx, cudaStream_t s) {
    const Layer& l = n->L[li];
    WgradArgs wa;
    wa.Z = w.Z >> lev; wa.Y = w.Y >> lev; wa.X = w.X >> lev;
    wa.nvox = (long long)wa.Z * wa.Y * wa.X;
    wa.Cout = l.co;
    wa.Cin = l.ci;
    wa.gy = gy;
    wa.gy_cstride = l.co;
    wa.mask = act;
    wa.x1 = x1;
    wa.x2 = x2;
    wa.C1 = l.c1;
    wa.gw = n->G + l.woff;
    wa.Cout_fwd = l.co;
    wa.gb = n->G + l.boff;
    conv_wgrad(wa, false, s);
    if (!gx) return;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Z = wa.Z; a.Y = wa.Y; a.X = wa.X;
    a.nvox = wa.nvox;
    a.C1 = l.co;
    a.C2 = 0;
    a.Cout = l.ci;
    a.in1 = gy;
    a.mask1 = act;
    a.W = n->Wt + l.wb_off;
    a.out_f = gx;
    a.out_cstride = l.ci;
    conv_forward(a, true, s);
}

static void backward(Net* n, const Work& w, const bf16* in, cudaStream_t s) {
    const int Z = w.Z, Y = w.Y, X = w.X;
    const long long v0 = (long long)Z * Y * X, v1 = v0 / 8, v2 = v1 / 8;
    cudaMemsetAsync(n->G, 0, sizeof(float) * n->nparam, s);
    bconv(n, OUT, w, 0, w.g_out, nullptr, w.d0, nullptr, w.g_d0, s);
    bconv(n, D0B, w, 0, w.g_d0, w.d0, w.d0a, nullptr, w.g_d0a, s);
    bconv(n, D0A, w, 0, w.g_d0a, w.d0a, w.u1, w.e0, w.g_cat0, s);
    up2_backward(w.g_cat0, 48, 0, w.g_d1, Z, Y, X, 32, 0, s);
    add_channels(w.g_cat0, 48, 32, w.g_e0, v0, 16, 0, s);
    bconv(n, D1B, w, 1, w.g_d1, w.d1, w.d1a, nullptr, w.g_d1a, s);
    bconv(n, D1A, w, 1, w.g_d1a, w.d1a, w.u2, w.e1, w.g_cat1, s);
    up2_backward(w.g_cat1, 96, 0, w.g_d2, Z >> 1, Y >> 1, X >> 1, 64, 0, s);
    add_channels(w.g_cat1, 96, 64, w.g_e1, v1, 32, 0, s);
    bconv(n, D2B, w, 2, w.g_d2, w.d2, w.d2a, nullptr, w.g_d2a, s);
    bconv(n, D2A, w, 2, w.g_d2a, w.d2a, w.u3, w.e2, w.g_cat2, s);
    up2_backward(w.g_cat2, 128, 0, w.g_e3, Z >> 2, Y >> 2, X >> 2, 64, 0, s);
    add_channels(w.g_cat2, 128, 64, w.g_e2, v2, 64, 0, s);
    bconv(n, E3B, w, 3, w.g_e3, w.e3, w.e3a, nullptr, w.g_e3a, s);
    bconv(n, E3A, w, 3, w.g_e3a, w.e3a, w.p2, nullptr, w.g_p2, s);
    pool2_backward(w.g_p2, 64, 0, w.g_e2, Z >> 2, Y >> 2, X >> 2, 64, 1, s);
    bconv(n, E2B, w, 2, w.g_e2, w.e2, w.e2a, nullptr, w.g_e2a, s);
    bconv(n, E2A, w, 2, w.g_e2a, w.e2a, w.p1, nullptr, w.g_p1, s);
    pool2_backward(w.g_p1, 32, 0, w.g_e1, Z >> 1, Y >> 1, X >> 1, 32, 1, s);
    bconv(n, E1B, w, 1, w.g_e1, w.e1, w.e1a, nullptr, w.g_e1a, s);
    bconv(n, E1A, w, 1, w.g_e1a, w.e1a, w.p0, nullptr, w.g_p0, s);
    pool2_backward(w.g_p0, 16, 0, w.g_e0, Z, Y, X, 16, 1, s);
    bconv(n, E0B, w, 0, w.g_e0, w.e0, w.e0a, nullptr, w.g_e0a, s);
    bconv(n, E0A, w, 0, w.g_e0a, w.e0a, in, nullptr, nullptr, s);
}

// ---- problem <-> network tensors
// in[v][16]: D^-1/2 r / s (0 on clamped dofs), log10 of the node density,
// zeros; rr = |D^-1/2 r|^2, s = sqrt(rr / 3N)
__global__ void k_make_input(const Grid g, int Zp, int Yp, int Xp, const double* __restrict__ r,
                             const double* __restrict__ dinv, const double* __restrict__ x,
                             const uint8_t* __restrict__ nodemask, const double* __restrict__ rr,
                             bf16* __restrict__ in) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nv = (long long)Zp * Yp * Xp;
    if (v >= nv) return;
    const int i = (int)(v % Xp), j = (int)((v / Xp) % Yp), k = (int)(v / ((long long)Xp * Yp));
    float ch[4] = {0.f, 0.f, 0.f, 0.f};
    if (i < g.nx && j < g.ny && k < g.nz) {
        const long long n = node_id(g, i, j, k);
        const double inv = *rr > 0.0 ? sqrt(dinv[n]) / sqrt(*rr / (3.0 * g.nnode)) : 0.0;
        const uint8_t m = nodemask[n];
        for (int c = 0; c < 3; ++c) ch[c] = ((m >> c) & 1) ? 0.f : (float)(r[3 * n + c] * inv);
        double s = 0.0;
        int cnt = 0;
        for (int d = 0; d < 8; ++d) {
            const int ei = i - 1 + (d & 1), ej = j - 1 + ((d >> 1) & 1), ek = k - 1 + (d >> 2);
            if (ei >= 0 && ei < g.nelx && ej >= 0 && ej < g.nely && ek >= 0 && ek < g.nelz) {
                s += x[elem_id(g, ei, ej, ek)];
                ++cnt;
            }
        }
        ch[3] = (float)log10(fmax(1e-3, cnt ? s / cnt : 1e-3));
    }
    bf16* o = in + v * 16;
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(c < 4 ? ch[c] : 0.f);
}

// z = D^-1 r + s D^-1/2 out on free dofs, 0 on clamped ones
__global__ void k_take_output(const Grid g, int Yp, int Xp, const float* __restrict__ out,
                              const double* __restrict__ r, const double* __restrict__ dinv,
                              const uint8_t* __restrict__ nodemask, const double* __restrict__ rr,
                              double* __restrict__ z) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nnode) return;
    const double d = dinv[n];
    const double s = sqrt(*rr / (3.0 * g.nnode)) * sqrt(d);
    const int i = n % g.nx, j = (n / g.nx) % g.ny, k = n / ((long long)g.nx * g.ny);
    const long long v = i + (long long)Xp * (j + (long long)Yp * k);
    const uint8_t m = nodemask[n];
    for (int c = 0; c < 3; ++c)
        z[3 * n + c] = ((m >> c) & 1) ? 0.0 : fma(s, (double)out[v * 16 + c], d * r[3 * n + c]);
}

// rr = sum_n dinv_n |r_n|^2 = |D^-1/2 r|^2
__global__ void k_scaled_norm2(long long nnode, const double* __restrict__ dinv,
                               const double* __restrict__ r, const Reducer red, double* out) {
    __shared__ double sh[64];
    __shared__ double o2[2];
    double a = 0.0;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const double r0 = r[3 * n], r1 = r[3 * n + 1], r2 = r[3 * n + 2];
        a = fma(dinv[n], r0 * r0 + r1 * r1 + r2 * r2, a);
    }
    double v[2] = {a, 0.0};
    if (grid_sum<2>(red, v, sh, o2) && threadIdx.x == 0) *out = o2[0];
}

// gradient of the energy loss with respect to the network output on the
// padded grid: 2 s D^-1/2 (K z - r) / (r^T e) on free dofs (channels 0..2),
// else 0
__global__ void k_energy_grad(const Grid g, int Zp, int Yp, int Xp, const double* __restrict__ q,
                              const double* __restrict__ r, const double* __restrict__ dinv,
                              const uint8_t* __restrict__ nodemask, const double* __restrict__ rr,
                              double rte, float* __restrict__ gout) {
    const long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long nv = (long long)Zp * Yp * Xp;
    if (v >= nv) return;
    const int i = (int)(v % Xp), j = (int)((v / Xp) % Yp), k = (int)(v / ((long long)Xp * Yp));
    float gv[3] = {0.f, 0.f, 0.f};
    if (i < g.nx && j < g.ny && k < g.nz) {
        const long long n = node_id(g, i, j, k);
        const double f = 2.0 * sqrt(*rr / (3.0 * g.nnode)) * sqrt(dinv[n]) / rte;
        const uint8_t m = nodemask[n];
        for (int c = 0; c < 3; ++c)
            gv[c] = ((m >> c) & 1) ? 0.f : (float)(f * (q[3 * n + c] - r[3 * n + c]));
    }
    float* o = gout + v * 16;
    for (int c = 0; c < 16; ++c) o[c] = c < 3 ? gv[c] : 0.f;
}

// ---- small FP64 vector helpers for flexible CG
__global__ void k_dots(long long n, const double* a, const double* b, const double* c,
                       const double* d, const Reducer red, double* out_dev) {
    __shared__ double sh[64];
    __shared__ double o2[2];
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        s0 = fma(a[i], b[i], s0);
        if (c) s1 = fma(c[i], d[i], s1);
    }
    double v[2] = {s0, s1};
    if (grid_sum<2>(red, v, sh, o2) && threadIdx.x == 0) {
        out_dev[0] = o2[0];
        out_dev[1] = o2[1];
    }
}

__global__ void k_fcg_step(long long n, double alpha, double* u, const double* p, double* r,
                           double* rprev, const double* q) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        u[i] = fma(alpha, p[i], u[i]);
        rprev[i] = r[i];
        r[i] = fma(-alpha, q[i], r[i]);
    }
}

__global__ void k_fcg_dir(long long n, double beta, double* p, const double* z) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        p[i] = fma(beta, p[i], z[i]);
}

// (r - rprev) . z  = r.z - rprev.z
__global__ void k_pr_dots(long long n, const double* r, const double* rprev, const double* z,
                          const Reducer red, double* out_dev) {
    __shared__ double sh[64];
    __shared__ double o2[2];
    double s0 = 0.0, s1 = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        s0 = fma(r[i] - rprev[i], z[i], s0);
        s1 = fma(r[i], z[i], s1);
    }
    double v[2] = {s0, s1};
    if (grid_sum<2>(red, v, sh, o2) && threadIdx.x == 0) {
        out_dev[0] = o2[0];
        out_dev[1] = o2[1];
    }
}

static unsigned blocks(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b > 1216 ? 1216 : (b < 1 ? 1 : b));
}

}  // namespace cnn

using namespace cnn;

static Net* net_of(to3d_ctx* c) { return (Net*)c->cnn; }

static bool ensure_net(to3d_ctx* c) {
    if (c->cnn) return true;
    Net* n = new (std::nothrow) Net();
    if (!n) return false;
    build_layers(n);
    n->Zp = (c->g.nz + 7) / 8 * 8;
    n->Yp = (c->g.ny + 7) / 8 * 8;
    n->Xp = (c->g.nx + 7) / 8 * 8;
    const long long ndof = 3 * c->g.nnode;
    if (cudaMalloc(&n->P, sizeof(float) * n->nparam) != cudaSuccess ||
        cudaMalloc(&n->G, sizeof(float) * n->nparam) != cudaSuccess ||
        cudaMalloc(&n->M, sizeof(float) * n->nparam) != cudaSuccess ||
        cudaMalloc(&n->V, sizeof(float) * n->nparam) != cudaSuccess ||
        cudaMalloc(&n->Wb, sizeof(bf16) * n->nwb) != cudaSuccess ||
        cudaMalloc(&n->Wt, sizeof(bf16) * n->nwb) != cudaSuccess ||
        cudaMalloc(&n->z, sizeof(double) * ndof) != cudaSuccess ||
        cudaMalloc(&n->rprev, sizeof(double) * ndof) != cudaSuccess ||
        cudaMalloc(&n->dots, sizeof(double) * 8) != cudaSuccess ||
        cudaMallocHost(&n->dots_h, sizeof(double) * 8) != cudaSuccess) {
        free_net(n);
        return false;
    }
    c->cnn = n;
    return true;
}

void destroy_cnn(to3d_ctx* c) {
    free_net(net_of(c));
    c->cnn = nullptr;
}

// z = M_cnn(r) for the context's grid; the operator (E, D^-1) must have
// been prepared for the densities the network reads
static to3d_status cnn_apply(to3d_ctx* c, const double* r, double* z) {
    Net* n = net_of(c);
    cudaStream_t s = c->stream;
    if (!alloc_work(n->inf, n->Zp, n->Yp, n->Xp, false))
        return set_err(c, TO3D_ENOMEM, "network workspace");
    k_scaled_norm2<<<blocks(c->g.nnode), 256, 0, s>>>(c->g.nnode, c->dinv, r, c->red, n->dots + 4);
    const long long nv = (long long)n->Zp * n->Yp * n->Xp;
    k_make_input<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(c->g, n->Zp, n->Yp, n->Xp, r,
                                                            c->dinv, c->xop ? c->xop : c->x,
                                                            c->nodemask, n->dots + 4, n->inf.in);
    forward(n, n->inf, n->inf.in, s);
    k_take_output<<<(unsigned)((c->g.nnode + 255) / 256), 256, 0, s>>>(
        c->g, n->Yp, n->Xp, n->inf.out, r, c->dinv, c->nodemask, n->dots + 4, z);
    c->launches += 26;
    return launch_check(c, "cnn apply");
}


static void init_weights(Net* n, unsigned long long seed, cudaStream_t s) {
    for (int i = 0; i < NLAYER; ++i) {
        const Layer& l = n->L[i];
        const int ci_used = (i == E0A) ? IN_CHANNELS : l.ci;
        const int co_used = (i == OUT) ? OUT_CHANNELS : l.co;
        const float std = sqrtf(2.f / (27.f * ci_used));
        const long long nw = 27LL * l.co * l.ci;
        k_init_layer<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(
            n->P + l.woff, n->P + l.boff, l.co, l.ci, ci_used, co_used, std, seed * 131 + i);
    }
    cudaMemsetAsync(n->M, 0, sizeof(float) * n->nparam, s);
    cudaMemsetAsync(n->V, 0, sizeof(float) * n->nparam, s);
    n->t = 0;
    refresh_bf16(n, s);
}

// Snapshot: Jacobi-PCG (source 0) or flexible CG with the current network
// (source 1) from u = 0, stopped after `iters` iterations (0: the load
// itself), gives a residual r of the kind a solver meets; r^T K^-1 r comes
// from an FP64 solve to 1e-10.
static to3d_status fcg_run_iters(to3d_ctx* c, const double* f, int iters);

static to3d_status add_snapshot(to3d_ctx* c, int iters, int source) {
    Net* n = net_of(c);
    cudaStream_t s = c->stream;
    to3d_status st;
    const long long ndof = 3 * c->g.nnode;
    if ((st = prepare_op(c, c->x))) return st;
    if (source == 1) st = fcg_run_iters(c, c->f, iters);
    else st = run_pcg64_iters(c, c->f, iters);
    if (st) return st;
    c->have_u = false;          // u now holds the snapshot's iterate, not the displacement
    // true residual of the truncated solve into tmp
    launch_matvec64(c, s, c->E, c->u, c->q, false);
    launch_residual64(c, s, c->f, c->q, c->tmp, false);
    launch_norm2(c, s, c->tmp, ndof, n->dots + 4);
    CK_RET(cudaMemcpyAsync(n->dots_h, n->dots, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    CK_RET(cudaStreamSynchronize(s));
    const double rn = std::sqrt(n->dots_h[4]);
    if (!(rn > 0.0)) return TO3D_OK;
    to3d_solve_info si{};
    if ((st = solve64_rtol(c, c->tmp, rn, 1e-10, &si))) return st;
    k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->tmp, c->u, nullptr, nullptr, c->red, n->dots);
    CK_RET(cudaMemcpyAsync(n->dots_h, n->dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    CK_RET(cudaStreamSynchronize(s));
    Net::Snap sn;
    sn.rte = n->dots_h[0];
    if (!(sn.rte > 0.0)) return TO3D_OK;
    const long long nv = (long long)n->Zp * n->Yp * n->Xp;
    if (cudaMalloc(&sn.in, sizeof(bf16) * 16 * nv) != cudaSuccess ||
        cudaMalloc(&sn.r, sizeof(double) * ndof) != cudaSuccess ||
        cudaMalloc(&sn.x, sizeof(double) * c->g.nel) != cudaSuccess) {
        cudaFree(sn.in);
        cudaFree(sn.r);
        cudaFree(sn.x);
        return set_err(c, TO3D_ENOMEM, "training snapshot");
    }
    n->snaps.push_back(sn);
    k_scaled_norm2<<<blocks(c->g.nnode), 256, 0, s>>>(c->g.nnode, c->dinv, c->tmp, c->red,
                                                      n->dots + 4);
    k_make_input<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(c->g, n->Zp, n->Yp, n->Xp, c->tmp,
                                                            c->dinv, c->x, c->nodemask,
                                                            n->dots + 4, sn.in);
    CK_RET(cudaMemcpyAsync(sn.r, c->tmp, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
    CK_RET(cudaMemcpyAsync(sn.x, c->x, sizeof(double) * c->g.nel, cudaMemcpyDeviceToDevice, s));
    return launch_check(c, "snapshot");
}

// One forward/backward pass of the energy loss on (in, r, x, rte): the
// parameter gradient lands in G, z^T K z and z^T r in zq_zr[0..1].
static void energy_pass(to3d_ctx* c, const bf16* in, const double* r, const double* x,
                        double rte, double* zq_zr) {
    Net* n = net_of(c);
    cudaStream_t s = c->stream;
    const long long ndof = 3 * c->g.nnode;
    const long long nv = (long long)n->Zp * n->Yp * n->Xp;
    prepare_op(c, x);                 // E and D^-1 of the sample's design
    k_scaled_norm2<<<blocks(c->g.nnode), 256, 0, s>>>(c->g.nnode, c->dinv, r, c->red, n->dots + 4);
    forward(n, n->trn, in, s);
    k_take_output<<<(unsigned)((c->g.nnode + 255) / 256), 256, 0, s>>>(
        c->g, n->Yp, n->Xp, n->trn.out, r, c->dinv, c->nodemask, n->dots + 4, n->z);
    launch_matvec64(c, s, c->E, n->z, c->q, false);
    k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, n->z, c->q, n->z, r, c->red, zq_zr);
    k_energy_grad<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(c->g, n->Zp, n->Yp, n->Xp, c->q, r,
                                                              c->dinv, c->nodemask, n->dots + 4,
                                                              rte, n->trn.g_out);
    backward(n, n->trn, in, s);
    c->launches += 70;
}

static unsigned long long mix(unsigned long long k) {
    k ^= k >> 33; k *= 0xff51afd7ed558ccdULL; k ^= k >> 33; k *= 0xc4ceb9fe1a85ec53ULL; k ^= k >> 33;
    return k;
}

// z = D^-1 r (Jacobi), the substitute when the network's z is no descent
// direction
__global__ void k_jacobi_z(long long nnode, const double* __restrict__ dinv,
                           const double* __restrict__ r, double* __restrict__ z) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < nnode;
         n += (long long)gridDim.x * blockDim.x) {
        const double d = dinv[n];
        for (int c = 0; c < 3; ++c) z[3 * n + c] = d * r[3 * n + c];
    }
}

struct FcgRun {
    int its = 0;             // iterations done
    int jacobi_steps = 0;    // iterations whose z was D^-1 r instead of the network's
    bool broke = false;      // stopped early: no progress or a non-positive curvature
    const char* why = "";
    double rr = 0.0;         // recurrence |r|^2 at exit
};

// Flexible CG (Polak-Ribiere beta, FP64) from the current u for at most
// max_its iterations or until |r|^2 <= rr_stop.  Whenever r^T z <= 0 the
// iteration takes z = D^-1 r instead (a flexible method may change its
// preconditioner every step).  With `stall_check`, it stops when the
// smallest |r| seen has dropped by less than 10 % over the last 200
// iterations (|r| of CG-type methods is not monotone, and plain Jacobi-PCG
// on SIMP designs can plateau for some 50 iterations), or when it loses to
// Jacobi-PCG: past 50 iterations, the smallest |r| is 10x above what the
// context's last plain solve (else params.fcg_ref_iters) would have reached
// at its average rate.
static to3d_status network_apply(to3d_ctx* c, const double* r, double* z, double) {
    return cnn_apply(c, r, z);
}

static FcgIO net_io(Net* n) {
    FcgIO io;
    io.z = n->z;
    io.rprev = n->rprev;
    io.dots = n->dots;
    io.dots_h = n->dots_h;
    io.apply = network_apply;
    return io;
}

static to3d_status fcg_run(to3d_ctx* c, const FcgIO& io, const double* f, int max_its,
                           double rr_stop, bool stall_check, double rtol, FcgRun* out) {
    cudaStream_t s = c->stream;
    const long long ndof = 3 * c->g.nnode;
    to3d_status st;
    FcgRun R;
    double rr_cur = 0.0;
    // z = M r with the preconditioner of `io`; z = D^-1 r when M gives no
    // descent direction (r^T z <= 0)
    auto precond_z = [&](double* rz, double* rr) -> to3d_status {
        k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->r, c->r, nullptr, nullptr, c->red, io.dots);
        CK_RET(cudaMemcpyAsync(io.dots_h, io.dots, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        rr_cur = io.dots_h[0];
        to3d_status e = io.apply(c, c->r, io.z, rr_cur);
        if (e) return e;
        k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->r, io.z, c->r, c->r, c->red, io.dots);
        CK_RET(cudaMemcpyAsync(io.dots_h, io.dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        *rz = io.dots_h[0];
        *rr = io.dots_h[1];
        if (!(*rz > 0.0) && *rr > 0.0) {
            R.jacobi_steps++;
            k_jacobi_z<<<blocks(c->g.nnode), 256, 0, s>>>(c->g.nnode, c->dinv, c->r, io.z);
            k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->r, io.z, nullptr, nullptr, c->red, io.dots);
            CK_RET(cudaMemcpyAsync(io.dots_h, io.dots, sizeof(double), cudaMemcpyDeviceToHost, s));
            CK_RET(cudaStreamSynchronize(s));
            *rz = io.dots_h[0];
        }
        return TO3D_OK;
    };
    // r = f - K u
    launch_matvec64(c, s, c->E, c->u, c->q, false);
    launch_residual64(c, s, f, c->q, c->r, false);
    double rz, rr;
    if ((st = precond_z(&rz, &rr))) return st;
    CK_RET(cudaMemcpyAsync(c->p, io.z, sizeof(double) * ndof, cudaMemcpyDeviceToDevice, s));
    double best = rr;
    std::vector<double> marks(1, rr);     // smallest |r|^2 seen, every 50 iterations
    const int ref_its = c->pcg_its_est > 0 ? c->pcg_its_est : c->prm.fcg_ref_iters;
    if (c->trace) std::fprintf(stderr, "to3d: fcg start |r|^2 %.3e\n", rr);
    while (rr > rr_stop && R.its < max_its) {
        if (!(rz > 0.0)) {
            R.broke = true;
            R.why = "r^T D^-1 r <= 0";
            break;
        }
        launch_matvec64(c, s, c->E, c->p, c->q, false);
        k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->p, c->q, c->p, c->r, c->red, io.dots);
        CK_RET(cudaMemcpyAsync(io.dots_h, io.dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        const double pq = io.dots_h[0], pr = io.dots_h[1];
        if (!(pq > 0.0) || !std::isfinite(pq)) {
            R.broke = true;
            R.why = "p^T K p <= 0";
            break;
        }
        // exact line search along p (alpha = p^T r / p^T K p, not r^T z /
        // p^T K p): the K-norm error decreases in every step even when the
        // preconditioner changes between steps
        k_fcg_step<<<blocks(ndof), 256, 0, s>>>(ndof, pr / pq, c->u, c->p, c->r, io.rprev, c->q);
        const double rz_old = rz;
        if ((st = precond_z(&rz, &rr))) return st;
        // Polak-Ribiere: beta = z^T (r - r_prev) / (z_prev^T r_prev)
        k_pr_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->r, io.rprev, io.z, c->red, io.dots);
        CK_RET(cudaMemcpyAsync(io.dots_h, io.dots, sizeof(double), cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        const double beta = io.dots_h[0] / rz_old;
        ++R.its;
        if (!std::isfinite(rr) || !std::isfinite(rz) || !std::isfinite(beta)) {
            R.broke = true;
            R.why = "non-finite";
            break;
        }
        if (c->trace && R.its % 20 == 0)
            std::fprintf(stderr, "to3d: fcg it %d |r|^2 %.3e (%d Jacobi steps)\n", R.its, rr,
                         R.jacobi_steps);
        best = std::fmin(best, rr);
        // losing to Jacobi-PCG: after 50 iterations, |r| is 10x above where
        // the last plain solve's average rate would have brought it
        if (stall_check && ref_its > 0 && R.its >= 50 && R.its % 10 == 0 &&
            best > 100.0 * marks[0] * std::pow(rtol * rtol, (double)R.its / ref_its)) {
            R.broke = true;
            R.why = "slower than Jacobi-PCG";
            break;
        }
        if (stall_check && R.its % 50 == 0) {
            marks.push_back(best);
            const size_t k = marks.size();
            if (k > 4 && best > 0.81 * marks[k - 5]) {
                R.broke = true;
                R.why = "stall";
                break;
            }
        }
        k_fcg_dir<<<blocks(ndof), 256, 0, s>>>(ndof, beta, c->p, io.z);
    }
    R.rr = rr;
    *out = R;
    return launch_check(c, "flexible CG");
}

// `iters` flexible-CG iterations from u = 0 (fewer if it converges or breaks)
static to3d_status fcg_run_iters(to3d_ctx* c, const double* f, int iters) {
    launch_fill_zero(c, c->stream, c->u, sizeof(double) * 3 * c->g.nnode);
    FcgRun R;
    return fcg_run(c, net_io(net_of(c)), f, iters, 0.0, false, 0.0, &R);
}

// Flexible CG with the network as preconditioner; Jacobi-PCG fallback.
to3d_status solve_fcg(to3d_ctx* c, const double* f, double fnorm, to3d_solve_info* info) {
    FcgIO io;
    to3d_status st;
    if (c->prm.precond == TO3D_LMG) {
        if ((st = mg_fcg_io(c, &io))) return st;
    } else {
        Net* n = net_of(c);
        if (!n || !n->trained) return set_err(c, TO3D_ESTATE, "learned preconditioner not trained");
        io = net_io(n);
    }
    cudaStream_t s = c->stream;
    const double tol = c->prm.cg_rtol;
    FcgRun R;
    if ((st = fcg_run(c, io, f, c->prm.cg_maxit, 0.25 * tol * tol * fnorm * fnorm, true, tol, &R)))
        return st;
    bool fellback = R.broke || R.its >= c->prm.cg_maxit;
    if (c->trace)
        std::fprintf(stderr, "to3d: fcg %d its, %d Jacobi steps%s%s\n", R.its, R.jacobi_steps,
                     fellback ? ", falls back: " : "", fellback ? R.why : "");
    to3d_solve_info fi{};
    int status = TO3D_OK;
    if (fellback) {
        // Jacobi-PCG continues from the flexible-CG iterate only if that made
        // real progress (true residual below 1e-2 |f|): from an iterate that
        // did not, it needed more iterations than from zero
        launch_matvec64(c, s, c->E, c->u, c->q, false);
        launch_residual64(c, s, f, c->q, c->r, true);
        CK_RET(cudaMemcpyAsync(c->ss_h, c->ss, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        if (!(std::sqrt(c->ss_h->rr_true) <= 1e-2 * fnorm))
            launch_fill_zero(c, s, c->u, sizeof(double) * 3 * c->g.nnode);
        if ((st = solve64_from_u(c, f, fnorm, &fi))) return st;
        status = fi.status;
    } else {
        launch_matvec64(c, s, c->E, c->u, c->q, false);
        launch_residual64(c, s, f, c->q, c->r, true);
        CK_RET(cudaMemcpyAsync(c->ss_h, c->ss, sizeof(SolverScalars), cudaMemcpyDeviceToHost, s));
        CK_RET(cudaStreamSynchronize(s));
        fi.relres = fnorm > 0 ? std::sqrt(c->ss_h->rr_true) / fnorm : 0.0;
        if (fi.relres > tol) {      // recurrence and true residual disagree: finish with PCG
            if ((st = solve64_from_u(c, f, fnorm, &fi))) return st;
            status = fi.status;
            fellback = true;
        }
    }
    if (info) {
        info->iters = R.its + (fellback ? fi.iters : 0);
        info->outer = fellback ? 2 : 1;     // 2: the Jacobi-PCG fallback finished the solve
        info->status = status;
        info->relres = fi.relres;
    }
    return launch_check(c, "flexible CG solve");
}

}  // namespace to3d

using namespace to3d;

extern "C" {

to3d_status to3d_cnn_init(to3d_ctx* c, uint64_t seed) {
    if (!c) return TO3D_EINVAL;
    if (!ensure_net(c)) return set_err(c, TO3D_ENOMEM, "network parameters");
    init_weights(net_of(c), seed, c->stream);
    net_of(c)->trained = false;
    return launch_check(c, "cnn init");
}

to3d_status to3d_cnn_param_count(to3d_ctx* c, int64_t* n) {
    if (!c || !n) return TO3D_EINVAL;
    if (!ensure_net(c)) return set_err(c, TO3D_ENOMEM, "network parameters");
    *n = (int64_t)net_of(c)->nparam;
    return TO3D_OK;
}

to3d_status to3d_cnn_get_params(to3d_ctx* c, float* p, int64_t n) {
    if (!c || !p || !c->cnn || n != (int64_t)net_of(c)->nparam) return TO3D_EINVAL;
    CK_RET(cudaMemcpyAsync(p, net_of(c)->P, sizeof(float) * n, cudaMemcpyDeviceToHost, c->stream));
    CK_RET(cudaStreamSynchronize(c->stream));
    return TO3D_OK;
}

to3d_status to3d_cnn_set_params(to3d_ctx* c, const float* p, int64_t n) {
    if (!c || !p) return TO3D_EINVAL;
    if (!ensure_net(c)) return set_err(c, TO3D_ENOMEM, "network parameters");
    Net* net = net_of(c);
    if (n != (int64_t)net->nparam) return TO3D_EINVAL;
    CK_RET(cudaMemcpyAsync(net->P, p, sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
    cudaMemsetAsync(net->M, 0, sizeof(float) * n, c->stream);
    cudaMemsetAsync(net->V, 0, sizeof(float) * n, c->stream);
    net->t = 0;
    refresh_bf16(net, c->stream);
    net->trained = true;
    CK_RET(cudaStreamSynchronize(c->stream));
    return launch_check(c, "cnn set params");
}

to3d_status to3d_cnn_apply(to3d_ctx* c, const double* x, const double* r, double* z,
                           int32_t on_device) {
    if (!c || !x || !r || !z || !c->cnn) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 8;
    cudaStream_t s = c->stream;
    const void *dx, *dr;
    to3d_status st;
    if ((st = stage_input(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_input(c, r, db, on_device, 1, &dr))) return st;
    if ((st = prepare_op(c, (const double*)dx))) return st;
    launch_mask_copy(c, s, (const double*)dr, c->tmp);
    st = cnn_apply(c, c->tmp, net_of(c)->z);
    if (st) return st;
    CK_RET(cudaMemcpyAsync(z, net_of(c)->z, db, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK_RET(cudaStreamSynchronize(s));
    return TO3D_OK;
}

// Training on residual snapshots from the context's own OC trajectory.
to3d_status to3d_cnn_train(to3d_ctx* c, int32_t nsnap, int32_t per_design, int32_t steps,
                           double lr, uint64_t seed, int32_t source, double* loss_first,
                           double* loss_last) {
    if (!c || nsnap < 0 || per_design < 1 || steps < 0 || !(lr > 0) || source < 0 || source > 1)
        return TO3D_EINVAL;
    if (!ensure_net(c)) return set_err(c, TO3D_ENOMEM, "network parameters");
    Net* n = net_of(c);
    cudaStream_t s = c->stream;
    to3d_status st;
    if (n->t == 0 && !n->trained) init_weights(n, seed, s);
    const int prec = c->prm.precision, pc = c->prm.precond;
    for (int i = 0; i < nsnap; ++i) {
        // the first snapshot of each design is the load itself (what a cold
        // solve starts from), the others are stopped after 1..200 iterations
        const int iters = (i % per_design == 0) ? 0 : 1 + (int)(mix(seed * 977 + i) % 200);
        if ((st = add_snapshot(c, iters, source))) return st;
        if ((i + 1) % per_design == 0 && i + 1 < nsnap) {
            // advance the design with the plain method
            c->prm.precond = TO3D_JACOBI;
            c->prm.precision = TO3D_F64;
            st = to3d_step(c, nullptr);
            c->prm.precision = prec;
            c->prm.precond = pc;
            if (st) return st;
        }
    }
    if (steps == 0) return TO3D_OK;
    if (n->snaps.empty()) return set_err(c, TO3D_ESTATE, "no training snapshots");
    if (!alloc_work(n->trn, n->Zp, n->Yp, n->Xp, true))
        return set_err(c, TO3D_ENOMEM, "training workspace");
    double* dz = nullptr;
    CK_RET(cudaMalloc(&dz, sizeof(double) * 2 * steps));
    std::vector<double> rte(steps);
    for (int t = 0; t < steps; ++t) {
        const Net::Snap& sn = n->snaps[(size_t)(mix(seed * 31 + t) % n->snaps.size())];
        rte[t] = sn.rte;
        energy_pass(c, sn.in, sn.r, sn.x, sn.rte, dz + 2 * t);
        adam(n->P, n->G, n->M, n->V, (long long)n->nparam, (float)lr, 0.9f, 0.999f, 1e-8f, ++n->t, s);
        refresh_bf16(n, s);
        c->launches += 31;
    }
    std::vector<double> h(2 * steps);
    cudaMemcpyAsync(h.data(), dz, sizeof(double) * 2 * steps, cudaMemcpyDeviceToHost, s);
    const cudaError_t err = cudaStreamSynchronize(s);
    cudaFree(dz);
    if (err != cudaSuccess) return cuda_check(c, err, "cnn train");
    c->have_u = false;
    const int w = steps < 20 ? 1 : steps / 10;
    double a = 0.0, b = 0.0;
    for (int t = 0; t < w; ++t) {
        const int u = steps - 1 - t;
        a += (h[2 * t] - 2.0 * h[2 * t + 1] + rte[t]) / rte[t];
        b += (h[2 * u] - 2.0 * h[2 * u + 1] + rte[u]) / rte[u];
    }
    if (loss_first) *loss_first = a / w;
    if (loss_last) *loss_last = b / w;
    n->trained = true;
    return launch_check(c, "cnn train");
}

// Energy loss and parameter gradient of one sample (r, e = K^-1 r) on the
// context's grid.
to3d_status to3d_cnn_loss_grad(to3d_ctx* c, const double* x, const double* r, const double* e,
                               int32_t on_device, float* grad, int64_t ngrad, double* loss) {
    if (!c || !x || !r || !e || !c->cnn) return TO3D_EINVAL;
    Net* n = net_of(c);
    if (grad && ngrad != (int64_t)n->nparam) return TO3D_EINVAL;
    const size_t nb = c->g.nel * 8, db = 3 * c->g.nnode * 8;
    const long long ndof = 3 * c->g.nnode;
    cudaStream_t s = c->stream;
    const void *dx, *dr, *de;
    to3d_status st;
    if ((st = stage_input(c, x, nb, on_device, 0, &dx))) return st;
    if ((st = stage_input(c, r, db, on_device, 1, &dr))) return st;
    if ((st = stage_input(c, e, db, on_device, 2, &de))) return st;
    if (!alloc_work(n->trn, n->Zp, n->Yp, n->Xp, true))
        return set_err(c, TO3D_ENOMEM, "training workspace");
    const long long nv = (long long)n->Zp * n->Yp * n->Xp;
    if ((st = prepare_op(c, (const double*)dx))) return st;
    launch_mask_copy(c, s, (const double*)dr, c->tmp);
    k_scaled_norm2<<<blocks(c->g.nnode), 256, 0, s>>>(c->g.nnode, c->dinv, c->tmp, c->red,
                                                      n->dots + 4);
    k_dots<<<blocks(ndof), 256, 0, s>>>(ndof, c->tmp, (const double*)de, nullptr, nullptr, c->red,
                                        n->dots + 2);
    k_make_input<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(c->g, n->Zp, n->Yp, n->Xp, c->tmp,
                                                            c->dinv, (const double*)dx,
                                                            c->nodemask, n->dots + 4, n->trn.in);
    CK_RET(cudaMemcpyAsync(n->dots_h, n->dots, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
    CK_RET(cudaStreamSynchronize(s));
    const double rte = n->dots_h[2];
    if (!(rte > 0.0)) return set_err(c, TO3D_EINVAL, "r^T e must be positive");
    energy_pass(c, n->trn.in, c->tmp, (const double*)dx, rte, n->dots);
    CK_RET(cudaMemcpyAsync(n->dots_h, n->dots, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
    if (grad) CK_RET(cudaMemcpyAsync(grad, n->G, sizeof(float) * n->nparam, cudaMemcpyDeviceToHost, s));
    CK_RET(cudaStreamSynchronize(s));
    if (loss) *loss = (n->dots_h[0] - 2.0 * n->dots_h[1] + rte) / rte;
    return launch_check(c, "cnn loss/gradient");
}

// ---- single convolutions on caller buffers (device pointers), for tests
to3d_status to3d_conv3d_forward(int32_t Z, int32_t Y, int32_t X, int32_t C1, int32_t C2,
                                int32_t Cout, const void* in1, const void* in2, const void* W,
                                const float* bias, int32_t relu, float* out, void* stream) {
    if (Z < 1 || Y < 1 || X < 1 || C1 < 16 || C1 % 16 || C2 < 0 || C2 % 16 || Cout % 8 ||
        Cout < 8 || Cout > 128 || (Cout / 8 != 1 && Cout / 8 != 2 && Cout / 8 != 4 &&
                                   Cout / 8 != 6 && Cout / 8 != 8 && Cout / 8 != 12 &&
                                   Cout / 8 != 16) || !in1 || !W || !out || (C2 && !in2))
        return TO3D_EINVAL;
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    a.Z = Z; a.Y = Y; a.X = X;
    a.nvox = (long long)Z * Y * X;
    a.C1 = C1; a.C2 = C2; a.Cout = Cout;
    a.in1 = in1; a.in2 = in2;
    a.W = (const bf16*)W;
    a.bias = bias;
    a.out_f = out;
    a.out_cstride = Cout;
    a.relu = relu;
    conv_forward(a, false, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? TO3D_OK : TO3D_ECUDA;
}

to3d_status to3d_conv3d_backward(int32_t Z, int32_t Y, int32_t X, int32_t C1, int32_t C2,
                                 int32_t Cout, const void* x1, const void* x2, const void* W,
                                 const float* gy, const void* act, float* gx, float* gw, float* gb,
                                 void* stream) {
    const int Cin = C1 + C2;
    if (Z < 1 || Y < 1 || X < 1 || C1 < 16 || C1 % 16 || C2 < 0 || C2 % 16 || Cout % 16 ||
        Cout < 16 || Cout > 64 || Cin > 128 || !x1 || !W || !gy || !gw || (C2 && !x2))
        return TO3D_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const long long nvox = (long long)Z * Y * X;
    WgradArgs wa;
    wa.Z = Z; wa.Y = Y; wa.X = X;
    wa.nvox = nvox;
    wa.Cout = Cout;
    wa.Cin = Cin;
    wa.gy = gy;
    wa.gy_cstride = Cout;
    wa.mask = (const bf16*)act;
    wa.x1 = x1;
    wa.x2 = x2;
    wa.C1 = C1;
    wa.gw = gw;
    wa.Cout_fwd = Cout;
    wa.gb = gb;
    conv_wgrad(wa, false, s);
    if (gx) {
        bf16* Wt = nullptr;
        if (cudaMallocAsync((void**)&Wt, sizeof(bf16) * 27 * Cout * Cin, s) != cudaSuccess)
            return TO3D_ENOMEM;
        transpose_flip((const bf16*)W, Wt, Cout, Cin, s);
        ConvArgs a;
        std::memset(&a, 0, sizeof(a));
        a.Z = Z; a.Y = Y; a.X = X;
        a.nvox = nvox;
        a.C1 = Cout; a.C2 = 0; a.Cout = Cin;
        a.in1 = gy;
        a.mask1 = (const bf16*)act;
        a.W = Wt;
        a.out_f = gx;
        a.out_cstride = Cin;
        conv_forward(a, true, s);
        cudaFreeAsync(Wt, s);
    }
    return cudaGetLastError() == cudaSuccess ? TO3D_OK : TO3D_ECUDA;
}

}  // extern "C"
