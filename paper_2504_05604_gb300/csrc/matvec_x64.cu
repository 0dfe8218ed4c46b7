// FP64-accurate matrix-free K p on the tensor cores by exact integer slicing.
//
// y = Kbar p with K = sum_e E_e P_e^T KE P_e (Section 2.2), the FP64
// operator of the FP64 paths.  KE = c * B with B an integer matrix
// (|entries| <= 256) exact in FP16; the element vector p_e (FP64) is written
// as a fixed-point integer relative to its largest entry,
//     V_i = rint(p_i * 2^S),  S = 1073 - e_max,  e_max the largest biased
//     exponent in p_e,
// so |V_i| <= 2^51, and |V_i| is cut into five 11-bit slices d_0..d_4 (top
// first), each an integer of at most 2047 carrying the sign of V_i: exact in
// FP16.  One tcgen05 MMA per slice (M = 128 elements, N = 32, K = 32) gives
// B d_s exactly in FP32 (24 terms of at most 256 * 2047 stay below 2^24);
// the slices recombine exactly in 64-bit integers,
//     Y = ((((B d_0) 2^11 + B d_1) 2^11 + B d_2) 2^11 + B d_3) 2^11 + B d_4 = B V,
// |Y| <= 24 max|B| 2^51 < 2^63 for max|B| < 170 (88 for nu = 0.3), and
// y_e = (c E_e 2^-S) Y in FP64.  The only roundings are the
// fixed-point rounding of p_e (2^-52 of its largest entry), the conversion
// of Y to FP64 and the FP64 scaling and node sums: FP64 accuracy.  Needs the
// combined integer form of KE (a nu whose lambda / mu is a small rational,
// e.g. 0.3); the library uses the CUDA-core FP64 kernel otherwise.
//
// One CTA of 128 threads owns a 15 x 7 node column over a z segment and
// walks up it one element layer (16 x 8 elements, one thread each) at a
// time: node planes of p are staged in shared memory (clamped dofs as 0),
// each thread slices its element into the five A tiles, one thread issues
// the MMAs into five TMEM accumulators, every thread reads its row back,
// recombines and scales it, adds the upper-half outputs of the element
// below it (carried in registers) to its lower-half ones, and the owned
// nodes sum the four element columns around them in FP64.  Clamped dofs
// are identity rows (y = p).  Deterministic, no atomics.
#include "internal.cuh"
#include "reduce.cuh"
#include "tc.cuh"

namespace to3d {

constexpr int X64_BX = 15, X64_BY = 7;              // owned nodes per layer
constexpr int X64_EX = 16, X64_EY = 8;              // elements per layer
constexpr int X64_PX = 17, X64_PY = 9;              // staged nodes per plane
constexpr int X64_PLANE = X64_PX * X64_PY * 3;      // doubles per staged plane
constexpr int X64_THREADS = 128;
constexpr int X64_SLICES = 5;        // five accumulators of 32 TMEM columns: 256 allocated, 2 CTAs per SM
constexpr int X64_TILE = 128 * 64;                  // one 128 x 32 FP16 operand tile
constexpr uint32_t X64_WAIT_POLLS = 1u << 20;
static_assert(X64_EX * X64_EY == X64_THREADS, "one element per thread, one MMA row each");

struct X64Smem {
    static constexpr int A = 0;                                   // 5 tiles
    static constexpr int B = A + X64_SLICES * X64_TILE;           // 32 x 32 FP16
    static constexpr int P = B + 32 * 64;                         // 2 node planes
    static constexpr int Y = P + 2 * X64_PLANE * 8;               // [128][12] FP64
    static constexpr int BAR = Y + 128 * 12 * 8;
    static constexpr int TADDR = BAR + 8;
    static constexpr int USED = TADDR + 8;
    static constexpr int BYTES = 1024 + USED;
};

__device__ __forceinline__ int x64_kmaj(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

struct X64Args {
    Grid g;
    int lz, ntx, nty, ntz;
    double cscale;              // KE = cscale * B
    const uint8_t* Bimg;        // FP16 image of B (32 x 32, canonical layout)
    const double* E;
    const double* p;
    const uint8_t* nodemask;
    double* y;
    Reducer red;
    SolverScalars* ss;
    int dot_pq;
    double* ce;                 // energy form: ce_e = u_e^T KE u_e per element, no y
    int* err;
};

// ENERGY: element energies into a.ce instead of K p into a.y (a separate
// instantiation, so the K p form carries none of its code)
template <bool ENERGY>
__global__ void __launch_bounds__(X64_THREADS, 2) k_matvec_x64(const __grid_constant__ X64Args a) {
    if (a.dot_pq && a.ss->done) return;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = sm + X64Smem::A;
    uint8_t* sB = sm + X64Smem::B;
    double* sP = (double*)(sm + X64Smem::P);
    double* sY = (double*)(sm + X64Smem::Y);
    uint64_t* bar = (uint64_t*)(sm + X64Smem::BAR);
    uint32_t* s_taddr = (uint32_t*)(sm + X64Smem::TADDR);
    __shared__ double sh[32];
    __shared__ double dout[1];
    __shared__ int s_fail;
    const Grid& g = a.g;
    const int tid = threadIdx.x, warp = tid >> 5;

    const int tile = blockIdx.x;
    const int tz = tile % a.ntz, ty = (tile / a.ntz) % a.nty, tx = tile / (a.ntz * a.nty);
    const int i0 = tx * X64_BX, j0 = ty * X64_BY, k0 = tz * a.lz;
    const int nown = min(a.lz, g.nz - k0);

    if (warp == 0) {
        tc::tmem_alloc(s_taddr, 256);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        s_fail = 0;
        tc::fence_mbar_init();
    }
    for (int i = tid; i < 32 * 4; i += X64_THREADS)
        reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(a.Bimg)[i];
    // operand columns 24..31 stay zero
    for (int i = tid; i < X64_SLICES * 128; i += X64_THREADS)
        *reinterpret_cast<uint4*>(sA + (i / 128) * X64_TILE + x64_kmaj(i % 128, 24)) = make_uint4(0, 0, 0, 0);
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *s_taddr;

    // node plane gz of p into ring slot `slot` (nodes outside the grid as 0,
    // and clamped dofs too unless in energy mode)
    auto load_plane = [&](int gz, int slot) {
        double* dst = sP + slot * X64_PLANE;
        for (int idx = tid; idx < X64_PLANE; idx += X64_THREADS) {
            const int c = idx % 3, n = idx / 3, li = n % X64_PX, lj = n / X64_PX;
            const int gi = i0 - 1 + li, gj = j0 - 1 + lj;
            double v = 0.0;
            if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny && gz >= 0 && gz < g.nz) {
                const long long nd = node_id(g, gi, gj, gz);
                // energies take u as given; K p treats clamped dofs as 0
                if (ENERGY || !((a.nodemask[nd] >> c) & 1)) v = a.p[3 * nd + c];
            }
            dst[idx] = v;
        }
    };

    const int ei = tid % X64_EX, ej = tid / X64_EX;
    double dot = 0.0;
    double carry[12];          // upper-half outputs of this column's element below
#pragma unroll
    for (int i = 0; i < 12; ++i) carry[i] = 0.0;
    uint32_t phase = 0;
    load_plane(k0 - 1, (k0 - 1) & 1);
    for (int kk = k0 - 1; kk < k0 + nown; ++kk) {
        load_plane(kk + 1, (kk + 1) & 1);
        __syncthreads();
        // ---- this thread's element: gather, fixed-point, five slices
        const int gi = i0 - 1 + ei, gj = j0 - 1 + ej;
        const bool valid = gi >= 0 && gi < g.nelx && gj >= 0 && gj < g.nely && kk >= 0 && kk < g.nelz;
        // Fixed point from the bit patterns (integer operations only): with
        // e_max the largest biased exponent of the element, an entry of
        // biased exponent e and 53-bit significand m is m * 2^(e - 1075), and
        // V = rint(m * 2^(e - e_max - 2)), |V| <= 2^51; the scale is
        // 2^(e_max - 1073).  Two passes over the staged planes keep the
        // register count low.
        auto entry = [&](int i) -> unsigned long long {
            const int b = i / 3, c = i - 3 * b;
            const double* src = sP + ((kk + (b >> 2)) & 1) * X64_PLANE +
                                3 * ((ei + (b & 1)) + X64_PX * (ej + ((b >> 1) & 1)));
            return valid ? (unsigned long long)__double_as_longlong(src[c]) : 0ull;
        };
        int emax = 1;
#pragma unroll
        for (int i = 0; i < 24; ++i) emax = max(emax, (int)((entry(i) >> 52) & 0x7FF));
#pragma unroll
        for (int kc = 0; kc < 3; ++kc) {
            long long V[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const unsigned long long u = entry(8 * kc + q);
                int e = (int)((u >> 52) & 0x7FF);
                unsigned long long m = u & 0xFFFFFFFFFFFFFull;
                if (e) m |= 1ull << 52;
                else e = 1;
                const int sh = emax - e + 2;
                const unsigned long long mag = sh >= 63 ? 0ull : (m + (1ull << (sh - 1))) >> sh;
                V[q] = (u >> 63) ? -(long long)mag : (long long)mag;
            }
#pragma unroll
            for (int s = 0; s < X64_SLICES; ++s) {
                const int sh = 11 * (X64_SLICES - 1 - s);
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    float f2[2];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const long long x = V[2 * h + q];
                        const int d = (int)(((x < 0 ? -x : x) >> sh) & 0x7FF);
                        f2[q] = (float)(x < 0 ? -d : d);
                    }
                    __half2 hv = __floats2half2_rn(f2[0], f2[1]);
                    w[h] = *reinterpret_cast<uint32_t*>(&hv);
                }
                *reinterpret_cast<uint4*>(sA + s * X64_TILE + x64_kmaj(tid, 8 * kc)) =
                    make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        // ---- MMAs: accumulator s (TMEM columns 32 s ..) = A_s B^T
        if (tid == 0) {
            tc::tc_fence_after();
            const uint32_t idesc = tc::make_idesc_f16(128, 32, 0);
            const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
#pragma unroll
            for (int s = 0; s < X64_SLICES; ++s)
#pragma unroll
                for (int k2 = 0; k2 < 2; ++k2)
                    tc::mma_f16_ss(tmem + 32u * s,
                                   tc::make_desc_kmajor(a_addr + s * X64_TILE + k2 * 256, 128, 512),
                                   tc::make_desc_kmajor(b_addr + k2 * 256, 128, 512), idesc,
                                   k2 ? 1u : 0u);
            tc::mma_commit(bar);
        }
        if (!tc::mbar_wait_sleep_bounded(bar, phase, X64_WAIT_POLLS, 1000u)) s_fail = 1;
        phase ^= 1u;
        tc::tc_fence_after();
        // ---- recombine the slices exactly and scale; the lower-half corners
        // (c = 0) plus the carried upper halves of the element below in this
        // column give this column's part of node plane kk
        constexpr bool energy = ENERGY;
        const double Ee = energy ? 1.0 : (valid ? a.E[elem_id(g, gi, gj, kk)] : 0.0);
        double ce = 0.0;
        // an Inf or NaN entry (biased exponent 2047) makes the element's
        // outputs NaN, as the FP64 kernel would
        const double scl = emax == 2047 ? __longlong_as_double(0x7FF8000000000000ll)
                                        : ldexp(a.cscale * Ee, emax - 1073);
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        double* yrow = sY + tid * 12;
#pragma unroll
        for (int half = 0; half < 2; ++half) {     // outputs 0..11 (c = 0), 12..23 (c = 1)
            long long Y[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) Y[i] = 0;
#pragma unroll
            for (int s = 0; s < X64_SLICES; ++s) {
                float d0[16];
                tc::tmem_ld16_sync(trow + 32u * s + (half ? 8u : 0u), d0);
#pragma unroll
                for (int i = 0; i < 12; ++i) Y[i] = Y[i] * 2048 + (long long)__float2int_rn(d0[half ? i + 4 : i]);
            }
            if (energy) {
                // u_e^T (KE u_e): the element's own entries times its outputs
#pragma unroll
                for (int i = 0; i < 12; ++i)
                    ce = fma(__longlong_as_double((long long)entry(12 * half + i)), __ll2double_rn(Y[i]) * scl, ce);
            } else if (half == 0) {
#pragma unroll
                for (int i = 0; i < 12; ++i) yrow[i] = fma(__ll2double_rn(Y[i]), scl, carry[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 12; ++i) carry[i] = __ll2double_rn(Y[i]) * scl;
            }
        }
        // every element is owned by exactly one tile: the one whose element
        // column, row and layer it is past the halo (ei, ej >= 1, kk >= k0)
        if (energy && valid && ei >= 1 && ej >= 1 && kk >= k0) a.ce[elem_id(g, gi, gj, kk)] = ce;
        tc::tc_fence_before();
        __syncthreads();
        // ---- owned nodes of plane kk: the four element columns around them
        if (!energy && kk >= k0 && tid < X64_BX * X64_BY) {
            const int ni = 1 + tid % X64_BX, nj = 1 + tid / X64_BX;
            const int gni = i0 - 1 + ni, gnj = j0 - 1 + nj;
            if (gni < g.nx && gnj < g.ny) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa) {
                        const double* w = sY + ((ni - aa) + X64_EX * (nj - b)) * 12 + 3 * (aa + 2 * b);
                        s0 += w[0];
                        s1 += w[1];
                        s2 += w[2];
                    }
                const long long nd = node_id(g, gni, gnj, kk);
                const uint8_t m = a.nodemask[nd];
                const double* pn = a.p + 3 * nd;
                if (m & 1) s0 = pn[0];
                if (m & 2) s1 = pn[1];
                if (m & 4) s2 = pn[2];
                double* yn = a.y + 3 * nd;
                yn[0] = s0;
                yn[1] = s1;
                yn[2] = s2;
                if (a.dot_pq) dot += pn[0] * s0 + pn[1] * s1 + pn[2] * s2;
            }
        }
        // the next layer overwrites the staged plane kk and the shared
        // outputs only after every thread is past this point
        __syncthreads();
        if (s_fail) {
            // after a timeout: the MMAs of this layer must finish before TMEM
            // is freed (bounded as well)
            if (tid == 0) tc::mbar_wait_sleep_bounded(bar, phase ^ 1u, X64_WAIT_POLLS, 1000u);
            break;
        }
    }
    __syncthreads();
    if (s_fail && tid == 0) atomicExch(a.err, (int)TO3D_ETIMEOUT);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
    if (a.dot_pq) {
        double vv[1] = {dot};
        if (grid_sum<1>(a.red, vv, sh, dout) && tid == 0) {
            const double pq = dout[0];
            a.ss->pq = pq;
            if (*a.err != 0) {
                a.ss->status = *a.err;
                a.ss->done = 1;
            } else if (!(pq > 0.0) || !isfinite(pq)) {
                a.ss->status = TO3D_ENUMERIC;
                a.ss->done = 1;
                a.ss->alpha = 0.0;
            } else {
                a.ss->alpha = a.ss->rz / pq;
            }
        }
    }
}

// Whether the sliced tensor-core form serves this context: the combined
// integer KE with max |B| < 170 (so |B V| < 2^63), and few enough tiles for
// the reduction's partial slots.
bool matvec_x64_available(const to3d_ctx* c) {
    if (c->tc_split || c->tc_bmax >= 170.0) return false;
    const Grid& g = c->g;
    const int nseg = (g.nz + 19) / 20, lz = (g.nz + nseg - 1) / nseg;
    const long long tiles = (long long)((g.nx + X64_BX - 1) / X64_BX) * ((g.ny + X64_BY - 1) / X64_BY) *
                            ((g.nz + lz - 1) / lz);
    return tiles <= kMaxBlocks;
}

void launch_matvec_x64(to3d_ctx* c, cudaStream_t s, const double* E, const double* p, double* y,
                       bool dot_pq) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_matvec_x64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, X64Smem::BYTES);
        attr = true;
    }
    const Grid& g = c->g;
    X64Args a;
    a.g = g;
    const int nseg = (g.nz + 19) / 20;
    a.lz = (g.nz + nseg - 1) / nseg;
    a.ntx = (g.nx + X64_BX - 1) / X64_BX;
    a.nty = (g.ny + X64_BY - 1) / X64_BY;
    a.ntz = (g.nz + a.lz - 1) / a.lz;
    a.cscale = c->tc_cscale_d;
    a.Bimg = c->tcB + 32 * 64;      // FP16 image of the combined B
    a.E = E;
    a.p = p;
    a.nodemask = c->nodemask;
    a.y = y;
    a.red = c->red;
    a.ss = c->ss;
    a.dot_pq = dot_pq ? 1 : 0;
    a.ce = nullptr;
    a.err = c->dev_err;
    const int ntiles = a.ntx * a.nty * a.ntz;
    k_matvec_x64<false><<<ntiles, X64_THREADS, X64Smem::BYTES, s>>>(a);
    c->launches++;
}

// Element energies ce_e = u_e^T KE u_e (unit modulus) by the same exact
// slicing: the element's products B V recombined and scaled as for K u,
// dotted with the element's own FP64 entries (24 FP64 FMAs instead of 300).
void launch_energies_x64(to3d_ctx* c, cudaStream_t s, const double* u, double* ce) {
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_matvec_x64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, X64Smem::BYTES);
        attr = true;
    }
    const Grid& g = c->g;
    X64Args a;
    a.g = g;
    const int nseg = (g.nz + 19) / 20;
    a.lz = (g.nz + nseg - 1) / nseg;
    a.ntx = (g.nx + X64_BX - 1) / X64_BX;
    a.nty = (g.ny + X64_BY - 1) / X64_BY;
    a.ntz = (g.nz + a.lz - 1) / a.lz;
    a.cscale = c->tc_cscale_d;
    a.Bimg = c->tcB + 32 * 64;
    a.E = nullptr;
    a.p = u;
    a.nodemask = c->nodemask;
    a.y = nullptr;
    a.red = c->red;
    a.ss = c->ss;
    a.dot_pq = 0;
    a.ce = ce;
    a.err = c->dev_err;
    const int ntiles = a.ntx * a.nty * a.ntz;
    k_matvec_x64<true><<<ntiles, X64_THREADS, X64Smem::BYTES, s>>>(a);
    c->launches++;
}

}  // namespace to3d
