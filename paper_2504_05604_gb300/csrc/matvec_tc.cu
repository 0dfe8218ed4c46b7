// Low-precision element matvec on the tcgen05 tensor cores.
//
// y = K p with K = sum_e E_e P_e^T KE P_e (Section 2.2), evaluated element by
// element as a dense contraction: for a chunk of 128 elements the gathered
// element vectors form A (128 x 24, padded to K = 32) and the unit-modulus
// stiffness forms B.  KE is split as KE = c_lam A_lam + c_mu A_mu with
// integer A_lam, A_mu (|entries| <= 8 and <= 32), which are exact in BF16 and
// FP16, so B = [A_lam; A_mu] (N = 48) carries no rounding at all; the only
// rounding is in the 16-bit displacement operand and the FP32 accumulation.
// D = A B^T sits in TMEM (128 lanes x 48 FP32 columns); the epilogue combines
// c_lam D_lam + c_mu D_mu, scales by E_e in FP32 and scatter-adds into a
// shared-memory tile of the nodes the CTA owns.
//
// Tiling: a CTA owns a 15 x 7 x 7 block of nodes and evaluates the 16 x 8 x 8
// elements that touch them (one 128-element MMA chunk per element layer), so
// every node is written by exactly one CTA with a plain store: no global
// atomics, no zero-fill of y, deterministic results.
//
// Operand formats (prec):
//   1  BF16:    A = bf16(p_e)
//   2  BF16X2:  A_hi = bf16(p_e), A_lo = bf16(p_e - A_hi); D accumulates both
//   3  FP16:    p_e scaled by a power of two so max|p_e| lies in [2^10, 2^11)
//
// Fused mode (inner PCG): the CTA first forms the new search direction
// p_new = M^-1 r + beta p_old for its tile (halo included, written only for
// owned nodes), multiplies that, and reduces p_new . q into alpha.
#include "internal.cuh"
#include "reduce.cuh"
#include "tc.cuh"

namespace to3d {

constexpr int TC_BX = 15, TC_BY = 7, TC_BZ = 7;                      // owned nodes
constexpr int TC_EX = TC_BX + 1, TC_EY = TC_BY + 1, TC_EZ = TC_BZ + 1;  // elements
constexpr int TC_PX = TC_BX + 2, TC_PY = TC_BY + 2, TC_PZ = TC_BZ + 2;  // node tile
constexpr int TC_THREADS = 128;
constexpr int TC_N = 48;                  // MMA N: A_lam rows then A_mu rows
constexpr int TC_TMEM_COLS = 64;
constexpr int TC_A_BYTES = 128 * 64;      // one 128 x 32 16-bit operand tile
constexpr int TC_B_BYTES = TC_N * 64;
constexpr int TC_P_FLOATS = 3 * TC_PX * TC_PY * TC_PZ;
constexpr int TC_Y_FLOATS = 3 * TC_BX * TC_BY * TC_BZ;
static_assert(TC_EX * TC_EY == 128, "one element layer per MMA chunk");

__host__ __device__ constexpr int tc_smem_bytes(int nslice) {
    return 1024 /*align slack*/ + nslice * TC_A_BYTES + TC_B_BYTES + 4 * TC_P_FLOATS +
           4 * TC_Y_FLOATS + 64;
}

// byte offset of (row, k) in a K-major, no-swizzle operand tile with
// K = 32 (4 core matrices of 8 rows x 16 B per 8-row group)
__device__ __forceinline__ int kmaj_off(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

template <bool BF>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    if constexpr (BF) {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

// Write one 32-wide operand row (24 values + 8 zeros) into tile `tile`.
template <bool BF>
__device__ __forceinline__ void store_row(uint8_t* tile, int row, const float (&v)[24]) {
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
        uint4 w;
        if (kc < 3) {
            w.x = pack2<BF>(v[8 * kc + 0], v[8 * kc + 1]);
            w.y = pack2<BF>(v[8 * kc + 2], v[8 * kc + 3]);
            w.z = pack2<BF>(v[8 * kc + 4], v[8 * kc + 5]);
            w.w = pack2<BF>(v[8 * kc + 6], v[8 * kc + 7]);
        } else {
            w = make_uint4(0u, 0u, 0u, 0u);
        }
        *reinterpret_cast<uint4*>(tile + kmaj_off(row, 8 * kc)) = w;
    }
}

template <int PREC, bool FUSED>
__global__ void __launch_bounds__(TC_THREADS)
    k_matvec_tc(const __grid_constant__ KESplit kes, const Grid g, const float* __restrict__ E32,
                const float* __restrict__ p_in, const float* __restrict__ r,
                const float* __restrict__ dinv, const uint8_t* __restrict__ nodemask,
                float* __restrict__ p_new, float* __restrict__ q, const Reducer red,
                SolverScalars* ss, int* err) {
    constexpr int NSLICE = (PREC == 2) ? 2 : 1;
    constexpr bool BF = (PREC != 3);
    if (FUSED && ss->done) return;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = base;                                   // NSLICE * 8 KB
    uint8_t* sB = sA + NSLICE * TC_A_BYTES;               // 3 KB
    float* sP = (float*)(sB + TC_B_BYTES);                // node tile
    float* sY = sP + TC_P_FLOATS;                         // owned-node accumulators
    uint64_t* bar = (uint64_t*)(sY + TC_Y_FLOATS);
    uint32_t* s_taddr = (uint32_t*)(bar + 1);
    __shared__ double sh[32];
    __shared__ double dout[1];

    const int tid = threadIdx.x, warp = tid >> 5;
    const int i0 = blockIdx.x * TC_BX, j0 = blockIdx.y * TC_BY, k0 = blockIdx.z * TC_BZ;

    if (warp == 0) {
        tc::tmem_alloc(s_taddr, TC_TMEM_COLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    // B = [A_lam; A_mu] (N x K, K-major), integer entries, exact in 16 bits
    for (int idx = tid; idx < TC_N * 32; idx += TC_THREADS) {
        const int n = idx >> 5, k = idx & 31;
        float v = 0.f;
        if (k < 24) v = (n < 24) ? kes.a_lam[n * 24 + k] : kes.a_mu[(n - 24) * 24 + k];
        if (BF) *reinterpret_cast<__nv_bfloat16*>(sB + kmaj_off(n, k)) = __float2bfloat16_rn(v);
        else *reinterpret_cast<__half*>(sB + kmaj_off(n, k)) = __float2half_rn(v);
    }
    // node tile (clamped dofs and outside nodes as 0); fused: new direction
    const float beta = FUSED ? (float)ss->beta : 0.f;
    constexpr int ROW = 3 * TC_PX;
    for (int idx = tid; idx < TC_P_FLOATS; idx += TC_THREADS) {
        const int o = idx % ROW, rj = (idx / ROW) % TC_PY, rk = idx / (ROW * TC_PY);
        const int li = o / 3, c = o - 3 * li;
        const int gi = i0 - 1 + li, gj = j0 - 1 + rj, gk = k0 - 1 + rk;
        float v = 0.f;
        if (gi >= 0 && gi < g.nx && gj >= 0 && gj < g.ny && gk >= 0 && gk < g.nz) {
            const long long n = node_id(g, gi, gj, gk);
            const bool clamped = (nodemask[n] >> c) & 1;
            const long long d = 3 * n + c;
            if (FUSED) {
                if (!clamped) v = fmaf(dinv[n], r[d], beta * p_in[d]);
                const bool owned = li >= 1 && li <= TC_BX && rj >= 1 && rj <= TC_BY && rk >= 1 &&
                                   rk <= TC_BZ;
                if (owned) p_new[d] = v;
            } else if (!clamped) {
                v = p_in[d];
            }
        }
        sP[idx] = v;
    }
    for (int idx = tid; idx < TC_Y_FLOATS; idx += TC_THREADS) sY[idx] = 0.f;
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t taddr = *s_taddr;

    const uint32_t idesc = tc::make_idesc_f16(128, TC_N, BF ? 1 : 0);
    const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
    const float c_lam = (float)kes.c_lam, c_mu = (float)kes.c_mu;
    const int ei = tid % TC_EX, ej = tid / TC_EX;
    bool failed = false;

    for (int ek = 0; ek < TC_EZ; ++ek) {
        // gather the element vector from the node tile
        float v[24];
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int pi = ei + (b & 1), pj = ej + ((b >> 1) & 1), pk = ek + (b >> 2);
            const float* src = sP + 3 * (pi + TC_PX * (pj + TC_PY * pk));
            v[3 * b + 0] = src[0];
            v[3 * b + 1] = src[1];
            v[3 * b + 2] = src[2];
        }
        float inv_scale = 1.f;
        if (PREC == 3) {
            float m = 0.f;
#pragma unroll
            for (int i = 0; i < 24; ++i) m = fmaxf(m, fabsf(v[i]));
            if (m > 0.f) {
                int ex;
                frexpf(m, &ex);                    // m in [2^(ex-1), 2^ex)
                const float s = ldexpf(1.f, 11 - ex);
                inv_scale = ldexpf(1.f, ex - 11);
#pragma unroll
                for (int i = 0; i < 24; ++i) v[i] *= s;
            }
        }
        store_row<BF>(sA, tid, v);
        if (PREC == 2) {
            float lo[24];
#pragma unroll
            for (int i = 0; i < 24; ++i) lo[i] = v[i] - __bfloat162float(__float2bfloat16_rn(v[i]));
            store_row<BF>(sA + TC_A_BYTES, tid, lo);
        }
        tc::fence_proxy_async_smem();
        __syncthreads();
        tc::tc_fence_after();
        if (tid == 0) {
#pragma unroll
            for (int s = 0; s < NSLICE; ++s)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                    const uint64_t ad = tc::make_desc_kmajor(a_addr + s * TC_A_BYTES + kk * 256, 128, 512);
                    const uint64_t bd = tc::make_desc_kmajor(b_addr + kk * 256, 128, 512);
                    tc::mma_f16_ss(taddr, ad, bd, idesc, (s | kk) ? 1u : 0u);
                }
            tc::mma_commit(bar);
        }
        const bool ok = tc::mbar_wait_bounded(bar, (uint32_t)(ek & 1), 1u << 24);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::tc_fence_after();
        float d0[32], d1[16];
        const uint32_t trow = taddr + ((uint32_t)(warp * 32) << 16);
        tc::tmem_ld32_sync(trow, d0);
        tc::tmem_ld16_sync(trow + 32, d1);
        // element modulus (0 outside the grid)
        const int gei = i0 - 1 + ei, gej = j0 - 1 + ej, gek = k0 - 1 + ek;
        float Ee = 0.f;
        if (gei >= 0 && gei < g.nelx && gej >= 0 && gej < g.nely && gek >= 0 && gek < g.nelz)
            Ee = E32[elem_id(g, gei, gej, gek)];
        const float sc = Ee * inv_scale;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int li = ei + (b & 1), lj = ej + ((b >> 1) & 1), lk = ek + (b >> 2);
            if (li >= 1 && li <= TC_BX && lj >= 1 && lj <= TC_BY && lk >= 1 && lk <= TC_BZ) {
                float* dst = sY + 3 * ((li - 1) + TC_BX * ((lj - 1) + TC_BY * (lk - 1)));
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    const int rr = 3 * b + c;
                    const float dl = d0[rr];
                    const float dm = (rr + 24 < 32) ? d0[rr + 24] : d1[rr + 24 - 32];
                    atomicAdd(dst + c, sc * fmaf(c_lam, dl, c_mu * dm));
                }
            }
        }
        tc::tc_fence_before();
        __syncthreads();
    }

    // write the owned nodes; q = 0 (fused) or p (plain) on clamped dofs
    __syncthreads();
    double dot = 0.0;
    if (!failed) {
        constexpr int OROW = 3 * TC_BX;
        float part = 0.f;
        for (int idx = tid; idx < TC_Y_FLOATS; idx += TC_THREADS) {
            const int o = idx % OROW, lj = (idx / OROW) % TC_BY, lk = idx / (OROW * TC_BY);
            const int li = o / 3, c = o - 3 * li;
            const int gi = i0 + li, gj = j0 + lj, gk = k0 + lk;
            if (gi < g.nx && gj < g.ny && gk < g.nz) {
                const long long n = node_id(g, gi, gj, gk);
                const long long d = 3 * n + c;
                const bool clamped = (nodemask[n] >> c) & 1;
                float y = sY[idx];
                if (clamped) y = FUSED ? 0.f : p_in[d];
                q[d] = y;
                if (FUSED) {
                    const float pn = sP[3 * ((li + 1) + TC_PX * ((lj + 1) + TC_PY * (lk + 1))) + c];
                    part = fmaf(pn, y, part);
                }
            }
        }
        dot = part;
    } else if (tid == 0) {
        atomicExch(err, (int)TO3D_ETIMEOUT);
    }
    // release TMEM before the grid-wide reduction (only the last block continues)
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(taddr, TC_TMEM_COLS);

    if (FUSED) {
        double vv[1] = {dot};
        if (grid_sum<1>(red, vv, sh, dout) && tid == 0) {
            const double pq = dout[0];
            ss->pq = pq;
            if (*err != 0) {
                ss->status = *err;
                ss->done = 1;
            } else if (!(pq > 0.0) || !isfinite(pq)) {
                ss->status = TO3D_ENUMERIC;
                ss->done = 1;
                ss->alpha = 0.0;
            } else {
                ss->alpha = ss->rz / pq;
            }
        }
    }
}

template <int PREC, bool FUSED>
static void launch_one(to3d_ctx* c, cudaStream_t s, const float* E32, const float* p_in,
                       const float* r, const float* dinv, float* p_new, float* q) {
    constexpr int NSLICE = (PREC == 2) ? 2 : 1;
    const int smem = tc_smem_bytes(NSLICE);
    const Grid& g = c->g;
    dim3 grd((g.nx + TC_BX - 1) / TC_BX, (g.ny + TC_BY - 1) / TC_BY, (g.nz + TC_BZ - 1) / TC_BZ);
    k_matvec_tc<PREC, FUSED><<<grd, TC_THREADS, smem, s>>>(c->kes, g, E32, p_in, r, dinv,
                                                           c->nodemask, p_new, q, c->red, c->ss,
                                                           c->dev_err);
    c->launches++;
}

template <int PREC, bool FUSED>
static void set_attr() {
    cudaFuncSetAttribute(k_matvec_tc<PREC, FUSED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         tc_smem_bytes(PREC == 2 ? 2 : 1));
}

// Raise the dynamic shared-memory limit of every instance once, before any
// launch or graph capture.
void init_tc_attributes() {
    set_attr<1, false>(); set_attr<2, false>(); set_attr<3, false>();
    set_attr<1, true>(); set_attr<2, true>(); set_attr<3, true>();
}

void launch_matvec_tc(to3d_ctx* c, cudaStream_t s, const float* E32, const float* p_in,
                      const float* r, const float* dinv, float* p_new, float* q, int prec,
                      bool fused) {
    if (fused) {
        if (prec == TO3D_BF16X2_DC) launch_one<2, true>(c, s, E32, p_in, r, dinv, p_new, q);
        else if (prec == TO3D_FP16_DC) launch_one<3, true>(c, s, E32, p_in, r, dinv, p_new, q);
        else launch_one<1, true>(c, s, E32, p_in, r, dinv, p_new, q);
    } else {
        if (prec == TO3D_BF16X2_DC) launch_one<2, false>(c, s, E32, p_in, r, dinv, p_new, q);
        else if (prec == TO3D_FP16_DC) launch_one<3, false>(c, s, E32, p_in, r, dinv, p_new, q);
        else launch_one<1, false>(c, s, E32, p_in, r, dinv, p_new, q);
    }
}

}  // namespace to3d
