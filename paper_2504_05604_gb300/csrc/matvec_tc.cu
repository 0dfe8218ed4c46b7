// Low-precision element matvec on the tcgen05 tensor cores, fed by TMA.
//
// y = K p with K = sum_e E_e P_e^T KE P_e (Section 2.2), evaluated element by
// element as a dense contraction: for a layer of 128 elements the gathered
// element vectors form A (128 x 24, padded to K = 32) and the unit-modulus
// stiffness forms B.  KE = c_lam A_lam + c_mu A_mu with integer A_lam, A_mu;
// when c_lam / c_mu is a small rational a/b (nu = 0.3: 3/2) the single
// integer matrix a A_lam + b A_mu (|entries| <= 88) is B (N = 32, rows 24..31
// zero), otherwise B = [A_lam; A_mu] (N = 48) and the epilogue combines the
// halves.  Either way B is exact in BF16 and FP16: the only rounding is in
// the 16-bit displacement operand and the FP32 accumulation.
//
// Data layout: the FP32 vectors of the inner solve are stored per component
// ("structure of arrays") on a node grid whose x extent is padded to a
// multiple of 4, so every node row starts on a 16-byte boundary and a TMA
// box can start at any multiple of 4 nodes.  Pad nodes hold zeros.
//
// Work decomposition.  A persistent grid of 3 CTAs per SM; a CTA owns a
// 15 x 7 column of nodes over a segment of LZ node layers and walks up it
// one element layer at a time (16 x 8 = 128 elements: one M = 128 MMA).
// Node layers arrive by TMA into a ring of 6 or 7 stages (r, p_old and M^-1
// boxes of 20 x 9 nodes, all three components, plus the layer's moduli).
// Warp roles (details at TC_ROLE_THREADS):
//   TMA warp      issues the loads several layers ahead;
//   builder warps turn each node layer in place into the new search
//                 direction p_new = zcoef M^-1 r + beta p_old (plain mode: p
//                 itself), store the 16-byte chunks of owned node rows of
//                 p_new, gather each element's 24 values from two ring
//                 stages and write one A row in the operand format;
//   MMA warp      issues the MMAs into one of four TMEM accumulators;
//   epilogue      reads TMEM, scales each element row by E_e, assembles the
//                 nodes through warp shuffles and one shared-memory exchange
//                 per layer, carries the upper halves to the next layer in
//                 registers, stores q once per owned node and accumulates
//                 p_new^T q.
// Every node is written once, by the CTA that owns it, with a plain store:
// no atomics, no zero fill of y, deterministic results.  TMEM allocation,
// barrier set-up and the B tile load happen once per CTA.  Clamped dofs hold
// r = p = 0 in the inner solve, so the kernel needs no mask; the update
// kernel masks q.

// Every element vector is taken relative to its local node 0 before it is
// rounded (p_e - t_e with t_e the node-0 displacement repeated: KE t_e = 0),
// so the 16-bit rounding and the FP32 accumulation act on differences, which
// for the smooth fields of the slow CG modes are far smaller than the values.
//
// Operand formats (prec), applied to those differences:
//   1  BF16:    A = bf16(p_e)
//   2  BF16X2:  A_hi = bf16(p_e), A_lo = bf16(p_e - A_hi); D accumulates both
//   3  FP16:    p_e scaled by a power of two so max|p_e| lies in [2^10, 2^11)
//   4  FP16X2:  the scaled p_e as FP16 hi + lo slices (about 22 significant bits)
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "reduce.cuh"
#include "tc.cuh"

namespace to3d {

constexpr int TC_BX = 15, TC_BY = 7;                 // owned nodes per layer
constexpr int TC_EX = TC_BX + 1, TC_EY = TC_BY + 1;  // elements per layer (16 x 8)
constexpr int TC_PY = TC_BY + 2;                     // node rows per stage (9)
constexpr int TC_BOXX = 20;                          // nodes per stage row (17 needed + shift)
constexpr int TC_PLANE = TC_BOXX * TC_PY;            // 180 nodes per stage plane
constexpr int TC_VEC_BYTES = 3 * TC_PLANE * 4;       // one 3-component box (2160 B)
constexpr int TC_STAGE_R = 0;                        // byte offsets inside a stage
constexpr int TC_STAGE_P = 2176;
constexpr int TC_STAGE_D = 4352;
constexpr int TC_STAGE_E = 5120;                     // element moduli of the layer (20 x 8)
constexpr int TC_STAGE_BYTES = 5760;
constexpr int TC_EBOX_BYTES = TC_BOXX * TC_EY * 4;   // 640 B
constexpr int TC_STAGE_TX = 2 * TC_VEC_BYTES + TC_PLANE * 4 + TC_EBOX_BYTES;   // fused stage
constexpr int TC_STAGE_TX_PLAIN = TC_VEC_BYTES + TC_EBOX_BYTES;
constexpr int TC_A_BYTES = 128 * 64;                 // one 128 x 32 16-bit operand tile
static_assert(TC_EX * TC_EY == 128, "one element layer per MMA");

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

// One operand row: 24 values in three 16-byte chunks (the zero fourth chunk
// is written once per CTA).
template <bool BF>
__device__ __forceinline__ void store_row(uint8_t* tile, int row, const float (&v)[24]) {
#pragma unroll
    for (int kc = 0; kc < 3; ++kc) {
        uint4 w;
        w.x = pack2<BF>(v[8 * kc + 0], v[8 * kc + 1]);
        w.y = pack2<BF>(v[8 * kc + 2], v[8 * kc + 3]);
        w.z = pack2<BF>(v[8 * kc + 4], v[8 * kc + 5]);
        w.w = pack2<BF>(v[8 * kc + 6], v[8 * kc + 7]);
        *reinterpret_cast<uint4*>(tile + kmaj_off(row, 8 * kc)) = w;
    }
}

// --- TMA (bulk tensor copies into shared memory, completion on an mbarrier)
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc::smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            int w, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w),
        "r"(tc::smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(tc::smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(tc::smem_addr(bar))
        : "memory");
}

struct TcArgs {
    Grid g;
    int px;                   // padded x extent of the FP32 node grid
    long long plane, vol;     // px*ny, px*ny*nz
    int lz, ntx, nty, ntz, ntiles;
    float cscale;             // combined mode: scale of B
    float c_lam, c_mu;        // split mode
    const uint8_t* Bglob;     // prepared operand tile (NMMA x 32, canonical layout)
    const float* E32;
    float* p_new;
    float* q;
    Reducer red;
    SolverScalars* ss;
    int* err;
};

__device__ __forceinline__ void named_bar(int id, int n) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_addr(bar)) : "memory");
}
constexpr uint32_t TC_WAIT_POLLS = 1u << 20;

// Warp roles: warps 0-3 build (direction update + A rows), warps 4-7 run the
// epilogue (TMEM -> scaled rows -> node assembly), warp 8 lane 0 issues TMA,
// warp 9 lane 0 issues the MMAs.  (The two single-thread roles live in
// different warps: a lane spinning on an mbarrier can hold up the rest of
// its warp.)  Hand-offs use mbarriers:
//   full[s]/empty[s]  node-layer stage s loaded / released (builders + epilogue)
//   conv[s]           stage s holds the converted direction p_new
//   afull/aempty[b]   A tile b written / consumed by the MMA
//   dfull/dempty[b]   TMEM accumulator b written / read out
// Barrier phases follow running counters of node layers (G) and element
// layers (H) that every role advances identically tile after tile.
constexpr int TC_ROLE_THREADS = 320;
constexpr int TC_CTAS_PER_SM = 3;

template <int NSL, int NMMA>
struct TcSmemWs {
    static constexpr int NS = (NSL == 1) ? 7 : 6;                 // ring stages
    static constexpr int STAGES = 0;
    static constexpr int A = STAGES + NS * TC_STAGE_BYTES;
    static constexpr int B = A + 2 * NSL * TC_A_BYTES;
    static constexpr int Z = B + NMMA * 64;                       // [2][4 warps][16][6] floats
    static constexpr int BAR = Z + 2 * 4 * 16 * 6 * 4;
    static constexpr int NBAR = 3 * NS + 4 + 2 * 4;
    static constexpr int TADDR = BAR + 8 * NBAR;
    static constexpr int USED = TADDR + 16;
    static constexpr int BYTES = 1024 + USED;
};

template <int PREC, bool FUSED, bool SPLIT>
__global__ void __launch_bounds__(TC_ROLE_THREADS, TC_CTAS_PER_SM)
    k_matvec_tc(const __grid_constant__ TcArgs a, const __grid_constant__ CUtensorMap tm_r,
                const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_d,
                const __grid_constant__ CUtensorMap tm_e) {
    constexpr int NSL = (PREC == 2 || PREC == 4) ? 2 : 1;
    constexpr bool BF = (PREC == 1 || PREC == 2);
    constexpr bool SCALED = (PREC == 3 || PREC == 4);
    constexpr int NMMA = SPLIT ? 64 : 32;            // split: A_lam rows, A_mu rows, 16 spare
    constexpr int TCOLS = SPLIT ? 64 : 32;           // TMEM columns per accumulator
    // accumulators in flight: 4 x 32 columns (3 CTAs per SM use 384 of the
    // 512 TMEM columns); the split form's 64-column ones allow 2
    constexpr int ND = SPLIT ? 2 : 4;
    using L = TcSmemWs<NSL, NMMA>;
    constexpr int NS = L::NS;
    if (a.ss && a.ss->done) return;

    extern __shared__ uint8_t smem_raw[];
    uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* stages = sm + L::STAGES;
    uint8_t* sA = sm + L::A;
    uint8_t* sB = sm + L::B;
    float* sZ = (float*)(sm + L::Z);
    uint64_t* full = (uint64_t*)(sm + L::BAR);
    uint64_t* empty = full + NS;
    uint64_t* conv = empty + NS;
    uint64_t* afull = conv + NS;
    uint64_t* aempty = afull + 2;
    uint64_t* dfull = aempty + 2;
    uint64_t* dempty = dfull + ND;
    uint32_t* s_taddr = (uint32_t*)(sm + L::TADDR);
    __shared__ double sh[32];
    __shared__ double dout[1];
    __shared__ int s_fail;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const Grid& g = a.g;

    if (warp == 0) {
        tc::tmem_alloc(s_taddr, ND * TCOLS);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&full[i], 1);
            tc::mbar_init(&empty[i], 8);      // one arrival per builder and epilogue warp
            tc::mbar_init(&conv[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&afull[i], 4);      // one arrival per builder warp
            tc::mbar_init(&aempty[i], 1);
        }
        for (int i = 0; i < ND; ++i) {
            tc::mbar_init(&dfull[i], 1);
            tc::mbar_init(&dempty[i], 4);     // one arrival per epilogue warp
        }
        s_fail = 0;
        tc::fence_mbar_init();
    }
    for (int i = tid; i < NMMA * 4; i += TC_ROLE_THREADS)
        reinterpret_cast<uint4*>(sB)[i] = reinterpret_cast<const uint4*>(a.Bglob)[i];
    for (int i = tid; i < 2 * NSL * 128; i += TC_ROLE_THREADS) {
        const int t = i / 128, row = i % 128;
        *reinterpret_cast<uint4*>(sA + t * TC_A_BYTES + kmaj_off(row, 24)) = make_uint4(0, 0, 0, 0);
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *s_taddr;
    const float beta = FUSED ? (float)a.ss->beta : 0.f;
    const float zcoef = FUSED ? (float)a.ss->zcoef : 1.f;
    constexpr uint32_t STAGE_TX = FUSED ? TC_STAGE_TX : TC_STAGE_TX_PLAIN;
    volatile int* vfail = &s_fail;
    double dot = 0.0;

    // Waits suspend the warp (up to 1 us per poll) rather than spin, so
    // waiting roles leave the issue slots to the working ones; 2^20 polls
    // bound a wait to about a second even if suspension were not honoured
    // for the full hint.
    auto wait = [&](uint64_t* bar, uint32_t par) -> bool {
        if (*vfail) return false;
        if (tc::mbar_wait_sleep_bounded(bar, par, TC_WAIT_POLLS, 1000u)) return true;
        *vfail = 1;
        return false;
    };
    auto tile_geom = [&](int tile, int& i0, int& j0, int& k0, int& nown) {
        const int tz = tile % a.ntz, ty = (tile / a.ntz) % a.nty, tx = tile / (a.ntz * a.nty);
        i0 = tx * TC_BX;
        j0 = ty * TC_BY;
        k0 = tz * a.lz;
        nown = min(a.lz, g.nz - k0);
    };

    if (warp == 8) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            uint32_t G = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                int i0, j0, k0, nown;
                tile_geom(tile, i0, j0, k0, nown);
                const int xs = ((i0 - 1) >= 0) ? ((i0 - 1) & ~3) : -4;
                for (int m = 0; m < nown + 2; ++m, ++G) {
                    const int s = G % NS;
                    if (!wait(&empty[s], ((G / NS) & 1u) ^ 1u)) break;
                    uint8_t* st = stages + s * TC_STAGE_BYTES;
                    tc::fence_proxy_async_smem();
                    mbar_expect_tx(&full[s], STAGE_TX);
                    const int gz = k0 - 1 + m;
                    if (FUSED) {
                        tma_load_4d(st + TC_STAGE_R, &tm_r, xs, j0 - 1, gz, 0, &full[s]);
                        tma_load_4d(st + TC_STAGE_P, &tm_p, xs, j0 - 1, gz, 0, &full[s]);
                        tma_load_3d(st + TC_STAGE_D, &tm_d, xs, j0 - 1, gz, &full[s]);
                    } else {
                        tma_load_4d(st + TC_STAGE_P, &tm_p, xs, j0 - 1, gz, 0, &full[s]);
                    }
                    // element layer with the same z index (elements k0-1+m)
                    tma_load_3d(st + TC_STAGE_E, &tm_e, xs, j0 - 1, gz, &full[s]);
                }
                if (*vfail) break;
            }
            if (*vfail) {
                // after a timeout: let the copies already issued land before
                // the CTA (and its shared memory) goes away; bounded as well
                const uint32_t first = G > (uint32_t)NS ? G - (uint32_t)NS : 0u;
                for (uint32_t k = first; k < G; ++k)
                    tc::mbar_wait_sleep_bounded(&full[k % NS], (k / NS) & 1u, TC_WAIT_POLLS, 1000u);
            }
        }
    } else if (warp == 9) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = tc::make_idesc_f16(128, NMMA, BF ? 1 : 0);
            const uint32_t a_addr = tc::smem_addr(sA), b_addr = tc::smem_addr(sB);
            uint32_t H = 0, issued = 0;
            for (int tile = blockIdx.x; tile < a.ntiles && !*vfail; tile += gridDim.x) {
                int i0, j0, k0, nown;
                tile_geom(tile, i0, j0, k0, nown);
                for (int l = 0; l <= nown; ++l, ++H) {
                    const int b = H & 1, db = H % ND;
                    if (!wait(&afull[b], (H >> 1) & 1u)) break;
                    if (!wait(&dempty[db], ((H / ND) & 1u) ^ 1u)) break;
                    tc::tc_fence_after();
                    const uint32_t d_tmem = tmem + (uint32_t)(db * TCOLS);
#pragma unroll
                    for (int s = 0; s < NSL; ++s)
#pragma unroll
                        for (int kk = 0; kk < 2; ++kk) {
                            const uint32_t aoff = (uint32_t)((b * NSL + s) * TC_A_BYTES + kk * 256);
                            tc::mma_f16_ss(d_tmem, tc::make_desc_kmajor(a_addr + aoff, 128, 512),
                                           tc::make_desc_kmajor(b_addr + kk * 256, 128, 512), idesc,
                                           (s | kk) ? 1u : 0u);
                        }
                    tc::mma_commit(&dfull[db]);
                    tc::mma_commit(&aempty[b]);
                    issued = H + 1;
                }
            }
            if (*vfail && issued) {
                // after a timeout: the last MMAs must finish before TMEM is freed
                const uint32_t h = issued - 1;
                tc::mbar_wait_sleep_bounded(&aempty[h & 1], (h >> 1) & 1u, TC_WAIT_POLLS, 1000u);
            }
        }
    } else if (warp < 4) {
        // ------------------------------------------------ builders
        const int ei = tid % TC_EX, ej = tid / TC_EX;
        uint32_t G = 0, H = 0;
        // Each thread converts the float4 chunks idx = tid and tid + 128 of
        // a stage (3 components x 9 rows x 5 chunks).  A chunk of an owned
        // node row that holds at least one owned node is stored whole to
        // p_new: it is 16-byte aligned in global memory (the box starts on a
        // multiple of 4 nodes), and its other nodes are halo or pad nodes
        // whose values the owning tile computes bit for bit the same.
        constexpr int Q = TC_PLANE / 4;
        long long goff[2];
        auto convert = [&](uint32_t Gm, int m, int k0, int nown) -> bool {
            const int s = Gm % NS;
            if (!wait(&full[s], (Gm / NS) & 1u)) return false;
            if (FUSED) {
                uint8_t* st = stages + s * TC_STAGE_BYTES;
                float4* P = (float4*)(st + TC_STAGE_P);
                const float4* R = (const float4*)(st + TC_STAGE_R);
                const float4* D = (const float4*)(st + TC_STAGE_D);
                const bool owned_layer = m >= 1 && m <= nown;
                const long long zoff = a.plane * (long long)(k0 - 1 + m);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int idx = tid + 128 * k;
                    if (idx < 3 * Q) {
                        const int c = idx / Q, rem = idx - c * Q;
                        const float4 d4 = D[rem], r4 = R[idx], p4 = P[idx];
                        float4 v;
                        v.x = fmaf(zcoef * d4.x, r4.x, beta * p4.x);
                        v.y = fmaf(zcoef * d4.y, r4.y, beta * p4.y);
                        v.z = fmaf(zcoef * d4.z, r4.z, beta * p4.z);
                        v.w = fmaf(zcoef * d4.w, r4.w, beta * p4.w);
                        P[idx] = v;
                        if (owned_layer && goff[k] >= 0)
                            *reinterpret_cast<float4*>(a.p_new + goff[k] + zoff) = v;
                    }
                }
            }
            return true;
        };
        for (int tile = blockIdx.x; tile < a.ntiles && !*vfail; tile += gridDim.x) {
            int i0, j0, k0, nown;
            tile_geom(tile, i0, j0, k0, nown);
            const int xs = ((i0 - 1) >= 0) ? ((i0 - 1) & ~3) : -4;
            const int xo = (i0 - 1) - xs;
            const uint32_t Gb = G;
            if (FUSED) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    goff[k] = -1;
                    const int idx = tid + 128 * k;
                    if (idx < 3 * Q) {
                        const int c = idx / Q, rem = idx - c * Q;
                        const int yy = rem / (TC_BOXX / 4), x0 = 4 * (rem - yy * (TC_BOXX / 4));
                        const int gj = j0 - 1 + yy, gx = xs + x0;
                        // local node index li = x0 + u - xo; owned: 1 <= li <= 15, gi < nx
                        const int lo_li = max(x0 - xo, 1), hi_li = min(x0 + 3 - xo, TC_BX);
                        const bool any_owned = lo_li <= hi_li && i0 - 1 + lo_li < g.nx;
                        if (yy >= 1 && yy <= TC_BY && gj < g.ny && gx >= 0 && gx < a.px && any_owned)
                            goff[k] = c * a.vol + (long long)a.px * gj + gx;
                    }
                }
            }
            bool ok = convert(Gb, 0, k0, nown) && convert(Gb + 1, 1, k0, nown);
            named_bar(1, 128);
            if (!ok || *vfail) break;
            if (tid == 0) {
                mbar_arrive(&conv[Gb % NS]);
                mbar_arrive(&conv[(Gb + 1) % NS]);
            }
            for (int l = 0; l <= nown; ++l, ++H) {
                if (l >= 1) {
                    ok = convert(Gb + l + 1, l + 1, k0, nown);
                    named_bar(1, 128);
                    if (!ok || *vfail) break;
                    if (tid == 0) mbar_arrive(&conv[(Gb + l + 1) % NS]);
                }
                const int b = H & 1;
                if (!wait(&aempty[b], ((H >> 1) & 1u) ^ 1u)) break;
                const float* lo = (const float*)(stages + ((Gb + l) % NS) * TC_STAGE_BYTES + TC_STAGE_P);
                const float* hi = (const float*)(stages + ((Gb + l + 1) % NS) * TC_STAGE_BYTES + TC_STAGE_P);
                float v[24];
#pragma unroll
                for (int bb = 0; bb < 8; ++bb) {
                    const float* src = ((bb >> 2) ? hi : lo) +
                                       (xo + ei + (bb & 1)) + TC_BOXX * (ej + ((bb >> 1) & 1));
                    v[3 * bb + 0] = src[0];
                    v[3 * bb + 1] = src[TC_PLANE];
                    v[3 * bb + 2] = src[2 * TC_PLANE];
                }
                // KE annihilates rigid translations, so the element vector
                // may be taken relative to its local node 0: for smooth
                // fields the differences are much smaller than the values,
                // and so are their 16-bit rounding and the FP32 accumulation
                // errors (the product itself is unchanged)
#pragma unroll
                for (int i = 3; i < 24; ++i) v[i] -= v[i % 3];
                v[0] = v[1] = v[2] = 0.f;
                float code = 0.f;
                if (SCALED) {
                    float m = 0.f;
#pragma unroll
                    for (int i = 0; i < 24; ++i) m = fmaxf(m, fabsf(v[i]));
                    int ex = 0;
                    frexpf(m, &ex);
                    // scale by 2^(11-ex); vectors below 2^-100 (the inner solve
                    // runs at unit RMS) are dropped.  The exponent code ex-11
                    // rides in operand column 24, which B copies exactly into
                    // an otherwise unused accumulator column for the epilogue.
                    float sc = 0.f;
                    if (m > 0.f && ex > -100) {
                        sc = ldexpf(1.f, 11 - ex);
                        code = (float)(ex - 11);
                    }
#pragma unroll
                    for (int i = 0; i < 24; ++i) v[i] *= sc;
                }
                uint8_t* At = sA + b * NSL * TC_A_BYTES;
                store_row<BF>(At, tid, v);
                if (SCALED)
                    *reinterpret_cast<uint4*>(At + kmaj_off(tid, 24)) = make_uint4(pack2<BF>(code, 0.f), 0u, 0u, 0u);
                if (NSL == 2) {
                    float r2[24];
#pragma unroll
                    for (int i = 0; i < 24; ++i)
                        r2[i] = BF ? v[i] - __bfloat162float(__float2bfloat16_rn(v[i]))
                                   : v[i] - __half2float(__float2half_rn(v[i]));
                    store_row<BF>(At + TC_A_BYTES, tid, r2);
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&afull[b]);
                    mbar_arrive(&empty[(Gb + l) % NS]);
                    if (l == nown) mbar_arrive(&empty[(Gb + l + 1) % NS]);
                }
            }
            G = Gb + nown + 2;
        }
    } else {
        // ------------------------------------------------ epilogue (warps 4-7)
        const int et = tid - 128;                       // TMEM lane = element of the layer
        const int ei = et % TC_EX, ej = et / TC_EX;
        const int ew = warp - 4;
        // this lane finishes node (ei, 2 ew + 1 + upper-half) of every layer
        const bool node_thread = ei >= 1 && !(lane >= 16 && ew == 3);
        uint32_t G = 0, H = 0;
        for (int tile = blockIdx.x; tile < a.ntiles && !*vfail; tile += gridDim.x) {
            int i0, j0, k0, nown;
            tile_geom(tile, i0, j0, k0, nown);
            const int xs = ((i0 - 1) >= 0) ? ((i0 - 1) & ~3) : -4;
            const int xo = (i0 - 1) - xs;
            const uint32_t Gb = G;
            float carry0 = 0.f, carry1 = 0.f, carry2 = 0.f, tdot = 0.f;
            // this thread's node: row nrow_t of the tile, global (gi, gj); q
            // index of node layer 0 of the tile (one plane per layer above)
            const int nrow_t = 2 * ew + 1 + (lane >= 16 ? 1 : 0);
            const int gi_t = i0 + ei - 1, gj_t = j0 + nrow_t - 1;
            const bool store_node = node_thread && gi_t < g.nx && gj_t < g.ny;
            const long long qoff = gi_t + (long long)a.px * (gj_t + (long long)g.ny * (k0 - 1));
            bool ok = true;
            for (int l = 0; l <= nown; ++l, ++H) {
                const int db = H % ND;
                if (!wait(&dfull[db], (H / ND) & 1u)) { ok = false; break; }
                tc::tc_fence_after();
                const uint32_t trow = tmem + (uint32_t)(db * TCOLS) + ((uint32_t)(ew * 32) << 16);
                float dcol[SPLIT ? 64 : 32];
                if (SPLIT) {
                    float d0[32], d1[32];
                    tc::tmem_ld32_sync(trow, d0);
                    tc::tmem_ld32_sync(trow + 32, d1);
#pragma unroll
                    for (int r = 0; r < 32; ++r) {
                        dcol[r] = d0[r];
                        dcol[32 + r] = d1[r];
                    }
                } else {
                    float d0[16], d1[16];
                    tc::tmem_ld16_sync(trow, d0);
                    tc::tmem_ld16_sync(trow + 16, d1);
#pragma unroll
                    for (int r = 0; r < 16; ++r) {
                        dcol[r] = d0[r];
                        dcol[16 + r] = d1[r];
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&dempty[db]);
                const uint32_t Gl = Gb + l;
                if (!wait(&full[Gl % NS], (Gl / NS) & 1u)) { ok = false; break; }
                float Ecur = reinterpret_cast<const float*>(stages + (Gl % NS) * TC_STAGE_BYTES +
                                                            TC_STAGE_E)[(xo + ei) + TC_BOXX * ej];
                if (SCALED) Ecur *= ldexpf(1.f, (int)dcol[SPLIT ? 48 : 24]);
                float y[24];
                if (SPLIT) {
#pragma unroll
                    for (int r = 0; r < 24; ++r) y[r] = Ecur * fmaf(a.c_lam, dcol[r], a.c_mu * dcol[24 + r]);
                } else {
                    const float s2 = Ecur * a.cscale;
#pragma unroll
                    for (int r = 0; r < 24; ++r) y[r] = s2 * dcol[r];
                }
                // Node assembly through registers.  Lane = ei + 16 * (ej & 1);
                // y[3 (a + 2b + 4c) + comp] is this element's contribution to
                // its local node (a, b, c).
                // x: node (ei, ej+b, c) = a=0 part here + a=1 part of element ei-1
                float X[2][2][3];
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                        for (int k = 0; k < 3; ++k) {
                            const float left = __shfl_up_sync(0xffffffffu, y[3 * (1 + 2 * bb + 4 * cc) + k], 1, 16);
                            X[bb][cc][k] = y[3 * (2 * bb + 4 * cc) + k] + (ei > 0 ? left : 0.f);
                        }
                // y: lower half-warp (element row 2w) finishes node row 2w+1 with
                // the upper half's b = 0 parts; the upper half (row 2w+1)
                // finishes node row 2w+2 with the next warp's lower b = 0 parts
                const bool upper = lane >= 16;
                // double-buffered by layer parity: one barrier per layer
                // orders the writes before the reads, and a warp can only
                // rewrite a buffer after every warp passed the next barrier
                float* sZb = sZ + (H & 1) * (4 * 16 * 6);
                float N[2][3];
#pragma unroll
                for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const float v = __shfl_down_sync(0xffffffffu, X[0][cc][k], 16);
                        N[cc][k] = X[1][cc][k] + (upper ? 0.f : v);
                    }
                if (!upper) {
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                        for (int k = 0; k < 3; ++k) sZb[(ew * 16 + ei) * 6 + 3 * cc + k] = X[0][cc][k];
                }
                named_bar(2, 128);
                if (upper && ew < 3) {
#pragma unroll
                    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
                        for (int k = 0; k < 3; ++k) N[cc][k] += sZb[((ew + 1) * 16 + ei) * 6 + 3 * cc + k];
                }
                // z: node layer l = carry (c = 1 halves of layer l-1) + c = 0 halves
                const float s0 = carry0 + N[0][0], s1 = carry1 + N[0][1], s2 = carry2 + N[0][2];
                carry0 = N[1][0];
                carry1 = N[1][1];
                carry2 = N[1][2];
                if (store_node && l >= 1) {
                    {
                        const long long pidx = qoff + a.plane * (long long)l;
                        a.q[pidx] = s0;
                        a.q[pidx + a.vol] = s1;
                        a.q[pidx + 2 * a.vol] = s2;
                        if (FUSED) {
                            const uint32_t Gm = Gb + l;
                            if (!wait(&conv[Gm % NS], (Gm / NS) & 1u)) ok = false;
                            const float* pn = (const float*)(stages + (Gm % NS) * TC_STAGE_BYTES + TC_STAGE_P) +
                                              (xo + ei) + TC_BOXX * nrow_t;
                            tdot = fmaf(pn[0], s0, fmaf(pn[TC_PLANE], s1, fmaf(pn[2 * TC_PLANE], s2, tdot)));
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(Gb + l) % NS]);
                if (!ok) break;
            }
            if (!ok) break;
            if (lane == 0) mbar_arrive(&empty[(Gb + nown + 1) % NS]);
            dot += (double)tdot;
            G = Gb + nown + 2;
        }
    }
    __syncthreads();
    if (s_fail && tid == 0) atomicExch(a.err, (int)TO3D_ETIMEOUT);
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    if (warp == 0) tc::tmem_dealloc(tmem, ND * TCOLS);

    if (FUSED) {
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

// ------------------------------------------------------------------ layout helpers
// AoS (unpadded, 3 comps per node) FP32 -> padded SoA with clamped dofs zeroed.
__global__ void k_aos_to_soa(const Grid g, int px, long long vol, const float* __restrict__ in,
                             const uint8_t* __restrict__ nodemask, float* __restrict__ out) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nnode) return;
    const int i = n % g.nx;
    const long long jk = n / g.nx;
    const long long p = i + (long long)px * jk;
    const uint8_t m = nodemask[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) out[c * vol + p] = ((m >> c) & 1) ? 0.f : in[3 * n + c];
}

// padded SoA q -> AoS y; clamped rows are identity rows (y = p)
__global__ void k_soa_to_aos(const Grid g, int px, long long vol, const float* __restrict__ q,
                             const float* __restrict__ p, const uint8_t* __restrict__ nodemask,
                             float* __restrict__ y) {
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (n >= g.nnode) return;
    const int i = n % g.nx;
    const long long jk = n / g.nx;
    const long long pp = i + (long long)px * jk;
    const uint8_t m = nodemask[n];
#pragma unroll
    for (int c = 0; c < 3; ++c) y[3 * n + c] = ((m >> c) & 1) ? p[3 * n + c] : q[c * vol + pp];
}

// ------------------------------------------------------------------ host side
template <int PREC, bool FUSED, bool SPLIT>
static void set_attr_one() {
    constexpr int NSL = (PREC == 2 || PREC == 4) ? 2 : 1;
    cudaFuncSetAttribute(k_matvec_tc<PREC, FUSED, SPLIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         TcSmemWs<NSL, SPLIT ? 64 : 32>::BYTES);
}

template <bool FUSED, bool SPLIT>
static void set_attr_prec() {
    set_attr_one<1, FUSED, SPLIT>();
    set_attr_one<2, FUSED, SPLIT>();
    set_attr_one<3, FUSED, SPLIT>();
    set_attr_one<4, FUSED, SPLIT>();
}

void init_tc_attributes() {
    set_attr_prec<false, false>();
    set_attr_prec<false, true>();
    set_attr_prec<true, false>();
    set_attr_prec<true, true>();
}

static inline int host_kmaj_off(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

static PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// 4D map over a 3-component padded SoA vector (x, y, z, component) with box
// 20 x 9 x 1 x 3, or the 3D map of a per-node array (box 20 x 9 x 1).
static bool encode_map(to3d_ctx* c, CUtensorMap* map, const float* base, int comps,
                       bool elements = false) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
    if (!enc) return false;
    const Grid& g = c->g;
    const cuuint64_t X = elements ? c->pex : c->px, Y = elements ? g.nely : g.ny,
                     Z = elements ? g.nelz : g.nz;
    cuuint64_t dims[4] = {X, Y, Z, 3};
    cuuint64_t strides[3] = {X * 4, X * Y * 4, X * Y * Z * 4};
    cuuint32_t box[4] = {TC_BOXX, (cuuint32_t)(elements ? TC_EY : TC_PY), 1, 3};
    cuuint32_t es[4] = {1, 1, 1, 1};
    const cuuint32_t rank = comps == 3 ? 4 : 3;
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, rank, (void*)base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

// Prepare the B operand images, z segmentation and TMA descriptors once per context.
bool prepare_tc_operands(to3d_ctx* c) {
    const double ratio = c->kes.c_lam / c->kes.c_mu;
    int ca = 0, cb = 0;
    for (int b = 1; b <= 16 && !cb; ++b) {
        const double av = ratio * b;
        const double ar = std::nearbyint(av);
        if (std::fabs(av - ar) < 1e-9 * std::fmax(1.0, av)) {
            float mx = 0.f;
            for (int k = 0; k < 576; ++k)
                mx = std::fmax(mx, std::fabs((float)ar * c->kes.a_lam[k] + (float)b * c->kes.a_mu[k]));
            if (mx <= 256.f) {
                ca = (int)ar;
                cb = b;
            }
        }
    }
    c->tc_split = (cb == 0);
    c->tc_cscale = c->tc_split ? 1.0f : (float)(c->kes.c_mu / cb);
    c->tc_cscale_d = c->tc_split ? 1.0 : c->kes.c_mu / cb;
    c->tc_bmax = 0.0;
    if (!c->tc_split)
        for (int k = 0; k < 576; ++k)
            c->tc_bmax = std::fmax(c->tc_bmax, std::fabs((double)ca * c->kes.a_lam[k] + (double)cb * c->kes.a_mu[k]));
    const int nmma = c->tc_split ? 64 : 32;
    // the spare row 24 (combined) or 48 (split) copies operand column 24 (the
    // per-element exponent code of the FP16 form) into the accumulator
    const int code_row = c->tc_split ? 48 : 24;
    std::vector<uint16_t> hb(nmma * 32, 0), hh(nmma * 32, 0);
    for (int n = 0; n < nmma; ++n)
        for (int k = 0; k < 32; ++k) {
            float v = (n == code_row && k == 24) ? 1.f : 0.f;
            if (k < 24) {
                if (c->tc_split) {
                    if (n < 24) v = c->kes.a_lam[n * 24 + k];
                    else if (n < 48) v = c->kes.a_mu[(n - 24) * 24 + k];
                } else if (n < 24) {
                    v = (float)ca * c->kes.a_lam[n * 24 + k] + (float)cb * c->kes.a_mu[n * 24 + k];
                }
            }
            const __nv_bfloat16 bv = __float2bfloat16(v);
            const __half hv = __float2half(v);
            const int off = host_kmaj_off(n, k) / 2;
            hb[off] = *reinterpret_cast<const uint16_t*>(&bv);
            hh[off] = *reinterpret_cast<const uint16_t*>(&hv);
        }
    if (cudaMalloc(&c->tcB, 2 * nmma * 64) != cudaSuccess) return false;
    if (cudaMemcpy(c->tcB, hb.data(), nmma * 64, cudaMemcpyHostToDevice) != cudaSuccess) return false;
    if (cudaMemcpy(c->tcB + nmma * 64, hh.data(), nmma * 64, cudaMemcpyHostToDevice) != cudaSuccess)
        return false;
    // z segments of about 20 node layers, balanced
    const int nz = c->g.nz;
    const int nseg = (nz + 19) / 20;
    c->tc_lz = (nz + nseg - 1) / nseg;
    int sms = 152;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
    c->tc_grid = sms;     // CTAs per SM are set per variant at launch
    return encode_map(c, &c->tm_r, c->r32, 3) && encode_map(c, &c->tm_pa, c->p32a, 3) &&
           encode_map(c, &c->tm_pb, c->p32b, 3) && encode_map(c, &c->tm_d, c->dinv32, 1) &&
           encode_map(c, &c->tm_e, c->E32, 1, true);
}

template <int PREC, bool FUSED, bool SPLIT>
static void launch_one(to3d_ctx* c, cudaStream_t s, const TcArgs& a, const CUtensorMap& tr,
                       const CUtensorMap& tp, const CUtensorMap& td) {
    constexpr int NSL = (PREC == 2 || PREC == 4) ? 2 : 1;
    const int per_sm = TC_CTAS_PER_SM;
    const int grid = a.ntiles < c->tc_grid * per_sm ? a.ntiles : c->tc_grid * per_sm;
    k_matvec_tc<PREC, FUSED, SPLIT><<<grid, TC_ROLE_THREADS, TcSmemWs<NSL, SPLIT ? 64 : 32>::BYTES, s>>>(
        a, tr, tp, td, c->tm_e);
    c->launches++;
}

template <bool FUSED, bool SPLIT>
static void launch_prec(to3d_ctx* c, cudaStream_t s, const TcArgs& a, int prec, const CUtensorMap& tr,
                        const CUtensorMap& tp, const CUtensorMap& td) {
    if (prec == TO3D_BF16X2_DC) launch_one<2, FUSED, SPLIT>(c, s, a, tr, tp, td);
    else if (prec == TO3D_FP16_DC) launch_one<3, FUSED, SPLIT>(c, s, a, tr, tp, td);
    else if (prec == TO3D_FP16X2_DC) launch_one<4, FUSED, SPLIT>(c, s, a, tr, tp, td);
    else launch_one<1, FUSED, SPLIT>(c, s, a, tr, tp, td);
}

// Fused: p_old is p32b (parity 0) or p32a (parity 1), p_new the other one.
// Plain: the input is p32a (padded SoA), the output q32.
void launch_matvec_tc(to3d_ctx* c, cudaStream_t s, int prec, bool fused, int parity) {
    const CUtensorMap& tp = fused ? (parity ? c->tm_pa : c->tm_pb) : c->tm_pa;
    launch_matvec_tc_io(c, s, prec, fused, c->tm_r, tp, c->tm_d,
                        fused ? (parity ? c->p32b : c->p32a) : nullptr, c->q32, fused ? c->ss : nullptr);
}

// General form: the maps of r (fused only), p (fused: p_old; plain: the
// input) and the per-node scaling d (fused only), the outputs p_new (fused
// only) and q.  `ss` (may be null in plain mode): the kernel returns at once
// when ss->done is set.
void launch_matvec_tc_io(to3d_ctx* c, cudaStream_t s, int prec, bool fused, const CUtensorMap& tr,
                         const CUtensorMap& tp, const CUtensorMap& td, float* p_new, float* q,
                         SolverScalars* ss) {
    const Grid& g = c->g;
    TcArgs a;
    a.g = g;
    a.px = c->px;
    a.plane = (long long)c->px * g.ny;
    a.vol = a.plane * g.nz;
    a.lz = c->tc_lz;
    a.ntx = (g.nx + TC_BX - 1) / TC_BX;
    a.nty = (g.ny + TC_BY - 1) / TC_BY;
    a.ntz = (g.nz + a.lz - 1) / a.lz;
    a.ntiles = a.ntx * a.nty * a.ntz;
    a.cscale = c->tc_cscale;
    a.c_lam = (float)c->kes.c_lam;
    a.c_mu = (float)c->kes.c_mu;
    const int nmma = c->tc_split ? 64 : 32;
    a.Bglob = c->tcB + ((prec == TO3D_FP16_DC || prec == TO3D_FP16X2_DC) ? nmma * 64 : 0);
    a.E32 = c->E32;
    a.p_new = p_new;
    a.q = q;
    a.red = c->red;
    a.ss = ss;
    a.err = c->dev_err;
    if (fused) {
        if (c->tc_split) launch_prec<true, true>(c, s, a, prec, tr, tp, td);
        else launch_prec<true, false>(c, s, a, prec, tr, tp, td);
    } else {
        if (c->tc_split) launch_prec<false, true>(c, s, a, prec, tr, tp, td);
        else launch_prec<false, false>(c, s, a, prec, tr, tp, td);
    }
}

// TMA map of a padded SoA vector of context c (3 components) or of a
// per-node array (1 component), for launch_matvec_tc_io.
bool encode_vec_map(to3d_ctx* c, CUtensorMap* map, const float* base, int comps) {
    return encode_map(c, map, base, comps);
}

void launch_aos_to_soa(to3d_ctx* c, cudaStream_t s, const float* in, float* out) {
    const Grid& g = c->g;
    k_aos_to_soa<<<(unsigned)((g.nnode + 255) / 256), 256, 0, s>>>(
        g, c->px, (long long)c->px * g.ny * g.nz, in, c->nodemask, out);
    c->launches++;
}

void launch_soa_to_aos(to3d_ctx* c, cudaStream_t s, const float* q, const float* p, float* y) {
    const Grid& g = c->g;
    k_soa_to_aos<<<(unsigned)((g.nnode + 255) / 256), 256, 0, s>>>(
        g, c->px, (long long)c->px * g.ny * g.nz, q, p, c->nodemask, y);
    c->launches++;
}

}  // namespace to3d

namespace to3d {

// ------------------------------------------------------------------ wait self-test
// One thread waits, with the tensor-core kernel's bounded suspend-and-poll
// loop, on an mbarrier phase that nothing completes; it gives up after
// `polls` polls and reports the timeout as the kernel would.
__global__ void k_selftest_wait(int polls, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    const bool ok = tc::mbar_wait_sleep_bounded(&bar, 0u, (uint32_t)polls, 1000u);
    *status = ok ? (int)TO3D_OK : (int)TO3D_ETIMEOUT;
}

// ------------------------------------------------------------------ autotuner
// The tensor-core kernel walks z segments of lz node layers per tile.  Short
// segments give more tiles (better balance on small grids), long ones less
// halo.  The best lz is timed once per grid shape and precision and cached.
// The timing runs the plain form with precision prec on the input mapped by
// tp and writes q; set_moduli first fills E32 from x, otherwise whatever E32
// holds is used (the time does not depend on the values).
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int, int>, int> g_tune;

cudaError_t tune_tc_lz(to3d_ctx* c, int prec, const CUtensorMap& tp, float* q, bool set_moduli) {
    const auto key = std::make_tuple(c->g.nx, c->g.ny, c->g.nz, prec);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            c->tc_lz = it->second;
            return cudaSuccess;
        }
    }
    if (set_moduli) launch_simp(c, c->stream, c->x);
    const int cand[] = {4, 6, 8, 12, 16, 20, 27, 40, 81};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    float best = 1e30f;
    int best_lz = c->tc_lz;
    for (int lz : cand) {
        if (err != cudaSuccess) break;
        if (lz > c->g.nz && lz != cand[0]) continue;
        c->tc_lz = lz;
        auto op = [&]() { launch_matvec_tc_io(c, c->stream, prec, false, c->tm_r, tp, c->tm_d, nullptr, q, nullptr); };
        op();
        err = cudaEventRecord(e0, c->stream);
        for (int r = 0; r < 3 && err == cudaSuccess; ++r) op();
        if (err == cudaSuccess) err = cudaEventRecord(e1, c->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
        if (err == cudaSuccess && ms < best) {
            best = ms;
            best_lz = lz;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    c->tc_lz = best_lz;
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune[key] = best_lz;
    return cudaGetLastError();
}

}  // namespace to3d

extern "C" TO3D_API to3d_status to3d_selftest_wait_timeout(int32_t polls, int32_t* status,
                                                           void* stream) {
    if (polls < 1 || polls > (1 << 16) || !status) return TO3D_EINVAL;
    int* d = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMallocAsync((void**)&d, sizeof(int), s) != cudaSuccess) return TO3D_ENOMEM;
    to3d::k_selftest_wait<<<1, 32, 0, s>>>(polls, d);
    int h = -1;
    cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return TO3D_ECUDA;
    *status = h;
    return TO3D_OK;
}
