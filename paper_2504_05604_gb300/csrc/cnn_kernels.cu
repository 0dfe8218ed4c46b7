// Kernels of the learned preconditioner (see cnn_kernels.cuh).
#include "cnn_kernels.cuh"

namespace to3d {
namespace cnn {

// D (16x8, FP32) += A (16x16, BF16, row) * B (16x8, BF16, col)
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
}

// keep the BF16 halves of v whose mask halves are > 0
__device__ __forceinline__ uint32_t mask_pair(uint32_t v, uint32_t m) {
    const __nv_bfloat162 mm = *reinterpret_cast<const __nv_bfloat162*>(&m);
    const uint32_t keep_lo = __bfloat162float(mm.x) > 0.f ? 0x0000ffffu : 0u;
    const uint32_t keep_hi = __bfloat162float(mm.y) > 0.f ? 0xffff0000u : 0u;
    return v & (keep_lo | keep_hi);
}

// Implicit-GEMM 3x3x3 convolution.  A block computes a 16 x 4R x 2 tile of
// output voxels (8 warps, R 16-voxel x-rows each: the M = 16 rows of an MMA
// per x-row) for all output channels.  The input tile with its one-voxel
// halo (18 x (4R + 2) x 4 voxels) is staged in shared memory 16 channels at
// a time (converted to BF16 and masked on the way in when the input is an
// FP32 gradient); K then runs over the 27 taps of that channel chunk, the A
// fragments coming from shared memory and the B fragments (weights) from L1,
// each B fragment serving the warp's R rows.  Narrow layers (few output
// channels) take R = 4 (16 channels) or 2 (32) to reuse their weight
// fragments; wide ones R = 1 to bound the accumulator registers.  Voxels are padded to 24 BF16 in shared
// memory so that the eight voxel rows of a fragment load fall in distinct
// banks.
constexpr int CT_X = 16, CT_Z = 2;
constexpr int CH_X = CT_X + 2, CH_Z = CT_Z + 2;
constexpr int CH_PITCH = 24;

template <bool F32, int NT, int R>
__global__ void __launch_bounds__(256) k_conv(const ConvArgs a, int tiles_x, int tiles_y) {
    constexpr int CT_Y = 4 * R, CH_Y = CT_Y + 2, CH_VOX = CH_X * CH_Y * CH_Z;
    extern __shared__ __align__(16) uint8_t conv_smem[];
    bf16* sx = reinterpret_cast<bf16*>(conv_smem);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;
    int blk = blockIdx.x;
    const int tx = blk % tiles_x;
    blk /= tiles_x;
    const int ty = blk % tiles_y, tz = blk / tiles_y;
    const int x0 = tx * CT_X, y0 = ty * CT_Y, z0 = tz * CT_Z;
    const int wy0 = (warp % 4) * R, wz = warp / 4;
    const int Cin = a.C1 + a.C2, nchunk = Cin / 16;
    float acc[R][NT][4];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int n = 0; n < NT; ++n) acc[r][n][0] = acc[r][n][1] = acc[r][n][2] = acc[r][n][3] = 0.f;
    for (int chunk = 0; chunk < nchunk; ++chunk) {
        const int k0 = chunk * 16;
        const bool first = k0 < a.C1;
        const void* src = first ? a.in1 : a.in2;
        const int cs = first ? a.C1 : a.C2;
        const int kk = first ? k0 : k0 - a.C1;
        const bf16* mk = first ? a.mask1 : nullptr;
        __syncthreads();
        for (int i = tid; i < CH_VOX * 2; i += 256) {
            const int vox = i >> 1, h = i & 1;
            const int hx = vox % CH_X, hy = (vox / CH_X) % CH_Y, hz = vox / (CH_X * CH_Y);
            const int x = x0 - 1 + hx, y = y0 - 1 + hy, z = z0 - 1 + hz;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (x >= 0 && x < a.X && y >= 0 && y < a.Y && z >= 0 && z < a.Z) {
                const long long off = (x + (long long)a.X * (y + (long long)a.Y * z)) * cs + kk + 8 * h;
                if (F32) {
                    const float4 f0 = *reinterpret_cast<const float4*>((const float*)src + off);
                    const float4 f1 = *reinterpret_cast<const float4*>((const float*)src + off + 4);
                    val = make_uint4(pack_bf16(f0.x, f0.y), pack_bf16(f0.z, f0.w),
                                     pack_bf16(f1.x, f1.y), pack_bf16(f1.z, f1.w));
                } else {
                    val = *reinterpret_cast<const uint4*>((const bf16*)src + off);
                }
                if (mk) {
                    const uint4 m = *reinterpret_cast<const uint4*>(mk + off);
                    val = make_uint4(mask_pair(val.x, m.x), mask_pair(val.y, m.y),
                                     mask_pair(val.z, m.z), mask_pair(val.w, m.w));
                }
            }
            *reinterpret_cast<uint4*>(sx + vox * CH_PITCH + 8 * h) = val;
        }
        __syncthreads();
        const bf16* Wc = a.W + k0 + 2 * q;
#pragma unroll 3
        for (int tap = 0; tap < 27; ++tap) {
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            uint32_t af[R][4];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const bf16* p0 =
                    sx + (((wz + dz) * CH_Y + (wy0 + r + dy)) * CH_X + (g + dx)) * CH_PITCH + 2 * q;
                const bf16* p1 = p0 + 8 * CH_PITCH;
                af[r][0] = *reinterpret_cast<const uint32_t*>(p0);
                af[r][1] = *reinterpret_cast<const uint32_t*>(p1);
                af[r][2] = *reinterpret_cast<const uint32_t*>(p0 + 8);
                af[r][3] = *reinterpret_cast<const uint32_t*>(p1 + 8);
            }
            const bf16* Wt = Wc + (size_t)tap * a.Cout * Cin;
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const bf16* wrow = Wt + (size_t)(n * 8 + g) * Cin;
                const uint32_t b0 = *reinterpret_cast<const uint32_t*>(wrow);
                const uint32_t b1 = *reinterpret_cast<const uint32_t*>(wrow + 8);
#pragma unroll
                for (int r = 0; r < R; ++r) mma16816(acc[r][n], af[r], b0, b1);
            }
        }
    }
    const int z = z0 + wz;
    if (z >= a.Z) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = y0 + wy0 + r;
        if (y >= a.Y) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int x = x0 + g + 8 * h;
            if (x >= a.X) continue;
            const long long v = x + (long long)a.X * (y + (long long)a.Y * z);
#pragma unroll
            for (int n = 0; n < NT; ++n) {
                const int c = n * 8 + 2 * q;
                float v0 = acc[r][n][2 * h], v1 = acc[r][n][2 * h + 1];
                if (a.bias) {
                    v0 += a.bias[c];
                    v1 += a.bias[c + 1];
                }
                if (a.relu) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                const long long o = v * a.out_cstride + a.out_coff + c;
                if (a.out_b) {
                    *reinterpret_cast<uint32_t*>(a.out_b + o) = pack_bf16(v0, v1);
                } else if (a.accumulate) {
                    a.out_f[o] += v0;
                    a.out_f[o + 1] += v1;
                } else {
                    a.out_f[o] = v0;
                    a.out_f[o + 1] = v1;
                }
            }
        }
    }
}

template <bool F32, int NT, int R>
static void launch_conv(const ConvArgs& a, unsigned blocks, int tiles_x, int tiles_y,
                        cudaStream_t s) {
    constexpr int bytes = CH_X * (4 * R + 2) * CH_Z * CH_PITCH * 2;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_conv<F32, NT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        attr = true;
    }
    k_conv<F32, NT, R><<<blocks, 256, bytes, s>>>(a, tiles_x, tiles_y);
}

void conv_forward(const ConvArgs& a, bool in_fp32, cudaStream_t s) {
    const int nt = a.Cout / 8;
    const int R = nt <= 2 ? 4 : (nt <= 4 ? 2 : 1);
    const int tiles_x = (a.X + CT_X - 1) / CT_X, tiles_y = (a.Y + 4 * R - 1) / (4 * R);
    const int tiles_z = (a.Z + CT_Z - 1) / CT_Z;
    const unsigned blocks = (unsigned)((long long)tiles_x * tiles_y * tiles_z);
#define TO3D_CONV(NTV, RV)                                                         \
    if (nt == NTV) {                                                               \
        if (in_fp32) launch_conv<true, NTV, RV>(a, blocks, tiles_x, tiles_y, s);   \
        else launch_conv<false, NTV, RV>(a, blocks, tiles_x, tiles_y, s);          \
        return;                                                                    \
    }
    TO3D_CONV(1, 4) TO3D_CONV(2, 4) TO3D_CONV(4, 2) TO3D_CONV(6, 1) TO3D_CONV(8, 1)
    TO3D_CONV(12, 1) TO3D_CONV(16, 1)
#undef TO3D_CONV
}

// Weight (and bias) gradient of a convolution, FP32 on the CUDA cores:
// gw[tap][co][ci] += sum_v gy[v][co] (mask) x[v + tap][ci].  A block owns a
// 16 x 16 (co, ci) tile of one tap and a chunk of voxels.
constexpr int WG_CHUNK = 128;
constexpr int WG_VOX_PER_BLOCK = 4096;

template <bool XF32>
__global__ void __launch_bounds__(256) k_wgrad(const WgradArgs a) {
    __shared__ float sg[WG_CHUNK][17];
    __shared__ float sx[WG_CHUNK][17];
    const int tap = blockIdx.y;
    const int nci = a.Cin / 16;
    const int co0 = (blockIdx.z / nci) * 16, ci0 = (blockIdx.z % nci) * 16;
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    const int t = threadIdx.x, tco = t / 16, tci = t % 16;
    float acc = 0.f, accb = 0.f;
    const long long vbeg = (long long)blockIdx.x * WG_VOX_PER_BLOCK;
    const long long vend = min(vbeg + WG_VOX_PER_BLOCK, a.nvox);
    for (long long v0 = vbeg; v0 < vend; v0 += WG_CHUNK) {
        for (int i = t; i < WG_CHUNK * 16; i += 256) {
            const int r = i / 16, c = i % 16;
            const long long v = v0 + r;
            float gv = 0.f, xv = 0.f;
            if (v < vend) {
                const int co = co0 + c;
                if (co < a.Cout_fwd) {
                    gv = a.gy[v * a.gy_cstride + co];
                    if (a.mask && !(__bfloat162float(a.mask[v * a.gy_cstride + co]) > 0.f)) gv = 0.f;
                }
                const int x = (int)(v % a.X), y = (int)((v / a.X) % a.Y), z = (int)(v / ((long long)a.X * a.Y));
                const int xx = x + dx, yy = y + dy, zz = z + dz;
                if (xx >= 0 && xx < a.X && yy >= 0 && yy < a.Y && zz >= 0 && zz < a.Z) {
                    const long long nbv = xx + (long long)a.X * (yy + (long long)a.Y * zz);
                    const int ci = ci0 + c;
                    const bool first = ci < a.C1;
                    const int cs = first ? a.C1 : a.Cin - a.C1;
                    const int cc = first ? ci : ci - a.C1;
                    const void* src = first ? a.x1 : a.x2;
                    xv = XF32 ? ((const float*)src)[nbv * cs + cc]
                              : __bfloat162float(((const bf16*)src)[nbv * cs + cc]);
                }
            }
            sg[r][c] = gv;
            sx[r][c] = xv;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < WG_CHUNK; ++r) {
            acc = fmaf(sg[r][tco], sx[r][tci], acc);
            accb += sg[r][tco];
        }
        __syncthreads();
    }
    const int co = co0 + tco, ci = ci0 + tci;
    if (co < a.Cout_fwd) {
        atomicAdd(&a.gw[((size_t)tap * a.Cout_fwd + co) * a.Cin + ci], acc);
        if (a.gb && tap == 0 && ci0 == 0 && tci == 0) atomicAdd(&a.gb[co], accb);
    }
}

void conv_wgrad(const WgradArgs& a, bool x_fp32, cudaStream_t s) {
    const int ncot = (a.Cout + 15) / 16;
    dim3 grid((unsigned)((a.nvox + WG_VOX_PER_BLOCK - 1) / WG_VOX_PER_BLOCK), 27,
              (unsigned)(ncot * (a.Cin / 16)));
    if (x_fp32) k_wgrad<true><<<grid, 256, 0, s>>>(a);
    else k_wgrad<false><<<grid, 256, 0, s>>>(a);
}

// Wt[tap][ci][co] = W[26 - tap][co][ci]: the data gradient is a convolution
// of the upstream gradient with the flipped, transposed kernel.
__global__ void k_transpose_flip(const bf16* W, bf16* Wt, int Cout, int Cin) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long n = 27LL * Cout * Cin;
    if (i >= n) return;
    const int co = (int)(i % Cout);
    const int ci = (int)((i / Cout) % Cin);
    const int tap = (int)(i / ((long long)Cout * Cin));
    Wt[i] = W[((size_t)(26 - tap) * Cout + co) * Cin + ci];
}

void transpose_flip(const bf16* W, bf16* Wt, int Cout, int Cin, cudaStream_t s) {
    const long long n = 27LL * Cout * Cin;
    k_transpose_flip<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(W, Wt, Cout, Cin);
}

// ---- 2x2x2 average pooling and nearest x2 upsampling (channels-last)
__global__ void k_pool2(const bf16* in, bf16* out, int Z, int Y, int X, int C) {
    const long long n = (long long)(Z / 2) * (Y / 2) * (X / 2) * C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long v = i / C;
    const int X2 = X / 2, Y2 = Y / 2;
    const int x = (int)(v % X2), y = (int)((v / X2) % Y2), z = (int)(v / ((long long)X2 * Y2));
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const long long u = (2 * x + (k & 1)) + (long long)X * ((2 * y + ((k >> 1) & 1)) + (long long)Y * (2 * z + (k >> 2)));
        s += __bfloat162float(in[u * C + c]);
    }
    out[i] = __float2bfloat16_rn(0.125f * s);
}

__global__ void k_pool2_bwd(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X,
                            int C, int accumulate) {
    const long long n = (long long)Z * Y * X * C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((long long)X * Y));
    const long long p = (x / 2) + (long long)(X / 2) * ((y / 2) + (long long)(Y / 2) * (z / 2));
    const float g = 0.125f * gout[p * gcs + gco + c];
    gin[i] = accumulate ? gin[i] + g : g;
}

__global__ void k_up2(const bf16* in, bf16* out, int Z, int Y, int X, int C) {
    // in: (Z/2, Y/2, X/2), out: (Z, Y, X)
    const long long n = (long long)Z * Y * X * C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % X), y = (int)((v / X) % Y), z = (int)(v / ((long long)X * Y));
    const long long p = (x / 2) + (long long)(X / 2) * ((y / 2) + (long long)(Y / 2) * (z / 2));
    out[i] = in[p * C + c];
}

__global__ void k_up2_bwd(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X,
                          int C, int accumulate) {
    // gout on (Z, Y, X); gin on (Z/2, Y/2, X/2)
    const int X2 = X / 2, Y2 = Y / 2;
    const long long n = (long long)(Z / 2) * Y2 * X2 * C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = (int)(i % C);
    const long long v = i / C;
    const int x = (int)(v % X2), y = (int)((v / X2) % Y2), z = (int)(v / ((long long)X2 * Y2));
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const long long u = (2 * x + (k & 1)) + (long long)X * ((2 * y + ((k >> 1) & 1)) + (long long)Y * (2 * z + (k >> 2)));
        s += gout[u * gcs + gco + c];
    }
    gin[i] = accumulate ? gin[i] + s : s;
}

__global__ void k_add_channels(const float* src, int scs, int sco, float* dst, long long nvox, int C,
                               int accumulate) {
    const long long n = nvox * C;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float v = src[(i / C) * scs + sco + (i % C)];
    dst[i] = accumulate ? dst[i] + v : v;
}

static unsigned nb(long long n) { return (unsigned)((n + 255) / 256); }

void pool2_forward(const bf16* in, bf16* out, int Z, int Y, int X, int C, cudaStream_t s) {
    k_pool2<<<nb((long long)(Z / 2) * (Y / 2) * (X / 2) * C), 256, 0, s>>>(in, out, Z, Y, X, C);
}
void pool2_backward(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X, int C,
                    int accumulate, cudaStream_t s) {
    k_pool2_bwd<<<nb((long long)Z * Y * X * C), 256, 0, s>>>(gout, gcs, gco, gin, Z, Y, X, C, accumulate);
}
void up2_forward(const bf16* in, bf16* out, int Z, int Y, int X, int C, cudaStream_t s) {
    k_up2<<<nb((long long)Z * Y * X * C), 256, 0, s>>>(in, out, Z, Y, X, C);
}
void up2_backward(const float* gout, int gcs, int gco, float* gin, int Z, int Y, int X, int C,
                  int accumulate, cudaStream_t s) {
    k_up2_bwd<<<nb((long long)(Z / 2) * (Y / 2) * (X / 2) * C), 256, 0, s>>>(gout, gcs, gco, gin, Z, Y, X, C, accumulate);
}
void add_channels(const float* src, int scs, int sco, float* dst, long long nvox, int C,
                  int accumulate, cudaStream_t s) {
    k_add_channels<<<nb(nvox * C), 256, 0, s>>>(src, scs, sco, dst, nvox, C, accumulate);
}

// ---- Adam on a flat FP32 parameter vector
__global__ void k_adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

void adam(float* p, const float* g, float* m, float* v, long long n, float lr, float b1, float b2,
          float eps, int t, cudaStream_t s) {
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    k_adam<<<nb(n), 256, 0, s>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
}

__global__ void k_to_bf16(const float* src, bf16* dst, long long n) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

void to_bf16(const float* src, bf16* dst, long long n, cudaStream_t s) {
    k_to_bf16<<<nb(n), 256, 0, s>>>(src, dst, n);
}

}  // namespace cnn
}  // namespace to3d
