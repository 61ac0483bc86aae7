// k_prop.cu -- the learned density propagator: a 3-D periodic conv net
// (4 -> 16 -> 16 -> 2 channels, 3x3x3 kernels, SiLU) on BF16 tensor cores.
//
// Activations are channels-last BF16 [V][16] (channels padded to 16 with
// zeros; V = Mz My Mx, x fastest).  A convolution is an implicit GEMM: a CTA
// owns a 8 x 8 x 2 tile of 128 output voxels, stages the periodic
// 10 x 10 x 4 input box in shared memory, and for each of the 27 kernel
// offsets multiplies the box shifted by that offset (16 voxels x 16 input
// channels per warp, read with ldmatrix) by the offset's 16 x 16 weight block
// with mma.sync m16n8k16 (BF16 in, FP32 accumulate).  The data-gradient pass
// is the same kernel with flipped and transposed weights; the weight
// gradient reduces over voxels on the tensor cores (ldmatrix.trans operands)
// and accumulates in registers over many tiles before one FP32 atomic add
// per weight and CTA.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <string>

#include "hpf_internal.cuh"

namespace hpf {

constexpr int kPC = 16;                      // padded channels
constexpr int kTX = 8, kTY = 8, kTZ = 8;     // output tile: one z-plane of 64 voxels per warp
constexpr int kBX = kTX + 2, kBY = kTY + 2, kBZ = kTZ + 2;
constexpr int kBoxVox = kBX * kBY * kBZ;     // 1000 (32 000 bytes)
constexpr int kTileVox = kTX * kTY * kTZ;    // 512
constexpr int kMTiles = kTileVox / 16 / 8;   // 16-voxel MMA row tiles per warp (4)
constexpr int kOffsets = 27;
// channels of the three layers: 4 -> 16 -> 16 -> 2
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? 4 : 16; }
__host__ __device__ constexpr int layer_out(int l) { return l == 2 ? 2 : 16; }

struct PropGeom {
    int mx, my, mz, V;
    int tiles_x, tiles_y, tiles_z, tiles;
};

__device__ __forceinline__ int pwrap(int i, int m) {
    i %= m;
    return i < 0 ? i + m : i;
}

__device__ __forceinline__ uint32_t saddr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                        uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2,
                                          uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
        "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void tile_origin(const PropGeom& g, int t, int& x0, int& y0, int& z0) {
    x0 = (t % g.tiles_x) * kTX;
    y0 = ((t / g.tiles_x) % g.tiles_y) * kTY;
    z0 = (t / (g.tiles_x * g.tiles_y)) * kTZ;
}

// Shared-memory rows are 16 channels = two 16-byte halves.  The halves of
// every other group of four rows are swapped so that the eight rows an
// ldmatrix phase reads (always eight consecutive rows here) hit distinct banks.
__device__ __forceinline__ int swz(int row, int half) { return 2 * row + (half ^ ((row >> 2) & 1)); }

// Periodic input box of a tile (all 16 channels), 16-byte asynchronous copies.
__device__ __forceinline__ void load_box(const __nv_bfloat16* __restrict__ in, const PropGeom& g,
                                         int x0, int y0, int z0, uint4* box) {
    const uint32_t box_s = saddr(box);
    for (int e = threadIdx.x; e < kBoxVox * 2; e += blockDim.x) {
        const int v = e >> 1, half = e & 1;
        const int bx = v % kBX, by = (v / kBX) % kBY, bz = v / (kBX * kBY);
        const int gx = pwrap(x0 - 1 + bx, g.mx), gy = pwrap(y0 - 1 + by, g.my),
                  gz = pwrap(z0 - 1 + bz, g.mz);
        const size_t gv = ((size_t)gz * g.my + gy) * g.mx + gx;
        cp_async16(box_s + 16 * swz(v, half), in + gv * kPC + 8 * half);
    }
}

// Voxel r (0..15) of 16-voxel row tile mt (0..31) of the tile: (lx, ly, lz);
// row tiles 4w .. 4w + 3 are the z-plane lz = w.
__device__ __forceinline__ void warp_voxel(int mt, int r, int& lx, int& ly, int& lz) {
    const int m = 16 * mt + r;
    lx = m % kTX;
    ly = (m / kTX) % kTY;
    lz = m / (kTX * kTY);
}

// Box row of tile voxel (lx, ly, lz) shifted by kernel offset o.
__device__ __forceinline__ int box_row(int lx, int ly, int lz, int o) {
    const int dz = o / 9 - 1, dy = (o / 3) % 3 - 1, dx = o % 3 - 1;
    return ((lz + 1 + dz) * kBY + (ly + 1 + dy)) * kBX + (lx + 1 + dx);
}

// ------------------------------------------------------------------ convolution

enum ConvMode { kHidden = 0, kLast = 1, kData = 2 };

// out(n)[co] = sum_offsets sum_ci W[o][co][ci] in(n + d_o)[ci]  (+ bias, SiLU).
// One CTA per 8 x 8 x 8 tile; warp w computes the 64 voxels of z-plane w as
// four 16-row MMA tiles against each offset's weight fragment (loaded once
// per offset and warp).  kN output n-tiles of 8 channels (1 for the
// two-channel last layer).  kHidden stores the FP32 pre-activation (when
// z_out is given) and the BF16 SiLU output; kLast and kData store FP32.
template <int kMode, int kN>
__global__ void __launch_bounds__(256) k_conv(const __nv_bfloat16* __restrict__ in,
                                              const __nv_bfloat16* __restrict__ W,
                                              const float* __restrict__ bias,
                                              float* __restrict__ z_out,
                                              __nv_bfloat16* __restrict__ act_out,
                                              float* __restrict__ f_out, PropGeom g) {
    __shared__ uint4 box[kBoxVox * 2];
    __shared__ uint4 sw[kOffsets * kPC * 2];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const uint32_t box_s = saddr(box), sw_s = saddr(sw);
    for (int e = tid; e < kOffsets * kPC * 2; e += blockDim.x)
        cp_async16(sw_s + 16 * swz(e >> 1, e & 1), reinterpret_cast<const uint4*>(W) + e);
    int x0, y0, z0;
    tile_origin(g, blockIdx.x, x0, y0, z0);
    load_box(in, g, x0, y0, z0, box);
    cp_async_wait_all();
    __syncthreads();

    // A rows: lane -> voxel (lane % 16) of each row tile, channel half (lane / 16)
    const int r = lane & 15, ch_half = lane >> 4;
    // B rows: lane -> output channel (lane & 7) + 8 (lane >= 16), input half ((lane >> 3) & 1)
    const int b_n = (lane & 7) + ((lane >> 4) << 3), b_half = (lane >> 3) & 1;
    const int gq = lane >> 2, q = lane & 3;
    float acc[kMTiles][kN][4];
#pragma unroll
    for (int i = 0; i < kMTiles; ++i)
#pragma unroll
        for (int j = 0; j < kN; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[i][j][c] = 0.f;
    // voxel (lx, ly0 + 2i, w) for row tile i
    const int lx = r % kTX, ly0 = r / kTX;
#pragma unroll 9
    for (int o = 0; o < kOffsets; ++o) {
        uint32_t b0, b1, b2, b3;
        ldsm_x4(sw_s + 16 * swz(o * kPC + b_n, b_half), b0, b1, b2, b3);
        const int row0 = box_row(lx, ly0, w, o);
#pragma unroll
        for (int i = 0; i < kMTiles; ++i) {
            uint32_t a0, a1, a2, a3;
            ldsm_x4(box_s + 16 * swz(row0 + 2 * i * kBX, ch_half), a0, a1, a2, a3);
            mma_bf16(acc[i][0], a0, a1, a2, a3, b0, b1);
            if (kN > 1) mma_bf16(acc[i][kN - 1], a0, a1, a2, a3, b2, b3);
        }
    }
    float b_lo[kN], b_hi[kN];
#pragma unroll
    for (int j = 0; j < kN; ++j) {
        b_lo[j] = kMode != kData ? bias[8 * j + 2 * q] : 0.f;
        b_hi[j] = kMode != kData ? bias[8 * j + 2 * q + 1] : 0.f;
    }
    // epilogue: lane holds voxels gq, gq + 8 of each row tile and channels 8j + 2q, + 1
#pragma unroll
    for (int i = 0; i < kMTiles; ++i)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            int vx, vy, vz;
            warp_voxel(kMTiles * w + i, gq + 8 * half, vx, vy, vz);
            const int X = x0 + vx, Y = y0 + vy, Z = z0 + vz;
            if (X >= g.mx || Y >= g.my || Z >= g.mz) continue;
            const size_t gv = ((size_t)Z * g.my + Y) * g.mx + X;
#pragma unroll
            for (int j = 0; j < kN; ++j) {
                const int ch = 8 * j + 2 * q;
                const float v0 = acc[i][j][2 * half] + b_lo[j];
                const float v1 = acc[i][j][2 * half + 1] + b_hi[j];
                if (kMode == kHidden) {
                    if (z_out)
                        *reinterpret_cast<float2*>(z_out + gv * kPC + ch) = make_float2(v0, v1);
                    const float s0 = v0 / (1.0f + expf(-v0)), s1 = v1 / (1.0f + expf(-v1));
                    *reinterpret_cast<__nv_bfloat162*>(act_out + gv * kPC + ch) =
                        __floats2bfloat162_rn(s0, s1);
                } else {
                    *reinterpret_cast<float2*>(f_out + gv * kPC + ch) = make_float2(v0, v1);
                }
            }
        }
}

// dW[o][ci][co] = sum_n in(n + d_o)[ci] gz(n)[co]: a voxel reduction on the
// tensor cores.  Warp w owns offsets w, w + 8, w + 16 (and 24 for w < 3); a
// CTA walks tiles grid-stride and writes its register sums to its own slice
// part[blockIdx.x] (every entry, once); k_sum_partials adds the slices in a
// fixed order, so the gradient is deterministic.
__global__ void __launch_bounds__(256) k_conv_wgrad(const __nv_bfloat16* __restrict__ in,
                                                    const __nv_bfloat16* __restrict__ gz,
                                                    float* __restrict__ part, PropGeom g) {
    __shared__ uint4 box[kBoxVox * 2];
    __shared__ uint4 gt[kTileVox * 2];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    float acc[4][2][4];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[s][j][c] = 0.f;
    // A = in^T (ci x voxels) by ldmatrix.trans of voxel rows: lane -> voxel
    // (lane & 7) + 8 (lane >= 16), channel half ((lane >> 3) & 1), so that
    // a0 = ci 0-7 / vox 0-7, a1 = ci 8-15 / vox 0-7, a2 = ci 0-7 / vox 8-15,
    // a3 = ci 8-15 / vox 8-15
    const int r_vox = (lane & 7) + ((lane >> 4) << 3), r_half = (lane >> 3) & 1;
    // B = gz (voxels x co): lane -> voxel (lane & 7) + 8 ((lane >> 3) & 1), co half
    // (lane >> 4): b0 = vox 0-7 / co 0-7, b1 = vox 8-15 / co 0-7, b2 = vox 0-7 /
    // co 8-15, b3 = vox 8-15 / co 8-15
    const int g_vox = (lane & 7) + (((lane >> 3) & 1) << 3), g_half = lane >> 4;
    const uint32_t box_s = saddr(box), gt_s = saddr(gt);
    for (int t = blockIdx.x; t < g.tiles; t += gridDim.x) {
        int x0, y0, z0;
        tile_origin(g, t, x0, y0, z0);
        __syncthreads();
        load_box(in, g, x0, y0, z0, box);
        for (int e = tid; e < kTileVox * 2; e += blockDim.x) {
            const int m = e >> 1, half = e & 1;
            const int X = x0 + m % kTX, Y = y0 + (m / kTX) % kTY, Z = z0 + m / (kTX * kTY);
            if (X < g.mx && Y < g.my && Z < g.mz)
                cp_async16(gt_s + 16 * swz(m, half),
                           gz + (((size_t)Z * g.my + Y) * g.mx + X) * kPC + 8 * half);
            else
                gt[swz(m, half)] = make_uint4(0u, 0u, 0u, 0u);  // outside the mesh: adds nothing
        }
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int o = w + 8 * s;
            if (o >= kOffsets) break;
#pragma unroll 4
            for (int ks = 0; ks < kTileVox / 16; ++ks) {  // 16 voxels per k-step
                int lx, ly, lz;
                warp_voxel(ks, r_vox, lx, ly, lz);
                uint32_t a0, a1, a2, a3, b0, b1, b2, b3;
                ldsm_x4_t(box_s + 16 * swz(box_row(lx, ly, lz, o), r_half), a0, a1, a2, a3);
                ldsm_x4_t(gt_s + 16 * swz(16 * ks + g_vox, g_half), b0, b1, b2, b3);
                mma_bf16(acc[s][0], a0, a1, a2, a3, b0, b1);
                mma_bf16(acc[s][1], a0, a1, a2, a3, b2, b3);
            }
        }
    }
    const int gq = lane >> 2, q = lane & 3;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int o = w + 8 * s;
        if (o >= kOffsets) break;
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int ci = gq + 8 * (c >> 1), co = 8 * j + 2 * q + (c & 1);
                part[(size_t)blockIdx.x * kOffsets * kPC * kPC + (o * kPC + ci) * kPC + co] =
                    acc[s][j][c];
            }
    }
}

// ------------------------------------------------------------------ elementwise

// The network's input channels from x = (phi_A, phi_B at t - K, phi_A, phi_B
// at t), planar FP32: the scaled changes scale * (phi(t) - phi(t - K)) and the
// current phi(t) per species, formed in FP32 before the BF16 rounding (a
// one-step change of about 1e-2 is far below the BF16 spacing of phi ~ 0.5),
// zero-padded to 16.
__global__ void k_pack_input(const float* __restrict__ x, int V, float scale,
                             __nv_bfloat16* __restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const float a0 = x[v], b0 = x[(size_t)V + v];
    const float a1 = x[(size_t)2 * V + v], b1 = x[(size_t)3 * V + v];
    const float f[4] = {scale * (a1 - a0), scale * (b1 - b0), a1, b1};
    __nv_bfloat16 vals[kPC];
#pragma unroll
    for (int c = 0; c < kPC; ++c) vals[c] = __float2bfloat16_rn(c < 4 ? f[c] : 0.f);
    reinterpret_cast<uint4*>(out + (size_t)v * kPC)[0] = reinterpret_cast<uint4*>(vals)[0];
    reinterpret_cast<uint4*>(out + (size_t)v * kPC)[1] = reinterpret_cast<uint4*>(vals)[1];
}

// The predicted change: the network's two output channels divided by scale.
__global__ void k_unpack_output(const float* __restrict__ y, int V, float scale,
                                float* __restrict__ out) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    out[v] = y[(size_t)v * kPC] / scale;
    out[(size_t)V + v] = y[(size_t)v * kPC + 1] / scale;
}

// Mean squared error of the network output y against scale * (phi_next -
// phi_cur) (planar [2][V] each) and its gradient 2 (y - target) / (2V) in BF16.
__global__ void __launch_bounds__(256) k_loss(const float* __restrict__ y,
                                              const float* __restrict__ phi_cur,
                                              const float* __restrict__ phi_next, int V,
                                              float scale,
                                              __nv_bfloat16* __restrict__ gy,
                                              double* __restrict__ loss_part) {
    __shared__ double sh[8];
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (v < V) {
        __nv_bfloat16 vals[kPC];
#pragma unroll
        for (int c = 0; c < kPC; ++c) vals[c] = __float2bfloat16_rn(0.f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const size_t k = (size_t)c * V + v;
            const float d = y[(size_t)v * kPC + c] - scale * (phi_next[k] - phi_cur[k]);
            l += (double)d * d;
            vals[c] = __float2bfloat16_rn(d / (float)V);
        }
        reinterpret_cast<uint4*>(gy + (size_t)v * kPC)[0] = reinterpret_cast<uint4*>(vals)[0];
        reinterpret_cast<uint4*>(gy + (size_t)v * kPC)[1] = reinterpret_cast<uint4*>(vals)[1];
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_down_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += sh[k];
        loss_part[blockIdx.x] = s / (2.0 * (double)V);
    }
}

// out[j] = sum_b part[b][j], b in order (deterministic reductions).
template <class T>
__global__ void k_sum_partials(const T* __restrict__ part, int nb, int m, T* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    T s = 0;
    for (int b = 0; b < nb; ++b) s += part[(size_t)b * m + j];
    out[j] = s;
}

// gz = gh * SiLU'(z), in BF16 for the next tensor-core pass.
__global__ void k_silu_backward(const float* __restrict__ gh, const float* __restrict__ z,
                                long long n, __nv_bfloat16* __restrict__ gz) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float zz = z[i];
    const float s = 1.0f / (1.0f + expf(-zz));
    gz[i] = __float2bfloat16_rn(gh[i] * s * (1.0f + zz * (1.0f - s)));
}

// Bias gradient partials: part[block][co] = sum over the block's voxels of
// gz(n)[co] (16 voxel rows x 16 channels per pass).
__global__ void __launch_bounds__(256) k_bias_grad(const __nv_bfloat16* __restrict__ gz, int V,
                                                   float* __restrict__ part) {
    __shared__ float rows[16][kPC];
    const int c = threadIdx.x & (kPC - 1), r = threadIdx.x >> 4;
    float s = 0.f;
    for (long long v = (long long)blockIdx.x * 16 + r; v < V; v += (long long)gridDim.x * 16)
        s += __bfloat162float(gz[v * kPC + c]);
    rows[r][c] = s;
    __syncthreads();
    if (threadIdx.x < kPC) {
        float t = 0.f;
        for (int k = 0; k < 16; ++k) t += rows[k][threadIdx.x];
        part[blockIdx.x * kPC + threadIdx.x] = t;
    }
}

// Packed FP32 parameters -> padded BF16 forward weights [o][co][ci], data-
// gradient weights [o'][ci][co] (o' = the opposite offset) and FP32 biases.
__global__ void k_pack_weights(const float* __restrict__ params, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wb, float* __restrict__ bias) {
    const int layer = blockIdx.x;
    const int ci_n = layer_in(layer), co_n = layer_out(layer);
    int off = 0;
    for (int l = 0; l < layer; ++l) off += kOffsets * layer_in(l) * layer_out(l) + layer_out(l);
    const float* Wl = params + off;
    const float* bl = Wl + kOffsets * ci_n * co_n;
    __nv_bfloat16* f = wf + (size_t)layer * kOffsets * kPC * kPC;
    __nv_bfloat16* b = wb + (size_t)layer * kOffsets * kPC * kPC;
    for (int e = threadIdx.x; e < kOffsets * kPC * kPC; e += blockDim.x) {
        const int o = e / (kPC * kPC), r = (e / kPC) % kPC, c = e % kPC;
        // forward: [o][co = r][ci = c]
        const float vf = (r < co_n && c < ci_n) ? Wl[(o * ci_n + c) * co_n + r] : 0.f;
        f[e] = __float2bfloat16_rn(vf);
        // data gradient: output channel = ci (r), input channel = co (c), offset flipped
        const int of = kOffsets - 1 - o;
        const float vb = (r < ci_n && c < co_n) ? Wl[(of * ci_n + r) * co_n + c] : 0.f;
        b[e] = __float2bfloat16_rn(vb);
    }
    if (threadIdx.x < kPC) bias[layer * kPC + threadIdx.x] = threadIdx.x < co_n ? bl[threadIdx.x] : 0.f;
}

// Padded weight / bias gradients -> packed gradient vector.
__global__ void k_pack_grads(const float* __restrict__ dW, const float* __restrict__ db,
                             float* __restrict__ grads) {
    const int layer = blockIdx.x;
    const int ci_n = layer_in(layer), co_n = layer_out(layer);
    int off = 0;
    for (int l = 0; l < layer; ++l) off += kOffsets * layer_in(l) * layer_out(l) + layer_out(l);
    const float* d = dW + (size_t)layer * kOffsets * kPC * kPC;
    for (int e = threadIdx.x; e < kOffsets * ci_n * co_n; e += blockDim.x) {
        const int o = e / (ci_n * co_n), ci = (e / co_n) % ci_n, co = e % co_n;
        grads[off + e] = d[(o * kPC + ci) * kPC + co];
    }
    if (threadIdx.x < co_n)
        grads[off + kOffsets * ci_n * co_n + threadIdx.x] = db[layer * kPC + threadIdx.x];
}

// Adam (Kingma & Ba, 2015) on the FP32 master parameters.
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ learned-step mesh kernels

constexpr int kErrBlocks = 1216;  // blocks of the force-error reduction (8 per SM)
constexpr int kBiasBlocks = 152;

// phi_K(n) = D_K(n) phi_c: the volume fractions of an int64 fixed-point mesh.
__global__ void k_mesh_to_phi(const unsigned long long* __restrict__ D, long long n, double phi_c,
                              float* __restrict__ phi) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) phi[i] = (float)((double)(long long)D[i] * phi_c);
}

// D_out = max(0, D_base + rint(dphi * frac / phi_c)): a predicted density in
// the mesh's fixed point (D_base == nullptr: from zero).  In place is allowed.
__global__ void k_mesh_predict(const unsigned long long* D_base, const float* __restrict__ dphi,
                               long long n, double frac_over_phi_c, unsigned long long* D_out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const long long base = D_base ? (long long)D_base[i] : 0ll;
    long long d = base + __double2ll_rn((double)dphi[i] * frac_over_phi_c);
    D_out[i] = (unsigned long long)(d > 0 ? d : 0ll);
}

// Partials part[block] = (sum (Fa - Fb)^2, sum Fb^2) in FP64.
__global__ void __launch_bounds__(256) k_force_error(const float* __restrict__ Fa,
                                                     const float* __restrict__ Fb, long long n,
                                                     double* __restrict__ part) {
    __shared__ double sh[2][8];
    double e = 0.0, r = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double b = Fb[i], d = (double)Fa[i] - b;
        e += d * d;
        r += b * b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        r += __shfl_down_sync(0xffffffffu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = e;
        sh[1][threadIdx.x >> 5] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sr = 0.0;
        for (int k = 0; k < 8; ++k) {
            se += sh[0][k];
            sr += sh[1][k];
        }
        part[2 * blockIdx.x] = se;
        part[2 * blockIdx.x + 1] = sr;
    }
}

void launch_mesh_to_phi(const unsigned long long* D, long long n, double phi_c, float* phi,
                        cudaStream_t s) {
    if (n > 0) k_mesh_to_phi<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D, n, phi_c, phi);
}

void launch_mesh_predict(const unsigned long long* D_base, const float* dphi, long long n,
                         double frac_over_phi_c, unsigned long long* D_out, cudaStream_t s) {
    if (n > 0)
        k_mesh_predict<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D_base, dphi, n,
                                                                   frac_over_phi_c, D_out);
}

int force_error_partials() { return kErrBlocks; }

void launch_force_error(const float* Fa, const float* Fb, long long n, double* acc,
                        cudaStream_t s) {
    long long blocks = (n + 255) / 256;
    if (blocks > kErrBlocks) blocks = kErrBlocks;
    if (blocks < 1) blocks = 1;
    k_force_error<<<(unsigned)blocks, 256, 0, s>>>(Fa, Fb, n, acc + 2);
    k_sum_partials<double><<<1, 32, 0, s>>>(acc + 2, (int)blocks, 2, acc);
}

// ------------------------------------------------------------------ host side

int prop_param_count() {
    int n = 0;
    for (int l = 0; l < 3; ++l) n += kOffsets * layer_in(l) * layer_out(l) + layer_out(l);
    return n;
}

}  // namespace hpf

using namespace hpf;

struct hpf_prop {
    cudaStream_t stream = nullptr;
    PropGeom g{};
    float scale = 1.f;  // change-channel scale (input times, output divided by)
    int np = 0;
    float* params = nullptr;  // FP32 master [np]
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_t = 0;
    __nv_bfloat16* wf = nullptr;  // [3][27][16][16]
    __nv_bfloat16* wb = nullptr;
    float* bias = nullptr;        // [3][16]
    float* dW = nullptr;          // [3][27][16][16]
    float* db = nullptr;          // [3][16]
    float* wpart = nullptr;       // weight-gradient partials [grid_wgrad][27][16][16]
    float* bpart = nullptr;       // bias-gradient partials [152][16]
    double* lpart = nullptr;      // loss partials [ceil(V / 256)]
    __nv_bfloat16* act[4] = {};   // input, h1, h2, and a gradient buffer [V][16]
    float* z[2] = {};             // pre-activations of layers 1, 2 [V][16]
    float* fbuf = nullptr;        // FP32 [V][16]: output / data gradient
    float* xin = nullptr;         // staging of the planar input [4][V]
    float* tin = nullptr;         // staging of the planar next densities [2][V]
    float* yout = nullptr;        // planar output [2][V]
    double* loss = nullptr;
    double* h_loss = nullptr;
    int grid_wgrad = 0;
};

namespace {

hpf_status prop_copy_out(hpf_prop* p, void* dst, const void* src, size_t bytes) {
    if (!dst) return HPF_OK;
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, dst) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (!dev && cudaStreamSynchronize(p->stream) != cudaSuccess) return HPF_ERR_CUDA;
    return HPF_OK;
}

// Forward pass of planar input x [4][V] (device); leaves the FP32 output in
// fbuf.  With keep_z the pre-activations are stored for a backward pass.
void prop_forward(hpf_prop* p, const float* x, bool keep_z, cudaStream_t s) {
    const int V = p->g.V, tb = (V + 255) / 256;
    const size_t wl = (size_t)kOffsets * kPC * kPC;
    k_pack_input<<<tb, 256, 0, s>>>(x, V, p->scale, p->act[0]);
    k_conv<kHidden, 2><<<p->g.tiles, 256, 0, s>>>(p->act[0], p->wf, p->bias,
                                                   keep_z ? p->z[0] : nullptr, p->act[1], nullptr,
                                                   p->g);
    k_conv<kHidden, 2><<<p->g.tiles, 256, 0, s>>>(p->act[1], p->wf + wl, p->bias + kPC,
                                                   keep_z ? p->z[1] : nullptr, p->act[2], nullptr,
                                                   p->g);
    // two output channels: one n-tile (channels 8..15 of fbuf are not written)
    k_conv<kLast, 1><<<p->g.tiles, 256, 0, s>>>(p->act[2], p->wf + 2 * wl, p->bias + 2 * kPC,
                                                 nullptr, nullptr, p->fbuf, p->g);
}

// Loss and packed gradients (p->grads, p->loss) after prop_forward(keep_z) of
// x; the target is phi_next - x[2:4].
void prop_backward(hpf_prop* p, const float* x, const float* phi_next) {
    const int V = p->g.V, tb = (V + 255) / 256;
    const long long nv = (long long)V * kPC;
    const size_t wl = (size_t)kOffsets * kPC * kPC;
    cudaStream_t s = p->stream;
    __nv_bfloat16* gbuf = p->act[3];
    // the last layer has no activation: its gz is dL/dy
    k_loss<<<tb, 256, 0, s>>>(p->fbuf, x + 2 * (size_t)V, phi_next, V, p->scale, gbuf, p->lpart);
    k_sum_partials<double><<<1, 32, 0, s>>>(p->lpart, tb, 1, p->loss);
    for (int layer = 2; layer >= 0; --layer) {
        k_conv_wgrad<<<p->grid_wgrad, 256, 0, s>>>(p->act[layer], gbuf, p->wpart, p->g);
        k_sum_partials<float><<<(unsigned)((wl + 255) / 256), 256, 0, s>>>(
            p->wpart, p->grid_wgrad, (int)wl, p->dW + layer * wl);
        k_bias_grad<<<kBiasBlocks, 256, 0, s>>>(gbuf, V, p->bpart);
        k_sum_partials<float><<<1, 32, 0, s>>>(p->bpart, kBiasBlocks, kPC, p->db + layer * kPC);
        if (layer == 0) break;
        // the data gradient of the layer input, then through the SiLU below it
        k_conv<kData, 2><<<p->g.tiles, 256, 0, s>>>(gbuf, p->wb + layer * wl, nullptr, nullptr,
                                                     nullptr, p->fbuf, p->g);
        k_silu_backward<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(p->fbuf, p->z[layer - 1], nv,
                                                                      gbuf);
    }
    k_pack_grads<<<3, 256, 0, s>>>(p->dW, p->db, p->grads);
}

void prop_adam(hpf_prop* p, const float* grads, float lr) {
    p->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = (float)(1.0 - pow(0.9, (double)p->adam_t));
    const float c2 = (float)(1.0 - pow(0.999, (double)p->adam_t));
    k_adam<<<(p->np + 255) / 256, 256, 0, p->stream>>>(p->params, grads, p->adam_m, p->adam_v,
                                                      p->np, lr, b1, b2, 1e-8f, c1, c2);
    k_pack_weights<<<3, 256, 0, p->stream>>>(p->params, p->wf, p->wb, p->bias);
}

// Planar inputs are staged into library buffers (host or device sources).
hpf_status prop_stage(hpf_prop* p, float* dst, const float* src, size_t n) {
    if (!src) return HPF_ERR_INVALID;
    if (cudaMemcpyAsync(dst, src, sizeof(float) * n, cudaMemcpyDefault, p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    return HPF_OK;
}

hpf_status prop_read_loss(hpf_prop* p, double* loss) {
    if (!loss) return HPF_OK;
    if (cudaMemcpyAsync(p->h_loss, p->loss, sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    *loss = *p->h_loss;
    return HPF_OK;
}

hpf_status prop_launched(hpf_prop* p) {
    (void)p;
    return cudaGetLastError() == cudaSuccess ? HPF_OK : HPF_ERR_CUDA;
}

}  // namespace

namespace hpf {

bool prop_mesh_is(const hpf_prop* p, const MeshGeom& g) {
    return p && p->g.mx == g.mx && p->g.my == g.my && p->g.mz == g.mz;
}

void prop_predict(hpf_prop* p, const float* x, float* dphi, cudaStream_t s) {
    prop_forward(p, x, false, s);
    k_unpack_output<<<(p->g.V + 255) / 256, 256, 0, s>>>(p->fbuf, p->g.V, p->scale, dphi);
}

}  // namespace hpf

extern "C" {

hpf_status hpf_prop_init(const int32_t mesh[3], void* stream, hpf_prop** out) {
    if (!out || !mesh) return HPF_ERR_INVALID;
    *out = nullptr;
    long long V = 1;
    for (int a = 0; a < 3; ++a) {
        if (mesh[a] < 2 || mesh[a] > 1024) return HPF_ERR_INVALID;
        V *= mesh[a];
    }
    if (V > (1ll << 26)) return HPF_ERR_INVALID;
    hpf_prop* p = new hpf_prop();
    p->stream = (cudaStream_t)stream;
    PropGeom& g = p->g;
    g.mx = mesh[0];
    g.my = mesh[1];
    g.mz = mesh[2];
    g.V = (int)V;
    g.tiles_x = (g.mx + kTX - 1) / kTX;
    g.tiles_y = (g.my + kTY - 1) / kTY;
    g.tiles_z = (g.mz + kTZ - 1) / kTZ;
    g.tiles = g.tiles_x * g.tiles_y * g.tiles_z;
    p->np = prop_param_count();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaGetLastError();
    if (sms < 1) sms = 1;
    p->grid_wgrad = g.tiles < 2 * sms ? g.tiles : 2 * sms;
    const size_t wl = (size_t)kOffsets * kPC * kPC, Vs = (size_t)g.V;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&p->params, sizeof(float) * p->np);
    e = e ? e : cudaMalloc(&p->grads, sizeof(float) * p->np);
    e = e ? e : cudaMalloc(&p->adam_m, sizeof(float) * p->np);
    e = e ? e : cudaMalloc(&p->adam_v, sizeof(float) * p->np);
    e = e ? e : cudaMalloc(&p->wf, sizeof(__nv_bfloat16) * 3 * wl);
    e = e ? e : cudaMalloc(&p->wb, sizeof(__nv_bfloat16) * 3 * wl);
    e = e ? e : cudaMalloc(&p->bias, sizeof(float) * 3 * kPC);
    e = e ? e : cudaMalloc(&p->dW, sizeof(float) * 3 * wl);
    e = e ? e : cudaMalloc(&p->db, sizeof(float) * 3 * kPC);
    e = e ? e : cudaMalloc(&p->wpart, sizeof(float) * (size_t)p->grid_wgrad * wl);
    e = e ? e : cudaMalloc(&p->bpart, sizeof(float) * kBiasBlocks * kPC);
    e = e ? e : cudaMalloc(&p->lpart, sizeof(double) * ((Vs + 255) / 256));
    for (int k = 0; k < 4; ++k) e = e ? e : cudaMalloc(&p->act[k], sizeof(__nv_bfloat16) * Vs * kPC);
    for (int k = 0; k < 2; ++k) e = e ? e : cudaMalloc(&p->z[k], sizeof(float) * Vs * kPC);
    e = e ? e : cudaMalloc(&p->fbuf, sizeof(float) * Vs * kPC);
    e = e ? e : cudaMalloc(&p->xin, sizeof(float) * Vs * 4);
    e = e ? e : cudaMalloc(&p->tin, sizeof(float) * Vs * 2);
    e = e ? e : cudaMalloc(&p->yout, sizeof(float) * Vs * 2);
    e = e ? e : cudaMalloc(&p->loss, sizeof(double));
    e = e ? e : cudaMallocHost(&p->h_loss, sizeof(double));
    if (e == cudaSuccess) {
        // zero weights until hpf_prop_set_weights: the network predicts no change
        cudaMemsetAsync(p->params, 0, sizeof(float) * p->np, p->stream);
        cudaMemsetAsync(p->adam_m, 0, sizeof(float) * p->np, p->stream);
        cudaMemsetAsync(p->adam_v, 0, sizeof(float) * p->np, p->stream);
        k_pack_weights<<<3, 256, 0, p->stream>>>(p->params, p->wf, p->wb, p->bias);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        hpf_prop_destroy(p);
        return e == cudaErrorMemoryAllocation ? HPF_ERR_NOMEM : HPF_ERR_CUDA;
    }
    *out = p;
    return HPF_OK;
}

hpf_status hpf_prop_destroy(hpf_prop* p) {
    if (!p) return HPF_OK;
    cudaStreamSynchronize(p->stream);
    cudaFree(p->params);
    cudaFree(p->grads);
    cudaFree(p->adam_m);
    cudaFree(p->adam_v);
    cudaFree(p->wf);
    cudaFree(p->wb);
    cudaFree(p->bias);
    cudaFree(p->dW);
    cudaFree(p->db);
    cudaFree(p->wpart);
    cudaFree(p->bpart);
    cudaFree(p->lpart);
    for (int k = 0; k < 4; ++k) cudaFree(p->act[k]);
    for (int k = 0; k < 2; ++k) cudaFree(p->z[k]);
    cudaFree(p->fbuf);
    cudaFree(p->xin);
    cudaFree(p->tin);
    cudaFree(p->yout);
    cudaFree(p->loss);
    cudaFreeHost(p->h_loss);
    cudaGetLastError();
    delete p;
    return HPF_OK;
}

int32_t hpf_prop_param_count(void) { return prop_param_count(); }

hpf_status hpf_prop_set_weights(hpf_prop* p, const float* params) {
    if (!p || !params) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->params, params, (size_t)p->np);
    if (s != HPF_OK) return s;
    cudaMemsetAsync(p->adam_m, 0, sizeof(float) * p->np, p->stream);
    cudaMemsetAsync(p->adam_v, 0, sizeof(float) * p->np, p->stream);
    p->adam_t = 0;
    k_pack_weights<<<3, 256, 0, p->stream>>>(p->params, p->wf, p->wb, p->bias);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess)
        return HPF_ERR_CUDA;
    return HPF_OK;
}

hpf_status hpf_prop_get_weights(hpf_prop* p, float* params) {
    if (!p || !params) return HPF_ERR_INVALID;
    return prop_copy_out(p, params, p->params, sizeof(float) * p->np);
}

hpf_status hpf_prop_set_scale(hpf_prop* p, float scale) {
    if (!p || !(scale > 0.f) || !(scale < 3.0e38f)) return HPF_ERR_INVALID;
    p->scale = scale;
    return HPF_OK;
}

hpf_status hpf_prop_get_scale(const hpf_prop* p, float* scale) {
    if (!p || !scale) return HPF_ERR_INVALID;
    *scale = p->scale;
    return HPF_OK;
}

hpf_status hpf_prop_forward(hpf_prop* p, const float* x, float* dphi) {
    if (!p || !dphi) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->xin, x, (size_t)p->g.V * 4);
    if (s != HPF_OK) return s;
    prop_predict(p, p->xin, p->yout, p->stream);
    if ((s = prop_launched(p)) != HPF_OK) return s;
    return prop_copy_out(p, dphi, p->yout, sizeof(float) * 2 * p->g.V);
}

hpf_status hpf_prop_backward(hpf_prop* p, const float* x, const float* phi_next, float* grads,
                             double* loss) {
    if (!p) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->xin, x, (size_t)p->g.V * 4);
    if (s == HPF_OK) s = prop_stage(p, p->tin, phi_next, (size_t)p->g.V * 2);
    if (s != HPF_OK) return s;
    prop_forward(p, p->xin, true, p->stream);
    prop_backward(p, p->xin, p->tin);
    if ((s = prop_launched(p)) != HPF_OK) return s;
    if ((s = prop_copy_out(p, grads, p->grads, sizeof(float) * p->np)) != HPF_OK) return s;
    return prop_read_loss(p, loss);
}

hpf_status hpf_prop_adam_step(hpf_prop* p, const float* grads, float lr) {
    if (!p || !grads || !(lr > 0.f)) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->grads, grads, (size_t)p->np);
    if (s != HPF_OK) return s;
    prop_adam(p, p->grads, lr);
    return prop_launched(p);
}

hpf_status hpf_prop_train_step(hpf_prop* p, const float* x, const float* phi_next, float lr,
                               double* loss) {
    if (!p || !(lr > 0.f)) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->xin, x, (size_t)p->g.V * 4);
    if (s == HPF_OK) s = prop_stage(p, p->tin, phi_next, (size_t)p->g.V * 2);
    if (s != HPF_OK) return s;
    prop_forward(p, p->xin, true, p->stream);
    prop_backward(p, p->xin, p->tin);
    prop_adam(p, p->grads, lr);
    if ((s = prop_launched(p)) != HPF_OK) return s;
    return prop_read_loss(p, loss);
}

}  // extern "C"
