// k_prop.cu -- the learned density propagator: a 3-D periodic conv net
// (4 -> 16 -> 16 -> 2 channels, 3x3x3 kernels, SiLU) on BF16 tensor cores.
//
// Forward convolutions (k_conv_sweep): persistent, warp-specialised kernels
// that sweep columns of the mesh along z -- TMA loads of padded activation
// planes, tcgen05 MMAs with tensor-memory accumulators in a ring of output
// planes, an epilogue that gathers the x offsets from neighbouring lanes.
// Activations between the forward layers live in a periodically padded
// layout [2][Mz + 2][PY][PX][8] (channel halves planar); the first layer's
// four input channels enter as an x-im2col, so its three x offsets share one
// K = 16 step.  Training keeps the plain channels-last layout [V][16] for the
// back-propagated gradients: the data-gradient convolutions run on a tiled
// tcgen05 kernel (k_conv_tc), the weight gradient reduces over voxels with
// warp-level MMAs (ldmatrix.trans operands), accumulating in registers over
// many tiles before writing one partial block per CTA.
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <chrono>
#include <string>

#include "hpf_internal.cuh"

namespace hpf {

constexpr int kPC = 16;                      // padded channels
constexpr int kTX = 8, kTY = 8, kTZ = 8;     // output tile: one z-plane of 64 voxels per warp
constexpr int kBX = kTX + 2, kBY = kTY + 2, kBZ = kTZ + 2;
constexpr int kBoxVox = kBX * kBY * kBZ;     // 1000 (32 000 bytes)
constexpr int kTileVox = kTX * kTY * kTZ;    // 512
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

// Where the voxels of an activation buffer live: channel half h (8 channels)
// of voxel (x, y, z) at element (((z + off) ly + y + off) lx + x + off) vs +
// h hs -- the plain layout [V][16] (lx = Mx, ly = My, off = 0, vs = 16, hs =
// 8) or the padded one of the forward convolutions [2][Mz + 2][PY][PX][8]
// (off = 1, vs = 8, hs = (Mz + 2) PY PX 8).
struct ActLayout {
    int lx, ly, off;
    long long vs, hs;
};

// Periodic input box of a tile (all 16 channels), 16-byte asynchronous copies.
__device__ __forceinline__ void load_box(const __nv_bfloat16* __restrict__ in, const PropGeom& g,
                                         const ActLayout& L, int x0, int y0, int z0, uint4* box) {
    const uint32_t box_s = saddr(box);
    for (int e = threadIdx.x; e < kBoxVox * 2; e += blockDim.x) {
        const int v = e >> 1, half = e & 1;
        const int bx = v % kBX, by = (v / kBX) % kBY, bz = v / (kBX * kBY);
        const int gx = pwrap(x0 - 1 + bx, g.mx), gy = pwrap(y0 - 1 + by, g.my),
                  gz = pwrap(z0 - 1 + bz, g.mz);
        const size_t gv = ((size_t)(gz + L.off) * L.ly + gy + L.off) * L.lx + gx + L.off;
        cp_async16(box_s + 16 * swz(v, half), in + gv * L.vs + half * L.hs);
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

// ------------------------------------------------------------------ tcgen05 data gradients
//
// The data-gradient convolutions of training (a convolution of the back-
// propagated gradient with flipped, transposed weights, no bias, FP32 out) on
// the fifth-generation tensor cores.  A CTA (one warpgroup) works on tiles of
// 8 x 16 x 4 voxels of the plain channels-last layout [V][16]; a
// z-plane of a tile is 128 voxels = the 128 rows of one MMA (eight
// x-consecutive voxels per 8-row core-matrix group, one group per y row).
// The periodic 10 x 18 x 6 input box sits in shared memory as two planes of
// 8-channel halves (16 bytes per voxel): the canonical K-major layout without
// swizzle, so the box shifted by any in-plane offset (dy, dx) is a matrix
// descriptor that starts at the shifted voxel (K halves one plane apart,
// 8-row groups one box row apart).
//
// Each input plane z (box planes -1 .. 4 of the tile) feeds the output planes
// z + 1, z and z - 1 through the kernel offsets dz = -1, 0, +1 (an output
// voxel n sums W[d] in(n + d)).  So the weights of one in-plane offset are
// stacked for the three dz values as N = 3 x 16 columns, and the accumulators
// of the four output planes sit in tensor memory in reverse order, 16 columns
// each: the three planes an input plane feeds are then 48 consecutive columns,
// and one tcgen05.mma (M 128, N 48, K 16, BF16 in, FP32 accumulate) per input
// plane and in-plane offset updates all three; at the tile's first and last
// input planes fewer planes exist (N = 16 or 32).  That is 6 x 9 MMAs per
// tile instead of 27 x 4 of width 16, and every MMA reads its A operand once
// for three output planes.  The accumulators are cleared by tcgen05.st
// before the tile's MMAs, which then all accumulate.
//
// One thread issues the MMAs and commits them to an mbarrier; all eight warps
// then read the accumulators back (tcgen05.ld) for the FP32 stores.  Waits are
// bounded (kTcWaitLimit polls);
// a wait that gives up sets kFlagTimeout and the CTA stops after releasing
// its tensor memory.
constexpr int kTcX = 8, kTcY = 16, kTcZ = 4;
constexpr int kTcBX = kTcX + 2, kTcBY = kTcY + 2, kTcBZ = kTcZ + 2;
constexpr int kTcPlane = kTcBX * kTcBY;   // box voxels per z-plane
constexpr int kTcBox = kTcPlane * kTcBZ;  // 1080 voxels per channel half
constexpr int kTcInPlane = 9;             // in-plane offsets (dy, dx)
constexpr int kTcRows16 = 48;             // B rows per in-plane offset: (dz, co)
constexpr int kTcCols = 64;               // accumulator columns per set: 4 planes x 16
constexpr unsigned kTcWaitLimit = 1u << 22;
constexpr int kTcThreads = 256;          // two warps per tensor-memory lane quarter
constexpr int kTcWCopies = 8;            // replicas of each packed weight image (spread L2 reads)
// shared memory of a CTA with kBuf box buffers (and kBuf accumulator sets)
constexpr size_t tc_smem_bytes(int kBuf) {
    return sizeof(uint4) * ((size_t)kBuf * 2 * kTcBox + 2 * kTcInPlane * kTcRows16) + 64;
}

// The weight images of the data-gradient convolutions, [copy][half][in-plane
// offset][B row]: 0 the second layer's, 1 the last layer's.
constexpr int kTcImages = 2;
constexpr int kTcImageWords = 2 * kTcInPlane * kTcRows16;  // uint4 per copy
__host__ __device__ constexpr int tc_image_offset(int k) {  // uint4, all copies
    return k * kTcWCopies * kTcImageWords;
}

// Shared-memory matrix descriptor: start address, leading and stride byte
// offsets (all in 16-byte units), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t umma_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (unsigned it = 0; it < kTcWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tc_origin(const PropGeom& g, int t, int& x0, int& y0, int& z0) {
    const int tx = (g.mx + kTcX - 1) / kTcX, ty = (g.my + kTcY - 1) / kTcY;
    x0 = (t % tx) * kTcX;
    y0 = ((t / tx) % ty) * kTcY;
    z0 = (t / (tx * ty)) * kTcZ;
}

// Box of the tile at (x0, y0, z0) into the buffer at shared address box_s:
// 16-byte asynchronous copies of channel halves, [half][voxel].
// i in [-1, m + box extent]: one period at most when m spans the box extent
// (near), the general remainder otherwise.
__device__ __forceinline__ int tc_wrap(int i, int m, bool near) {
    if (near) return i < 0 ? i + m : (i >= m ? i - m : i);
    return pwrap(i, m);
}

// A thread's share of the box copies: elements e = tid + kTcThreads k of the
// [voxel][half] order, their box coordinates and shared-memory offsets, the
// same for every tile.
constexpr int kTcSlots = (kTcBox * 2 + kTcThreads - 1) / kTcThreads;

struct TcSlots {
    int c[kTcSlots];       // bx | by << 8 | bz << 16 | half << 24, or -1
    uint32_t s[kTcSlots];  // byte offset in a box buffer
};

__device__ __forceinline__ void tc_slots(TcSlots& sl) {
#pragma unroll
    for (int k = 0; k < kTcSlots; ++k) {
        const int e = threadIdx.x + kTcThreads * k;
        const int v = e >> 1, half = e & 1;
        const int bx = v % kTcBX, by = (v / kTcBX) % kTcBY, bz = v / kTcPlane;
        sl.c[k] = e < kTcBox * 2 ? (bx | (by << 8) | (bz << 16) | (half << 24)) : -1;
        sl.s[k] = (uint32_t)sizeof(uint4) * (uint32_t)(half * kTcBox + v);
    }
}

__device__ __forceinline__ void tc_load_box(const __nv_bfloat16* __restrict__ in,
                                            const PropGeom& g, int x0, int y0, int z0,
                                            uint32_t box_s, const TcSlots& sl, bool near) {
#pragma unroll
    for (int k = 0; k < kTcSlots; ++k) {
        const int c = sl.c[k];
        if (c < 0) continue;
        const int gx = tc_wrap(x0 - 1 + (c & 0xff), g.mx, near);
        const int gy = tc_wrap(y0 - 1 + ((c >> 8) & 0xff), g.my, near);
        const int gz = tc_wrap(z0 - 1 + ((c >> 16) & 0xff), g.mz, near);
        const int gv = (gz * g.my + gy) * g.mx + gx;
        cp_async16(box_s + sl.s[k], in + (size_t)gv * kPC + 8 * (c >> 24));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void tc_zero_cols16(uint32_t taddr) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(0u)
        : "memory");
}

// Epilogue of one output plane: the warp's 32 accumulator rows (lanes 32w ..)
// from columns col .. col + 15, voxel (x0 + row % 8, y0 + row / 8, z), FP32.
__device__ __forceinline__ void tc_epilogue(uint32_t tcol, const PropGeom& g, int x0, int y0,
                                            int z, float* __restrict__ f_out) {
    const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) & 3;  // lane quarter
    const uint32_t taddr = tcol + ((uint32_t)(32 * w) << 16);
    float acc[16];
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = __uint_as_float(r[c]);
    const int row = 32 * w + lane;
    const int X = x0 + (row & 7), Y = y0 + (row >> 3);
    if (X >= g.mx || Y >= g.my || z >= g.mz) return;
    const size_t gv = ((size_t)z * g.my + Y) * g.mx + X;
    float4* fo = reinterpret_cast<float4*>(f_out + gv * kPC);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        fo[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
}

// Wp: a packed weight image (k_pack_tc_image) of the data-gradient weights
// [27][16 out][16 in], offset index 9 dz_index + in-plane offset (dy, dx);
// K = 16 input channels of the plain layout [V][16].
template <int kBuf>
__global__ void __launch_bounds__(kTcThreads, kBuf == 1 ? 4 : 1)
    k_conv_tc(const __nv_bfloat16* __restrict__ in, const uint4* __restrict__ Wp,
              float* __restrict__ f_out, PropGeom g, int n_tiles, int* __restrict__ flag) {
    constexpr int kRows = kTcRows16, kIP = kTcInPlane;
    extern __shared__ __align__(128) uint4 tc_smem[];
    uint4* boxp = tc_smem;                    // [buffer][channel half][kTcBox]
    uint4* wp = tc_smem + kBuf * 2 * kTcBox;  // [channel half][in-plane offset][kRows]
    unsigned long long* bar =
        reinterpret_cast<unsigned long long*>(wp + 2 * kTcInPlane * kTcRows16);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar + 3);
    const int tid = threadIdx.x, w = tid >> 5;
    if (w == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_slot)),
                     "r"(kBuf * kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar[1])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar[2])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // B, pre-packed in its shared-memory layout (tc_pack_weights): one bulk
    // copy from one of kTcWCopies replicas of the image in global memory
    constexpr uint32_t kWBytes = (uint32_t)sizeof(uint4) * 2 * kIP * kRows;
    if (tid == 0) {
        const uint4* src = Wp + (size_t)(blockIdx.x % kTcWCopies) * (kWBytes / sizeof(uint4));
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         saddr(&bar[2])),
                     "r"(kWBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(saddr(wp)),
            "l"(src), "r"(kWBytes), "r"(saddr(&bar[2]))
            : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const uint32_t lbo_a = sizeof(uint4) * kTcBox, sbo_a = sizeof(uint4) * kTcBX;
    const uint32_t lbo_b = sizeof(uint4) * kIP * kRows, sbo_b = sizeof(uint4) * 8;
    const uint32_t box0 = saddr(boxp), wp0 = saddr(wp);
    const bool near = g.mx >= kTcBY && g.my >= kTcBY && g.mz >= kTcBY;
    TcSlots sl;
    tc_slots(sl);
    uint32_t phase[2] = {0u, 0u};
    int px0 = 0, py0 = 0, pz0 = 0;  // origin of the previous tile
    int i = 0;
    bool failed = false;
    bool w_ok = true;  // the weights arrived (thread 0)
    // the box of a tile is loaded one iteration ahead, into the buffer that the
    // MMAs of the tile before the previous one have finished reading
    int t = blockIdx.x;
    if (t < n_tiles) {
        int x0, y0, z0;
        tc_origin(g, t, x0, y0, z0);
        tc_load_box(in, g, x0, y0, z0, box0, sl, near);
    }
    for (; t < n_tiles; t += gridDim.x, ++i) {
        if (kBuf == 1 && i > 0) break;  // one tile per CTA (the grid covers the tiles)
        const int b = kBuf == 1 ? 0 : (i & 1);
        int x0, y0, z0;
        tc_origin(g, t, x0, y0, z0);
        if (i > 0) {
            // the MMAs of the previous tile: done before its box buffer is refilled
            // and before its epilogue
            const bool ok = tc_wait(saddr(&bar[b ^ 1]), phase[b ^ 1]);
            if (__syncthreads_or(!ok)) {  // every thread takes the same branch
                if (tid == 0) atomicOr(flag, kFlagTimeout);
                failed = true;
                break;
            }
            phase[b ^ 1] ^= 1u;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        const int tn = t + (int)gridDim.x;
        if (kBuf > 1 && tn < n_tiles) {
            int xn, yn, zn;
            tc_origin(g, tn, xn, yn, zn);
            tc_load_box(in, g, xn, yn, zn,
                        box0 + (uint32_t)(sizeof(uint4) * 2 * kTcBox) * (b ^ 1), sl, near);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        const uint32_t boxb = box0 + (uint32_t)(sizeof(uint4) * 2 * kTcBox) * b;
        // accumulator set b was last read by the epilogue of tile i - 2
        const uint32_t accb = tmem + (uint32_t)(kTcCols * b);
#pragma unroll
        for (int c = 0; c < kTcCols / 2; c += 16)
            tc_zero_cols16(accb + (w >> 2) * (kTcCols / 2) + c + ((uint32_t)(32 * (w & 3)) << 16));
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0 && i == 0) {
            // the bulk copy of the weights (issued in the prologue)
            w_ok = tc_wait(saddr(&bar[2]), 0u);
            if (!w_ok) atomicOr(flag, kFlagTimeout);
        }
        if (tid == 0 && w_ok) {
            // descriptors: the start-address field is the low 14 bits (16-byte
            // units); offsets inside shared memory are added to it directly
            const uint64_t a0 = umma_smem_desc(boxb, lbo_a, sbo_a);
            const uint64_t b0 = umma_smem_desc(wp0, lbo_b, sbo_b);
#pragma unroll
            for (int z = -1; z <= kTcZ; ++z) {
                const int pf = z + 1 < kTcZ - 1 ? z + 1 : kTcZ - 1;  // first plane fed
                const int pl = z - 1 > 0 ? z - 1 : 0;                 // last plane fed
                const int N = 16 * (pf - pl + 1);
                const uint32_t idesc = umma_idesc_bf16(128, N);
                const uint32_t d = accb + (uint32_t)(16 * (kTcZ - 1 - pf));
                const int row0 = 16 * (z - pf + 1);  // B row of the first plane's dz
#pragma unroll
                for (int o9 = 0; o9 < kIP; ++o9) {
                    const int dy = o9 / 3 - 1, dx = o9 % 3 - 1;
                    const int v0 = ((z + 1) * kTcBY + (1 + dy)) * kTcBX + (1 + dx);
                    const uint64_t ad = a0 + (uint64_t)v0;
                    const uint64_t bd = b0 + (uint64_t)(o9 * kRows + row0);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\t"
                        "setp.ne.u32 p, 1, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                        "l"(ad), "l"(bd), "r"(idesc)
                        : "memory");
                }
            }
        }
        if (tid == 0)
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    saddr(&bar[b]))
                : "memory");
        if (i > 0) {
            // epilogue of the previous tile while this one is on the tensor cores
            const uint32_t accp = tmem + (uint32_t)(kTcCols * (b ^ 1));
#pragma unroll 1
            for (int p = 2 * (w >> 2); p < 2 * (w >> 2) + 2; ++p)
                tc_epilogue(accp + (uint32_t)(16 * (kTcZ - 1 - p)), g, px0, py0, pz0 + p, f_out);
        }
        px0 = x0;
        py0 = y0;
        pz0 = z0;
    }
    if (!failed && i > 0) {
        const int pb = (i - 1) & 1;
        const bool ok = tc_wait(saddr(&bar[pb]), phase[pb]);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) atomicOr(flag, kFlagTimeout);
            failed = true;
        } else {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t accp = tmem + (uint32_t)(kTcCols * pb);
#pragma unroll 1
            for (int p = 2 * (w >> 2); p < 2 * (w >> 2) + 2; ++p)
                tc_epilogue(accp + (uint32_t)(16 * (kTcZ - 1 - p)), g, px0, py0, pz0 + p, f_out);
        }
    }
    if (failed) {
        // MMAs of the last tiles may still be in flight: one more bounded wait on
        // each accumulator set before the tensor memory is released
        tc_wait(saddr(&bar[0]), phase[0]);
        if (kBuf > 1) tc_wait(saddr(&bar[1]), phase[1]);
    }
    if (tid == 0 && (!w_ok || i == 0)) tc_wait(saddr(&bar[2]), 0u);  // the weights' bulk copy
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (w == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kBuf * kTcCols)
                     : "memory");
}

int conv_tc_tiles(const PropGeom& g) {
    return ((g.mx + kTcX - 1) / kTcX) * ((g.my + kTcY - 1) / kTcY) * ((g.mz + kTcZ - 1) / kTcZ);
}

// One tile per CTA, single-buffered (48 KB of shared memory and 64
// tensor-memory columns per CTA, four CTAs per SM overlap one another's box
// loads, MMAs and epilogues); the attribute is set once per device.
void conv_tc_setup() {
    static std::once_flag once[64];
    once_per_device(once, [] {
        cudaFuncSetAttribute(k_conv_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tc_smem_bytes(1));
        cudaGetLastError();
    });
}

// Data-gradient convolution of in [V][16] with weight image k of tcw into
// f_out [V][16] FP32.
void launch_conv_tc(const __nv_bfloat16* in, const uint4* tcw, int k, float* f_out,
                    const PropGeom& g, int* flag, cudaStream_t s) {
    conv_tc_setup();
    const int n = conv_tc_tiles(g);
    k_conv_tc<1><<<n, kTcThreads, tc_smem_bytes(1), s>>>(in, tcw + tc_image_offset(k), f_out, g,
                                                         n, flag);
}

// Weight image k in the B layout of k_conv_tc, kTcWCopies times: from the
// padded BF16 weights W [27][16 out][16 in] (offset 9 dz_index + in-plane
// offset), row n = dz_index 16 + out channel.
__global__ void k_pack_tc_image(const __nv_bfloat16* __restrict__ W, int k,
                                uint4* __restrict__ tcw) {
    const int per = kTcImageWords, rows = kTcRows16, ip = kTcInPlane;
    const uint4* W4 = reinterpret_cast<const uint4*>(W);
    uint4* out = tcw + tc_image_offset(k);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int half = e / (ip * rows), rest = e % (ip * rows);
        const int o9 = rest / rows, n = rest % rows;
        const uint4 v = W4[(((n / 16) * ip + o9) * kPC + n % 16) * 2 + half];
        for (int c = 0; c < kTcWCopies; ++c) out[c * per + e] = v;
    }
}

// ------------------------------------------------------------------ z-sweep convolution
//
// The forward convolutions: persistent and warp-specialised.  The mesh is cut
// into columns of 14 x 8 output voxels (x, y) through the whole z extent; the
// output planes of all columns, in column-major order (column, z), are split
// evenly over the CTAs (one per SM), and a CTA sweeps its share plane by plane.
//
// Activations live in a periodically padded layout [2][Mz + 2][PY][PX][8] BF16
// (channel halves planar; one halo voxel on each side in x, y and z holding
// the opposite face; PX >= Mx + 2, PY >= My + 2), so the 16 x 10 voxel boxes
// of two consecutive input planes -- the column's 14 x 8 voxels with their x
// and y neighbours -- are one TMA box of twenty 256-byte rows per channel half
// (x and channel form the innermost dimension of the tensor map).  A stage
// holds two input planes.  In shared memory a plane's box is the canonical
// K-major layout without swizzle (8 channels = 16 bytes per voxel, core
// matrices of 8 x-consecutive voxels, the channel halves 5120 bytes apart),
// and its 128 voxels from box row dy + 1 on are the A operand
// (M = 128: 8 rows of 16) of the in-plane offset dy, a descriptor into the
// same box for every dy.
//
// For each dy, N stacks the weights of the three dz and, in the 16 -> 16
// layer, of the three dx as well.  An output voxel n sums W[d] in(n + d):
// input plane zi feeds output planes zi + 1, zi, zi - 1 (dz = -1, 0, +1), and
// the dx block of the product at box voxel u belongs to the output voxel
// u - dx, which the epilogue gathers from the neighbouring tensor-memory lanes
// with warp shuffles (a 16-voxel box row keeps x - 1 and x + 1 of each of its
// 14 interior voxels in the same warp).  So an input plane costs three MMAs
// (one per dy) of N up to 3 x 48 = 144 that read the box three times, not
// nine.  The first layer's x-im2col input (K index (dx + 1) 4 + ci) needs no
// dx block (N up to 48); the two-channel last layer keeps 16 columns per
// plane, 6 of them used (zero weight rows behind).
//
// Output planes accumulate in a ring of kSwRing tensor-memory slots in
// reverse column order, so the planes an input plane feeds are adjacent
// columns except where the ring wraps (the MMA is split there).  A slot
// starts at the bias (dx = 0 block) or zero and every MMA accumulates; the
// epilogue reads a finished plane, resets its slot and hands it back before
// its own arithmetic and stores.
//
// Warp 0: TMA producer (a ring of kSwStages two-plane stages); warp 1: owner
// of the tensor memory and MMA issuer; warps 2..9: epilogue, two per
// tensor-memory lane quarter, each with one channel half (8 channels).  Every wait is bounded; one that gives up raises
// kFlagTimeout and a shared abort word that ends every role's loop, after
// which the CTA waits (bounded) for its copies and MMAs in flight and
// releases its tensor memory.
constexpr int kSwOX = 14;                                // output voxels of a column along x
constexpr int kSwBX = 16, kSwY = 8, kSwBY = 10;          // box: x with halo, output rows, rows
constexpr uint32_t kSwPlaneBytes = 16u * kSwBX * kSwBY;  // one channel half of a plane box
constexpr uint32_t kSwHalfBytes = 2u * kSwPlaneBytes;    // one channel half of a stage
constexpr uint32_t kSwStageBytes = 2u * kSwHalfBytes;    // two input planes
constexpr int kSwStages = 9;
constexpr int kSwRingMax = 10;
constexpr int kSwEpiWarps = 8;                           // two per tensor-memory lane quarter
constexpr int kSwThreads = 32 * (2 + kSwEpiWarps);
constexpr int kSwPerSM = 2;                              // CTAs (sweeps) per SM
constexpr size_t kSwSmemFloor = 80 * 1024;               // at most two CTAs per SM

// layer kL: 0 first (x-im2col input), 1 second (16 -> 16), 2 last (16 -> 2)
__host__ __device__ constexpr int sw_cols(int L) { return L == 1 ? 48 : 16; }  // per plane
__host__ __device__ constexpr int sw_rows(int L) { return 3 * sw_cols(L); }    // B rows per dy
__host__ __device__ constexpr int sw_image_words(int L) { return 2 * 3 * sw_rows(L); }
__host__ __device__ constexpr int sw_image_offset(int L) {
    return L == 0 ? 0 : sw_image_offset(L - 1) + kTcWCopies * sw_image_words(L - 1);
}
// accumulator slots: 5 x 48 or 10 x 16 columns, 256 allocated (two CTAs per SM)
__host__ __device__ constexpr int sw_ring(int L) { return L == 1 ? 5 : 10; }
__host__ __device__ constexpr uint32_t sw_tmem_cols(int L) { return 256u; }
constexpr int kSwBars = 2 * kSwStages + kSwRingMax + 2;  // full, empty, acc full, weights, done
constexpr size_t sw_smem_bytes(int L) {
    return (size_t)1024 + (size_t)kSwStages * kSwStageBytes + 16 * (size_t)sw_image_words(L) +
                   8 * (size_t)kSwBars + 64 <
                   kSwSmemFloor
               ? kSwSmemFloor
               : (size_t)1024 + (size_t)kSwStages * kSwStageBytes +
                     16 * (size_t)sw_image_words(L) + 8 * (size_t)kSwBars + 64;
}

struct SweepArgs {
    const uint4* w;            // packed weight image of the layer (kTcWCopies replicas)
    const float* bias;         // [16]
    float* z_out;              // hidden: pre-activations [V][16] FP32 (optional)
    __nv_bfloat16* act_out;    // hidden: SiLU output, padded layout [2][Mz + 2][PY][PX][8]
    float* f_out;              // last: [V][16] FP32, channels 0 and 1 (optional)
    float* y_out;              // last: planar [2][V], times inv_scale (optional)
    float inv_scale;
    int* flag;
    int mx, my, mz, px, py;    // mesh and padded pitches
    int ncx, total;            // columns along x; output planes of all columns
    int withhold;              // self-test: no finished plane is signalled, so the
                               // epilogue's waits give up (hpf_prop_selftest_timeout)
};

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// A wait gives up after kTcWaitLimit polls or kSwWaitNs of wall time,
// whichever comes first (work that arrives at all arrives within
// microseconds); the clock is read every 64 polls.
constexpr unsigned long long kSwWaitNs = 200000000ull;

__device__ __forceinline__ unsigned long long sw_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool sw_late(unsigned it, unsigned long long t0) {
    return (it & 63u) == 63u && sw_now() - t0 > kSwWaitNs;
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool sw_wait(uint32_t bar, uint32_t parity, volatile int* abort_w,
                                        int* flag) {
    const unsigned long long t0 = sw_now();
    for (unsigned it = 0; it < kTcWaitLimit && !sw_late(it, t0); ++it) {
        if (mbar_test(bar, parity)) return true;
        if (*abort_w) return false;
    }
    *abort_w = 1;
    atomicOr(flag, kFlagTimeout);
    return false;
}

// Each epilogue warp counts the accumulator slots it has released (a release
// add after its tensor-memory reads and resets); a slot is free once every
// warp's count has passed it (acquire loads before the MMAs that reuse it).
// One count per warp: the warps drift apart by a few planes, and a sum could
// pass a plane that a slow warp has not read yet.
__device__ __forceinline__ void count_release(uint32_t addr) {
    asm volatile("red.release.cta.shared::cta.add.u32 [%0], 1;" ::"r"(addr) : "memory");
}

__device__ __forceinline__ uint32_t count_acquire(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.acquire.cta.shared::cta.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ bool mbar_test_now(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ void count_publish(uint32_t addr, uint32_t v) {
    asm volatile("st.release.cta.shared::cta.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ bool sw_wait_count(uint32_t addr, uint32_t target, uint32_t& known,
                                              volatile int* abort_w, int* flag) {
    if (known >= target) return true;
    const unsigned long long t0 = sw_now();
    for (unsigned it = 0; it < kTcWaitLimit && !sw_late(it, t0); ++it) {
        if (it) __nanosleep(32);
        known = count_acquire(addr);
        if (known >= target) return true;
        if (*abort_w) return false;
    }
    *abort_w = 1;
    atomicOr(flag, kFlagTimeout);
    return false;
}

// known: the smallest count seen so far (counts only grow), so that a target
// it already covers needs no loads.
__device__ __forceinline__ bool sw_wait_released(uint32_t addr, uint32_t target, uint32_t& known,
                                                 volatile int* abort_w, int* flag) {
    if (known >= target) return true;
    const unsigned long long t0 = sw_now();
    for (unsigned it = 0; it < kTcWaitLimit && !sw_late(it, t0); ++it) {
        if (it) __nanosleep(32);  // a poll leaves the issue slots to the working warps
        uint32_t m = count_acquire(addr);
#pragma unroll
        for (int w = 1; w < kSwEpiWarps; ++w) {
            const uint32_t c = count_acquire(addr + 4u * w);
            m = c < m ? c : m;
        }
        known = m;
        if (m >= target) return true;
        if (*abort_w) return false;
    }
    *abort_w = 1;
    atomicOr(flag, kFlagTimeout);
    return false;
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t ad, uint64_t bd, uint32_t idesc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, 1, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(ad), "l"(bd), "r"(idesc)
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
        "%10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(taddr));
#pragma unroll
    for (int c = 0; c < 8; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
        : "memory");
}

// Initial value of a slot, the columns of this warp's channel half g: the
// bias in the dx = 0 block (channels 8g .. 8g + 7 of the first layer, columns
// 16 + 8g .. of the second), zero elsewhere; the last layer's 16 columns
// (bias in columns 2 and 3) belong to the g = 0 warps.
template <int kL>
__device__ __forceinline__ void sw_reset_slot(uint32_t taddr, int g, const float (&binit)[16]) {
    float zero[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) zero[c] = 0.f;
    if (kL == 1) {
        tmem_st8(taddr + 8 * g, zero);
        tmem_st8(taddr + 16 + 8 * g, binit);
        tmem_st8(taddr + 32 + 8 * g, zero);
    } else if (kL == 0) {
        tmem_st8(taddr + 8 * g, binit);
    } else if (g == 0) {
        tmem_st16(taddr, binit);
    }
}

// One channel half (8 BF16 channels) of a voxel to the padded layout, with
// its periodic copies in the halo when it lies on a face (up to eight at a
// corner).
__device__ __forceinline__ void sw_store_half(__nv_bfloat16* __restrict__ act, const SweepArgs& a,
                                              int X, int Y, int Z, int h, uint4 v) {
    const int xs[2] = {X + 1, X == 0 ? a.mx + 1 : (X == a.mx - 1 ? 0 : -1)};
    const int ys[2] = {Y + 1, Y == 0 ? a.my + 1 : (Y == a.my - 1 ? 0 : -1)};
    const int zs[2] = {Z + 1, Z == 0 ? a.mz + 1 : (Z == a.mz - 1 ? 0 : -1)};
    uint4* base = reinterpret_cast<uint4*>(act) + (size_t)h * (a.mz + 2) * a.py * a.px;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (zs[k] < 0) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (ys[j] < 0) continue;
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                if (xs[i] < 0) continue;
                base[((size_t)zs[k] * a.py + ys[j]) * a.px + xs[i]] = v;
            }
        }
    }
}

// The output planes [q0, q1) of this CTA in the order q = column Mz + z.
__device__ __forceinline__ void sw_share(const SweepArgs& a, long long& q0, long long& q1) {
    q0 = (long long)a.total * blockIdx.x / gridDim.x;
    q1 = (long long)a.total * (blockIdx.x + 1) / gridDim.x;
}

// The run of output planes [zs, ze) of one column starting at q.
__device__ __forceinline__ void sw_chunk(const SweepArgs& a, long long q, long long q1, int& x0,
                                         int& y0, int& zs, int& ze) {
    const int col = (int)(q / a.mz);
    zs = (int)(q % a.mz);
    const long long left = q1 - q;
    ze = zs + (int)(left < (long long)(a.mz - zs) ? left : (long long)(a.mz - zs));
    x0 = (col % a.ncx) * kSwOX;
    y0 = (col / a.ncx) * kSwY;
}

// The stages of a CTA in order: each run of input planes zs - 1 .. ze of a
// column, two planes per stage (an odd run ends with a padding plane that no
// MMA reads).  zi: the stage's first input plane.
struct SwStages {
    long long q, q1;
    int x0, y0, zs, ze, zi;
    __device__ __forceinline__ void begin(const SweepArgs& a, long long q0, long long q1_) {
        q = q0;
        q1 = q1_;
        if (q < q1) {
            sw_chunk(a, q, q1, x0, y0, zs, ze);
            zi = zs - 1;
        }
    }
    __device__ __forceinline__ void next(const SweepArgs& a) {
        zi += 2;
        if (zi > ze) {
            q += ze - zs;
            if (q < q1) {
                sw_chunk(a, q, q1, x0, y0, zs, ze);
                zi = zs - 1;
            }
        }
    }
};

template <int kL>
__global__ void __launch_bounds__(kSwThreads, kSwPerSM)
    k_conv_sweep(const __grid_constant__ CUtensorMap tmap, const SweepArgs a) {
    constexpr int C = sw_cols(kL), RW = sw_rows(kL), kSwRing = sw_ring(kL);
    constexpr uint32_t kWBytes = 16u * sw_image_words(kL);
    extern __shared__ __align__(1024) uint8_t sw_raw[];
    const uint32_t raw_s = saddr(sw_raw);
    const uint32_t stage_s = (raw_s + 1023u) & ~1023u;  // TMA boxes, 1024-byte aligned
    uint8_t* base = sw_raw + (stage_s - raw_s);
    const uint32_t w_s = stage_s + kSwStages * kSwStageBytes;
    unsigned long long* bars =
        reinterpret_cast<unsigned long long*>(base + kSwStages * kSwStageBytes + kWBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + kSwBars);
    volatile int* abort_w = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint32_t* released = tmem_slot + 2;  // [kSwEpiWarps] slot releases per epilogue warp
    uint32_t* loaded = released + kSwEpiWarps;  // input planes landed in shared memory
    const uint32_t rel_s = saddr(released), loaded_s = saddr(loaded);
    const uint32_t bar0 = saddr(bars);
    // barrier k at bar0 + 8 k: full [0, S), empty [S, 2S), acc full [2S, 2S + R),
    // weights, done
    const uint32_t full_b = bar0, empty_b = bar0 + 8 * kSwStages;
    const uint32_t accf_b = bar0 + 16 * kSwStages;
    const uint32_t w_b = accf_b + 8 * kSwRingMax, done_b = w_b + 8;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the next layer may be scheduled now: its CTAs take an SM as ours leave it
    // and run their prologue while this grid finishes
    griddep_launch_dependents();
    if (tid == 0) {
        for (int k = 0; k < kSwBars; ++k)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * k) : "memory");
        *abort_w = 0;
        for (int w = 0; w < kSwEpiWarps; ++w) released[w] = 0;
        *loaded = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_slot)),
                     "r"(sw_tmem_cols(kL))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    const int eg = (warp - 2) >> 2;  // an epilogue warp's channel half
    float binit[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) binit[c] = 0.f;
    if (warp >= 2) {
        if (kL == 2) {
            binit[2] = a.bias[0];
            binit[3] = a.bias[1];
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) binit[c] = a.bias[8 * eg + c];
        }
    }
    const uint32_t lane_off = (uint32_t)(32 * (warp & 3)) << 16;
    if (warp >= 2) {
#pragma unroll 1
        for (int s = 0; s < kSwRing; ++s)
            sw_reset_slot<kL>(tmem + (uint32_t)((kSwRing - 1 - s) * C) + lane_off, eg, binit);
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    long long q0, q1;
    sw_share(a, q0, q1);
    int n_stages = 0;  // every run of input planes zs - 1 .. ze, padded to an even count
    for (long long q = q0; q < q1;) {
        int x0, y0, zs, ze;
        sw_chunk(a, q, q1, x0, y0, zs, ze);
        n_stages += (ze - zs + 3) / 2;
        q += ze - zs;
    }

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------------------- producer
        const uint4* src = a.w + (size_t)(blockIdx.x % kTcWCopies) * sw_image_words(kL);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(w_b),
                     "r"(kWBytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(w_s),
            "l"(src), "r"(kWBytes), "r"(w_b)
            : "memory");
        griddep_wait();  // the activations are the previous layer's output
        // Stages run up to kSwStages ahead (a stage is reused once the MMAs that
        // read it are done); between issues the producer watches the copies
        // land, in order, and publishes their count, so that the MMA thread
        // polls one word instead of a barrier per stage.
        SwStages in;
        in.begin(a, q0, q1);
        int si = 0, pub = 0;
        unsigned idle = 0;
        unsigned long long idle_t0 = 0;
        while (si < n_stages || pub < si) {
            bool progress = false;
            const int st = si % kSwStages;
            if (si < n_stages && mbar_test_now(empty_b + 8 * st, ((si / kSwStages) & 1) ^ 1)) {
                const uint32_t dst = stage_s + st * kSwStageBytes, fb = full_b + 8 * st;
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                             "r"(kSwStageBytes)
                             : "memory");
                // planes zi, zi + 1 at padded z = zi + 1 (0 .. Mz + 1): one box per
                // channel half; x0 8 elements = 16 x0 bytes keeps the copy aligned
#pragma unroll
                for (int h = 0; h < 2; ++h)
                    asm volatile(
                        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::"
                        "bytes [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst + h * kSwHalfBytes),
                        "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(8 * in.x0), "r"(in.y0),
                        "r"(in.zi + 1), "r"(h), "r"(fb)
                        : "memory");
                in.next(a);
                ++si;
                progress = true;
            }
            if (pub < si &&
                mbar_test_now(full_b + 8 * (pub % kSwStages), (pub / kSwStages) & 1)) {
                ++pub;
                count_publish(loaded_s, (uint32_t)pub);
                progress = true;
            }
            if (progress) {
                idle = 0;
            } else if (*abort_w) {
                break;
            } else {
                if (idle == 0) idle_t0 = sw_now();
                if (++idle >= kTcWaitLimit || sw_late(idle, idle_t0)) {
                    *abort_w = 1;
                    atomicOr(a.flag, kFlagTimeout);
                    break;
                }
                __nanosleep(64);  // nothing to issue or publish yet
            }
        }
        // every copy issued lands before the CTA ends (the last phase of each
        // stage is the one to wait for)
        const int used = si < kSwStages ? si : kSwStages;
        const unsigned long long t0 = sw_now();
        for (int st = 0; st < used; ++st) {
            const int j = si - 1 - ((si - 1 - st) % kSwStages);
            for (unsigned k = 0; k < kTcWaitLimit && !sw_late(k, t0) &&
                                 !mbar_test(full_b + 8 * st, (j / kSwStages) & 1);
                 ++k) {
            }
        }
        for (unsigned k = 0; k < kTcWaitLimit && !sw_late(k, t0) && !mbar_test(w_b, 0); ++k) {
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------------------------------------------------------- MMA issuer
        // A single thread: descriptors are formed once and offset per MMA (the
        // start-address field, in 16-byte units, is the low bits).
        griddep_wait();
        bool ok = sw_wait(w_b, 0, abort_w, a.flag);
        const uint64_t adesc0 = umma_smem_desc(stage_s, kSwHalfBytes, 128u);
        const uint64_t bdesc0 = umma_smem_desc(w_s, 16u * 3 * RW, 128u);
        const uint32_t idesc0 = umma_idesc_bf16(128, 0);
        SwStages in;
        in.begin(a, q0, q1);
        int kb = 0;       // ring index of the run's first plane
        int s_first = 0;  // its slot
        uint32_t known_loaded = 0, known_released = 0;
        for (int si = 0; si < n_stages && ok; ++si) {
            if (!sw_wait_count(loaded_s, (uint32_t)(si + 1), known_loaded, abort_w, a.flag)) {
                ok = false;
                break;
            }
            const int st = si % kSwStages;
            const int zs = in.zs, ze = in.ze;
            if (in.zi == zs - 1) s_first = kb % kSwRing;
#pragma unroll 1
            for (int pl = 0; pl < 2; ++pl) {
                const int zi = in.zi + pl;
                if (zi > ze) break;  // the padding plane of an odd run
                const int hi = zi + 1 < ze - 1 ? zi + 1 : ze - 1;
                const int lo = zi - 1 > zs ? zi - 1 : zs;
                const int khi = kb + hi - zs;
                if (zi + 1 < ze && khi >= kSwRing) {
                    // plane khi is first fed now: its slot was released with plane khi - R
                    if (!sw_wait_released(rel_s, (uint32_t)(khi - kSwRing + 1), known_released,
                                          abort_w, a.flag)) {
                        ok = false;
                        break;
                    }
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                int slot = s_first + (hi - zs);
                while (slot >= kSwRing) slot -= kSwRing;
                const uint64_t a_pl =
                    adesc0 + (uint64_t)((st * kSwStageBytes + pl * kSwPlaneBytes) >> 4);
                int dzi = zi - hi + 1;
                for (int left = hi - lo + 1; left > 0;) {
                    const int n = left < slot + 1 ? left : slot + 1;  // adjacent columns
                    const uint32_t d = tmem + (uint32_t)((kSwRing - 1 - slot) * C);
                    const uint32_t idesc = idesc0 + ((uint32_t)(n * C) >> 3 << 17);
                    const uint64_t b_run = bdesc0 + (uint64_t)(dzi * C);
#pragma unroll
                    for (int dyi = 0; dyi < 3; ++dyi)
                        umma_bf16(d, a_pl + (uint64_t)(16 * dyi), b_run + (uint64_t)(dyi * RW),
                                  idesc);
                    left -= n;
                    dzi += n;
                    slot = kSwRing - 1;
                }
                if (zi - 1 >= zs && !a.withhold) {  // plane zi - 1 has all its inputs
                    int s1 = s_first + (zi - 1 - zs);
                    while (s1 >= kSwRing) s1 -= kSwRing;
                    umma_commit(accf_b + 8 * s1);
                }
            }
            if (!ok) break;
            umma_commit(empty_b + 8 * st);  // the stage is read once these MMAs are done
            if (in.zi + 2 > ze) kb += ze - zs;  // the run's last stage
            in.next(a);
        }
        umma_commit(done_b);
        const unsigned long long t0 = sw_now();
        for (unsigned k = 0; k < kTcWaitLimit && !sw_late(k, t0) && !mbar_test(done_b, 0); ++k) {
        }
    } else if (warp >= 2) {
        // ---------------------------------------------------------------- epilogue
        griddep_wait();  // before the first store
        const int r = 32 * (warp & 3) + lane, bx = r & 15, by = r >> 4;
        int k = 0;
        bool ok = true;
        for (long long q = q0; q < q1 && ok;) {
            int x0, y0, zs, ze;
            sw_chunk(a, q, q1, x0, y0, zs, ze);
            const int X = x0 - 1 + bx, Y = y0 + by;
            const bool valid = bx >= 1 && bx <= kSwOX && X < a.mx && Y < a.my;
            for (int zo = zs; zo < ze; ++zo, ++k) {
                const int slot = k % kSwRing;
                int got = 1;
                if (lane == 0) got = sw_wait(accf_b + 8 * slot, (k / kSwRing) & 1, abort_w, a.flag);
                got = __shfl_sync(0xffffffffu, got, 0);
                if (!got) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t taddr = tmem + (uint32_t)((kSwRing - 1 - slot) * C) + lane_off;
                // this warp's columns: per dx block (second layer) its 8 channels
                float v[24];
                if (kL == 1) {
#pragma unroll
                    for (int b = 0; b < 3; ++b) tmem_ld8(taddr + 16 * b + 8 * eg, v + 8 * b);
                } else if (kL == 0 || eg == 0) {
                    tmem_ld8(taddr + (kL == 0 ? 8 * eg : 0), v);
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                sw_reset_slot<kL>(taddr, eg, binit);
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) count_release(rel_s + 4u * (warp - 2));
                const size_t gv = ((size_t)zo * a.my + Y) * a.mx + X;
                if (kL == 2) {
                    if (eg != 0) continue;
                    float o[2];
#pragma unroll
                    for (int c = 0; c < 2; ++c)
                        o[c] = __shfl_up_sync(0xffffffffu, v[c], 1) + v[2 + c] +
                               __shfl_down_sync(0xffffffffu, v[4 + c], 1);
                    if (valid) {
                        if (a.f_out)
                            *reinterpret_cast<float2*>(a.f_out + gv * kPC) = make_float2(o[0], o[1]);
                        if (a.y_out) {
                            const size_t V = (size_t)a.mx * a.my * a.mz;
                            a.y_out[gv] = o[0] * a.inv_scale;
                            a.y_out[V + gv] = o[1] * a.inv_scale;
                        }
                    }
                } else {
                    float o[8];
                    if (kL == 1) {
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            o[c] = __shfl_up_sync(0xffffffffu, v[c], 1) + v[8 + c] +
                                   __shfl_down_sync(0xffffffffu, v[16 + c], 1);
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) o[c] = v[c];
                    }
                    if (valid) {
                        if (a.z_out) {
                            float4* zo4 = reinterpret_cast<float4*>(a.z_out + gv * kPC + 8 * eg);
                            zo4[0] = make_float4(o[0], o[1], o[2], o[3]);
                            zo4[1] = make_float4(o[4], o[5], o[6], o[7]);
                        }
                        __nv_bfloat162 h[4];
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float u = o[2 * c], w = o[2 * c + 1];
                            h[c] = __floats2bfloat162_rn(__fdividef(u, 1.0f + __expf(-u)),
                                                         __fdividef(w, 1.0f + __expf(-w)));
                        }
                        sw_store_half(a.act_out, a, X, Y, zo, eg, *reinterpret_cast<uint4*>(h));
                    }
                }
            }
            q += ze - zs;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(sw_tmem_cols(kL))
                     : "memory");
    }
}

template <int kL>
void sweep_attr() {
    cudaFuncSetAttribute(k_conv_sweep<kL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sw_smem_bytes(kL));
}

void conv_sweep_setup() {
    static std::once_flag once[64];
    once_per_device(once, [] {
        sweep_attr<0>();
        sweep_attr<1>();
        sweep_attr<2>();
        cudaGetLastError();
    });
}

// The padded-activation geometry of a mesh: pitches PX, PY (at least one box).
void sweep_pitches(const PropGeom& g, int& px, int& py) {
    px = g.mx + 2 > kSwBX ? g.mx + 2 : kSwBX;
    py = g.my + 2 > kSwBY ? g.my + 2 : kSwBY;
}

// Tensor map of a padded activation buffer [2 halves][Mz + 2][PY][PX][8] with
// x and channel folded into one innermost dimension of 8 PX elements, so that
// a box row (16 voxels x 8 channels, 256 bytes) is one contiguous TMA row; the
// box is one channel half of the 16 x 10 voxel boxes of two planes.
bool make_act_tensor_map(CUtensorMap* map, __nv_bfloat16* act, const PropGeom& g) {
    int px, py;
    sweep_pitches(g, px, py);
    const cuuint64_t pz = (cuuint64_t)g.mz + 2;
    const cuuint64_t dims[4] = {8ull * px, (cuuint64_t)py, pz, 2};
    const cuuint64_t strides[3] = {16ull * px, 16ull * px * py, 16ull * px * py * pz};
    const cuuint32_t box[4] = {8 * kSwBX, (cuuint32_t)kSwBY, 2, 1};
    return encode_tiled_map(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, act, dims, strides, box);
}

template <int kL>
void launch_conv_sweep(const CUtensorMap& tmap, const SweepArgs& a, int ctas, cudaStream_t s) {
    conv_sweep_setup();
    const int grid = a.total < ctas ? a.total : ctas;
    // programmatic launch: the prologue overlaps the previous layer's tail;
    // every role waits for the previous grid before touching its output
    if (grid > 0) launch_pdl(k_conv_sweep<kL>, grid, kSwThreads, sw_smem_bytes(kL), s, tmap, a);
}

// Weight image of layer kL in the B layout of k_conv_sweep, kTcWCopies times:
// [half][dy index][row][8 channels], row = dz index C + column, column = co
// (first layer), dx index 16 + co (second), dx index 2 + co < 6 (last); from
// the forward weights wf [o][co][ci] (o = 9 dz index + 3 dy index + dx index)
// or, for the first layer, wx [3 dz index + dy index][co][K].
__global__ void k_pack_sweep_images(const __nv_bfloat16* __restrict__ wf,
                                    const __nv_bfloat16* __restrict__ wx, uint4* __restrict__ out) {
    const int L = blockIdx.x;
    const int C = sw_cols(L), RW = sw_rows(L), per = sw_image_words(L);
    const uint4* wf4 = reinterpret_cast<const uint4*>(wf + (size_t)L * kOffsets * kPC * kPC);
    const uint4* wx4 = reinterpret_cast<const uint4*>(wx);
    uint4* o = out + sw_image_offset(L);
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
        const int half = e / (3 * RW), dyi = (e / RW) % 3, row = e % RW;
        const int dzi = row / C, c = row % C;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (L == 0) {
            v = wx4[((dzi * 3 + dyi) * kPC + c) * 2 + half];
        } else if (L == 1) {
            const int dxi = c / 16, co = c % 16;
            v = wf4[((dzi * 9 + dyi * 3 + dxi) * kPC + co) * 2 + half];
        } else if (c < 6) {
            const int dxi = c / 2, co = c % 2;
            v = wf4[((dzi * 9 + dyi * 3 + dxi) * kPC + co) * 2 + half];
        }
        for (int k = 0; k < kTcWCopies; ++k) o[k * per + e] = v;
    }
}

// dW[o][ci][co] = sum_n in(n + d_o)[ci] gz(n)[co]: a voxel reduction on the
// tensor cores.  Warp w owns offsets w, w + 8, w + 16 (and 24 for w < 3); a
// CTA walks tiles grid-stride and writes its register sums to its own slice
// part[blockIdx.x] (every entry, once); k_sum_partials adds the slices in a
// fixed order, so the gradient is deterministic.
__global__ void __launch_bounds__(256) k_conv_wgrad(const __nv_bfloat16* __restrict__ in,
                                                    const __nv_bfloat16* __restrict__ gz,
                                                    float* __restrict__ part, PropGeom g,
                                                    ActLayout L) {
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
        load_box(in, g, L, x0, y0, z0, box);
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
//
// out_x: the same four channels as the x-im2col input of the first layer's
// tensor-core convolution, K index (dx + 1) * 4 + ci holding channel ci of
// voxel (x + dx, y, z) (periodic in x) for dx = -1, 0, 1, zeros from 12 on.
__device__ __forceinline__ void input_features(const float* __restrict__ x, int V, int v,
                                               float scale, float (&f)[4]) {
    const float a0 = x[v], b0 = x[(size_t)V + v];
    const float a1 = x[(size_t)2 * V + v], b1 = x[(size_t)3 * V + v];
    f[0] = scale * (a1 - a0);
    f[1] = scale * (b1 - b0);
    f[2] = a1;
    f[3] = b1;
}

// One thread per voxel of the padded array [Mz + 2][My + 2][Mx + 2] (grid y:
// the padded plane; halo
// included, each halo voxel a copy of the opposite face): out_x in the padded
// layout of the forward convolutions [2][Mz + 2][py][px][8]; out (optional, for the
// weight gradient): the plain four channels [V][16] at the interior voxels.
__global__ void k_pack_input(const float* __restrict__ x, PropGeom g, int px, int py, float scale,
                             __nv_bfloat16* __restrict__ out, __nv_bfloat16* __restrict__ out_x) {
    // the first convolution (a programmatic launch) may start its prologue now;
    // it waits for this grid before reading what it writes
    griddep_launch_dependents();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;  // voxel of the padded plane hz
    const int wx = g.mx + 2, wy = g.my + 2, wz = g.mz + 2;
    if (i >= wx * wy) return;
    const int hy = i / wx, hx = i - hy * wx, hz = blockIdx.y;
    const int xi = hx == 0 ? g.mx - 1 : (hx == g.mx + 1 ? 0 : hx - 1);
    const int yi = hy == 0 ? g.my - 1 : (hy == g.my + 1 ? 0 : hy - 1);
    const int z = hz == 0 ? g.mz - 1 : (hz == g.mz + 1 ? 0 : hz - 1);
    const int row = (z * g.my + yi) * g.mx;
    const int xm = xi == 0 ? g.mx - 1 : xi - 1, xp = xi == g.mx - 1 ? 0 : xi + 1;
    float f[3][4];
    input_features(x, g.V, row + xm, scale, f[0]);
    input_features(x, g.V, row + xi, scale, f[1]);
    input_features(x, g.V, row + xp, scale, f[2]);
    __nv_bfloat16 vals[kPC], cols[kPC];
#pragma unroll
    for (int c = 0; c < kPC; ++c) {
        vals[c] = __float2bfloat16_rn(c < 4 ? f[1][c] : 0.f);
        cols[c] = __float2bfloat16_rn(c < 12 ? f[c >> 2][c & 3] : 0.f);
    }
    uint4* ox = reinterpret_cast<uint4*>(out_x) + ((size_t)hz * py + hy) * px + hx;
    ox[0] = reinterpret_cast<uint4*>(cols)[0];
    ox[(size_t)wz * py * px] = reinterpret_cast<uint4*>(cols)[1];
    if (out && hx >= 1 && hx <= g.mx && hy >= 1 && hy <= g.my && hz >= 1 && hz <= g.mz) {
        uint4* o = reinterpret_cast<uint4*>(out + (size_t)(row + xi) * kPC);
        o[0] = reinterpret_cast<uint4*>(vals)[0];
        o[1] = reinterpret_cast<uint4*>(vals)[1];
    }
}

// One autoregressive step on the planar input x [4][V] = (phi(t - 1), phi(t))
// with the predicted change dphi [2][V]: x becomes (phi(t), phi(t) + dphi).
__global__ void k_rollout_shift(float* __restrict__ x, const float* __restrict__ dphi, int V) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const float cur = x[(size_t)(2 + c) * V + v];
        x[(size_t)c * V + v] = cur;
        x[(size_t)(2 + c) * V + v] = cur + dphi[(size_t)c * V + v];
    }
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
// wx: the first layer's weights for its x-im2col input, [dz_index * 3 + dy_index]
// [co][K = (dx + 1) * 4 + ci], zeros from K = 12 on.
__global__ void k_pack_weights(const float* __restrict__ params, __nv_bfloat16* __restrict__ wf,
                               __nv_bfloat16* __restrict__ wb, float* __restrict__ bias,
                               __nv_bfloat16* __restrict__ wx) {
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
    if (layer == 0) {
        for (int e = threadIdx.x; e < 9 * kPC * kPC; e += blockDim.x) {
            const int o = e / (kPC * kPC), co = (e / kPC) % kPC, k = e % kPC;
            const int dzi = o / 3, dyi = o % 3, dxi = k >> 2, ci = k & 3;
            const float v = k < 12 ? Wl[((dzi * 9 + dyi * 3 + dxi) * ci_n + ci) * co_n + co] : 0.f;
            wx[e] = __float2bfloat16_rn(v);
        }
    }
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

// One pass of the periodic binomial filter (1/4, 1/2, 1/4) along one axis of
// C channels of an FP32 [C][Mz][My][Mx] mesh: out(n) = (in(n - e) + 2 in(n) +
// in(n + e)) / 4 with the neighbours e along the axis (periodic).
__global__ void k_binomial_pass(const float* __restrict__ in, float* __restrict__ out, int mx,
                                int my, int mz, int C, int axis) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)C * mx * my * mz;
    if (i >= n) return;
    const int x = (int)(i % mx), y = (int)((i / mx) % my), z = (int)((i / ((long long)mx * my)) % mz);
    long long lo, hi;
    if (axis == 0) {
        lo = i - x + (x == 0 ? mx - 1 : x - 1);
        hi = i - x + (x == mx - 1 ? 0 : x + 1);
    } else if (axis == 1) {
        const long long r = (long long)mx;
        lo = i + (long long)((y == 0 ? my - 1 : y - 1) - y) * r;
        hi = i + (long long)((y == my - 1 ? 0 : y + 1) - y) * r;
    } else {
        const long long r = (long long)mx * my;
        lo = i + (long long)((z == 0 ? mz - 1 : z - 1) - z) * r;
        hi = i + (long long)((z == mz - 1 ? 0 : z + 1) - z) * r;
    }
    out[i] = 0.25f * (in[lo] + in[hi]) + 0.5f * in[i];
}

// passes x 3 axes of the binomial filter from in to out, ping-ponging between
// out and tmp (same size, distinct from out) so that the last pass writes out;
// in may equal out.
void launch_smooth_phi(const float* in, float* out, float* tmp, int mx, int my, int mz, int C,
                       int passes, cudaStream_t s) {
    const long long n = (long long)C * mx * my * mz;
    if (n <= 0) return;
    const unsigned blocks = (unsigned)((n + 255) / 256);
    const int total = 3 * (passes > 0 ? passes : 0);
    if (total == 0) {
        if (in != out) cudaMemcpyAsync(out, in, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
        return;
    }
    const float* src = in;
    for (int k = 0; k < total; ++k) {
        float* dst = ((total - 1 - k) % 2 == 0) ? out : tmp;
        if (dst == src) {  // only at the first pass, when in is the target buffer
            float* other = dst == out ? tmp : out;
            cudaMemcpyAsync(other, src, sizeof(float) * n, cudaMemcpyDeviceToDevice, s);
            src = other;
        }
        k_binomial_pass<<<blocks, 256, 0, s>>>(src, dst, mx, my, mz, C, k % 3);
        src = dst;
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
    // act[0]: the plain input [V][16] (training only); act[1], act[2]: the
    // hidden activations in the padded layout [2][Mz + 2][py][px][8]; act[3]:
    // a gradient buffer [V][16]
    __nv_bfloat16* act[4] = {};
    __nv_bfloat16* act_x = nullptr;  // the input as x-im2col, padded layout
    __nv_bfloat16* wx = nullptr;     // first-layer weights for it [9][16][16]
    uint4* tcw = nullptr;            // packed weight images of the data-gradient convolutions
    uint4* sww = nullptr;            // packed weight images of the forward convolutions
    CUtensorMap tmap[3];             // act_x, act[1], act[2]
    int px = 0, py = 0;              // padded pitches
    int ctas = 1;                    // CTAs of the persistent convolutions (kSwPerSM per SM)
    float* z[2] = {};             // pre-activations of layers 1, 2 [V][16]
    float* fbuf = nullptr;        // FP32 [V][16]: output / data gradient
    float* xin = nullptr;         // staging of the planar input [4][V]
    float* tin = nullptr;         // staging of the planar next densities [2][V]
    float* yout = nullptr;        // planar output [2][V]
    double* loss = nullptr;
    double* h_loss = nullptr;
    int* flag = nullptr;          // device status bits of the tensor-core waits
    int* h_flag = nullptr;        // pinned mirror
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

// The padded BF16 weights, biases and the tensor-core weight images from the
// FP32 parameters.
void pack_all_weights(hpf_prop* p, cudaStream_t s) {
    const size_t wl = (size_t)kOffsets * kPC * kPC;
    k_pack_weights<<<3, 256, 0, s>>>(p->params, p->wf, p->wb, p->bias, p->wx);
    k_pack_sweep_images<<<3, 256, 0, s>>>(p->wf, p->wx, p->sww);
    k_pack_tc_image<<<1, 256, 0, s>>>(p->wb + wl, 0, p->tcw);
    k_pack_tc_image<<<1, 256, 0, s>>>(p->wb + 2 * wl, 1, p->tcw);
}

SweepArgs sweep_args(const hpf_prop* p, int layer, int* flag) {
    SweepArgs a{};
    a.w = p->sww + sw_image_offset(layer);
    a.bias = p->bias + layer * kPC;
    a.inv_scale = 1.0f / p->scale;
    a.flag = flag;
    a.mx = p->g.mx;
    a.my = p->g.my;
    a.mz = p->g.mz;
    a.px = p->px;
    a.py = p->py;
    a.ncx = (p->g.mx + kSwOX - 1) / kSwOX;
    a.total = a.ncx * ((p->g.my + kSwY - 1) / kSwY) * p->g.mz;
    return a;
}

// Forward pass of planar input x [4][V] (device).  keep_z: the pre-activations
// and the plain input are stored and the FP32 output goes to fbuf [V][16] for
// a backward pass; y_planar (optional): the predicted change [2][V] (the
// output divided by scale).
void prop_forward(hpf_prop* p, const float* x, bool keep_z, cudaStream_t s, int* flag,
                  float* y_planar = nullptr) {
    const int hp = (p->g.mx + 2) * (p->g.my + 2);  // padded voxels per plane
    k_pack_input<<<dim3((unsigned)((hp + 255) / 256), (unsigned)(p->g.mz + 2)), 256, 0, s>>>(
        x, p->g, p->px, p->py, p->scale, keep_z ? p->act[0] : nullptr, p->act_x);
    SweepArgs a = sweep_args(p, 0, flag);
    a.z_out = keep_z ? p->z[0] : nullptr;
    a.act_out = p->act[1];
    launch_conv_sweep<0>(p->tmap[0], a, p->ctas, s);
    a = sweep_args(p, 1, flag);
    a.z_out = keep_z ? p->z[1] : nullptr;
    a.act_out = p->act[2];
    launch_conv_sweep<1>(p->tmap[1], a, p->ctas, s);
    a = sweep_args(p, 2, flag);
    a.f_out = keep_z ? p->fbuf : nullptr;
    a.y_out = y_planar;
    launch_conv_sweep<2>(p->tmap[2], a, p->ctas, s);
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
        const ActLayout lay =
            layer == 0 ? ActLayout{p->g.mx, p->g.my, 0, kPC, 8}
                       : ActLayout{p->px, p->py, 1, 8, 8ll * (p->g.mz + 2) * p->py * p->px};
        k_conv_wgrad<<<p->grid_wgrad, 256, 0, s>>>(p->act[layer], gbuf, p->wpart, p->g, lay);
        k_sum_partials<float><<<(unsigned)((wl + 255) / 256), 256, 0, s>>>(
            p->wpart, p->grid_wgrad, (int)wl, p->dW + layer * wl);
        k_bias_grad<<<kBiasBlocks, 256, 0, s>>>(gbuf, V, p->bpart);
        k_sum_partials<float><<<1, 32, 0, s>>>(p->bpart, kBiasBlocks, kPC, p->db + layer * kPC);
        if (layer == 0) break;
        // the data gradient of the layer input, then through the SiLU below it
        launch_conv_tc(gbuf, p->tcw, layer - 1, p->fbuf, p->g, p->flag, s);
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
    pack_all_weights(p, p->stream);
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

// The loss of the last backward pass (synchronises), with the status of the
// tensor-core waits: HPF_ERR_TIMEOUT once if a wait gave up.
hpf_status prop_read_loss(hpf_prop* p, double* loss) {
    if (!loss) return HPF_OK;
    if (cudaMemcpyAsync(p->h_loss, p->loss, sizeof(double), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaMemcpyAsync(p->h_flag, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    *loss = *p->h_loss;
    if (*p->h_flag & kFlagTimeout) {
        cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream);
        return HPF_ERR_TIMEOUT;
    }
    return HPF_OK;
}

// A device (or managed) array of the current device.
bool prop_on_device(const void* ptr) {
    cudaPointerAttributes a;
    int dev = -1;
    const bool ok = cudaPointerGetAttributes(&a, ptr) == cudaSuccess && cudaGetDevice(&dev) == cudaSuccess &&
                    (a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev));
    cudaGetLastError();
    return ok;
}

hpf_status prop_launched(hpf_prop* p) {
    (void)p;
    return cudaGetLastError() == cudaSuccess ? HPF_OK : HPF_ERR_CUDA;
}

// Status of the tensor-core waits of the work enqueued so far (synchronises):
// HPF_ERR_TIMEOUT once if a wait gave up.
hpf_status prop_flag_status(hpf_prop* p) {
    if (cudaMemcpyAsync(p->h_flag, p->flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    if (*p->h_flag & kFlagTimeout) {
        cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream);
        return HPF_ERR_TIMEOUT;
    }
    return HPF_OK;
}

}  // namespace

namespace hpf {

bool prop_mesh_is(const hpf_prop* p, const MeshGeom& g) {
    return p && p->g.mx == g.mx && p->g.my == g.my && p->g.mz == g.mz;
}

void prop_predict(hpf_prop* p, const float* x, float* dphi, cudaStream_t s, int* flag) {
    prop_forward(p, x, false, s, flag ? flag : p->flag, dphi);
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
    p->ctas = kSwPerSM * sms;
    sweep_pitches(g, p->px, p->py);
    const size_t Vp = (size_t)(g.mz + 2) * p->py * p->px;  // padded voxels
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
    for (int k = 0; k < 4; ++k)
        e = e ? e : cudaMalloc(&p->act[k], sizeof(__nv_bfloat16) * (k == 1 || k == 2 ? Vp : Vs) * kPC);
    for (int k = 0; k < 2; ++k) e = e ? e : cudaMalloc(&p->z[k], sizeof(float) * Vs * kPC);
    e = e ? e : cudaMalloc(&p->fbuf, sizeof(float) * Vs * kPC);
    e = e ? e : cudaMalloc(&p->xin, sizeof(float) * Vs * 4);
    e = e ? e : cudaMalloc(&p->tin, sizeof(float) * Vs * 2);
    e = e ? e : cudaMalloc(&p->yout, sizeof(float) * Vs * 2);
    e = e ? e : cudaMalloc(&p->loss, sizeof(double));
    e = e ? e : cudaMallocHost(&p->h_loss, sizeof(double));
    e = e ? e : cudaMalloc(&p->flag, sizeof(int));
    e = e ? e : cudaMalloc(&p->act_x, sizeof(__nv_bfloat16) * Vp * kPC);
    e = e ? e : cudaMalloc(&p->sww, sizeof(uint4) * sw_image_offset(3));
    e = e ? e : cudaMalloc(&p->wx, sizeof(__nv_bfloat16) * 9 * kPC * kPC);
    e = e ? e : cudaMalloc(&p->tcw, sizeof(uint4) * tc_image_offset(kTcImages));
    e = e ? e : cudaMallocHost(&p->h_flag, sizeof(int));
    if (e == cudaSuccess) {
        // padded buffers: the pitch beyond the halo (meshes narrower than a box)
        // is read by the box copies and stays zero
        cudaMemsetAsync(p->act_x, 0, sizeof(__nv_bfloat16) * Vp * kPC, p->stream);
        cudaMemsetAsync(p->act[1], 0, sizeof(__nv_bfloat16) * Vp * kPC, p->stream);
        cudaMemsetAsync(p->act[2], 0, sizeof(__nv_bfloat16) * Vp * kPC, p->stream);
        if (!make_act_tensor_map(&p->tmap[0], p->act_x, g) ||
            !make_act_tensor_map(&p->tmap[1], p->act[1], g) ||
            !make_act_tensor_map(&p->tmap[2], p->act[2], g))
            e = cudaErrorNotSupported;
    }
    if (e == cudaSuccess) {
        cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream);
        // zero weights until hpf_prop_set_weights: the network predicts no change
        cudaMemsetAsync(p->params, 0, sizeof(float) * p->np, p->stream);
        cudaMemsetAsync(p->adam_m, 0, sizeof(float) * p->np, p->stream);
        cudaMemsetAsync(p->adam_v, 0, sizeof(float) * p->np, p->stream);
        pack_all_weights(p, p->stream);
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
    cudaFree(p->flag);
    cudaFreeHost(p->h_flag);
    cudaFree(p->act_x);
    cudaFree(p->wx);
    cudaFree(p->tcw);
    cudaFree(p->sww);
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
    pack_all_weights(p, p->stream);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess)
        return HPF_ERR_CUDA;
    return HPF_OK;
}

hpf_status hpf_prop_get_weights(hpf_prop* p, float* params) {
    if (!p || !params) return HPF_ERR_INVALID;
    return prop_copy_out(p, params, p->params, sizeof(float) * p->np);
}

hpf_status hpf_prop_selftest_timeout(hpf_prop* p, double* seconds) {
    if (!p) return HPF_ERR_INVALID;
    if (cudaStreamSynchronize(p->stream) != cudaSuccess ||
        cudaMemsetAsync(p->flag, 0, sizeof(int), p->stream) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    // the first layer on the handle's current input, its finished planes never
    // signalled: every CTA's epilogue waits run out, the CTAs abort and release
    // their tensor memory
    SweepArgs a = sweep_args(p, 0, p->flag);
    a.act_out = p->act[1];
    a.withhold = 1;
    const auto t0 = std::chrono::steady_clock::now();
    launch_conv_sweep<0>(p->tmap[0], a, p->ctas, p->stream);
    hpf_status st = prop_launched(p);
    if (st == HPF_OK) st = prop_flag_status(p);  // synchronises; clears the flag it reports
    if (seconds)
        *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return st;
}

hpf_status hpf_prop_set_ctas(hpf_prop* p, int32_t ctas) {
    if (!p || ctas < 0) return HPF_ERR_INVALID;
    if (ctas == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaGetLastError();
        ctas = kSwPerSM * (sms > 0 ? sms : 1);
    }
    p->ctas = ctas;
    return HPF_OK;
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
    if (!p || !dphi || !x) return HPF_ERR_INVALID;
    // device arrays of the current device are read and written in place (the
    // input is consumed by the first kernel, so x may even alias dphi); host
    // arrays go through the handle's staging buffers
    const bool dev_in = prop_on_device(x), dev_out = prop_on_device(dphi);
    hpf_status s = HPF_OK;
    if (!dev_in && (s = prop_stage(p, p->xin, x, (size_t)p->g.V * 4)) != HPF_OK) return s;
    prop_predict(p, dev_in ? x : p->xin, dev_out ? dphi : p->yout, p->stream, p->flag);
    if ((s = prop_launched(p)) != HPF_OK) return s;
    if (dev_out) return HPF_OK;  // the wait status comes with the next synchronising call
    if ((s = prop_copy_out(p, dphi, p->yout, sizeof(float) * 2 * p->g.V)) != HPF_OK) return s;
    return prop_flag_status(p);  // the host copy has synchronised: the status is known
}

hpf_status hpf_prop_rollout(hpf_prop* p, const float* x, int32_t steps, float* phi_out) {
    if (!p || !phi_out || steps < 1) return HPF_ERR_INVALID;
    const int V = p->g.V;
    hpf_status s = prop_stage(p, p->xin, x, (size_t)V * 4);
    if (s != HPF_OK) return s;
    for (int k = 0; k < steps; ++k) {
        prop_predict(p, p->xin, p->yout, p->stream, p->flag);
        k_rollout_shift<<<(V + 255) / 256, 256, 0, p->stream>>>(p->xin, p->yout, V);
    }
    if ((s = prop_launched(p)) != HPF_OK) return s;
    if ((s = prop_copy_out(p, phi_out, p->xin + 2 * (size_t)V, sizeof(float) * 2 * V)) != HPF_OK)
        return s;
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, phi_out) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev ? HPF_OK : prop_flag_status(p);
}

hpf_status hpf_prop_backward(hpf_prop* p, const float* x, const float* phi_next, float* grads,
                             double* loss) {
    if (!p) return HPF_ERR_INVALID;
    hpf_status s = prop_stage(p, p->xin, x, (size_t)p->g.V * 4);
    if (s == HPF_OK) s = prop_stage(p, p->tin, phi_next, (size_t)p->g.V * 2);
    if (s != HPF_OK) return s;
    prop_forward(p, p->xin, true, p->stream, p->flag);
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
    prop_forward(p, p->xin, true, p->stream, p->flag);
    prop_backward(p, p->xin, p->tin);
    prop_adam(p, p->grads, lr);
    if ((s = prop_launched(p)) != HPF_OK) return s;
    return prop_read_loss(p, loss);
}

}  // extern "C"
