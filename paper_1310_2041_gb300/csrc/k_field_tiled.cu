// k_field_tiled.cu -- the field stencil (V_K and periodic central-difference
// grad V_K, MD-SCF section; Algorithm 1, kernel 3) on shared-memory tiles.
//
// A CTA computes a TX x TY x TZ tile of the ghosted field array.  It needs the
// density of the tile plus one node on every side (x: two, so the copy starts
// on a 16-byte boundary): a (TX+4) x (TY+2) x (TZ+2) box per species, staged
// in shared memory by one TMA tensor copy (cp.async.bulk.tensor, completion on
// an mbarrier) when the mesh allows it (x extent even: rows are multiples of
// 16 bytes), else by plain loads.  TMA has no periodic mode: box elements
// outside the mesh arrive as zeros and are then replaced by their periodic
// images with plain loads (only tiles on the mesh boundary have any).  The
// tile shape is chosen per mesh by timing the candidates (hpf_api.cu).
#include <cuda.h>

#include "hpf_internal.cuh"

namespace hpf {

// Candidate tiles (x, y, z): a CTA has x * y threads, each computing z nodes
// along a z column.  Shape {0, 0, 0} is the untiled one-node-per-thread stencil
// with direct L1/L2 loads, so the autotuner can never pick a slower kernel.
// Shape {2, 1, 1} is the untiled two-nodes-per-thread stencil (16-byte pair
// loads, ghost copies written directly).
constexpr int kTileCandidates = 8;
constexpr int kTileShapes[kTileCandidates][3] = {
    {32, 8, 4}, {32, 8, 8}, {16, 16, 4}, {64, 4, 4}, {16, 16, 8}, {32, 4, 8}, {0, 0, 0},
    {2, 1, 1}};
constexpr int kPairTile = 7;
constexpr unsigned kWaitLimit = 1u << 22;          // polls of an mbarrier before giving up
constexpr unsigned long long kWaitNs = 200000000ull;  // or 0.2 s, whichever comes first

int field_tile_candidates() { return kTileCandidates; }

void field_tile_shape(int id, int out[3]) {
    for (int a = 0; a < 3; ++a) out[a] = kTileShapes[id][a];
}

size_t field_tile_smem(int id, int S) {
    const int* t = kTileShapes[id];
    if (t[0] == 0 || id == kPairTile) return 0;
    return sizeof(long long) * (size_t)(t[0] + 4) * (t[1] + 2) * (t[2] + 2) * S;
}

bool field_tile_is_plain(int id) { return kTileShapes[id][0] == 0 || id == kPairTile; }

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false if the barrier did not complete within kWaitLimit polls or
// kWaitNs nanoseconds (a tensor copy completes within microseconds).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    for (unsigned it = 0; it < kWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 63) == 63 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

// Self-test of the bounded wait: an mbarrier nothing ever arrives on (no
// copy is issued), so the wait must give up, raise the timeout flag and
// return.
__global__ void k_wait_selftest(int* flag) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = smem_u32(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !mbar_wait(b, 0)) atomicOr(flag, kFlagTimeout);
}

// Periodic image of an index that is at most one period outside [0, m) (the
// general remainder only for meshes smaller than a box).
__device__ __forceinline__ int wrap_near(int i, int m) {
    if (i < 0) i += m;
    else if (i >= m) i -= m;
    if (i < 0 || i >= m) i = ((i % m) + m) % m;
    return i;
}

// Replica of block b: the last record with blk_begin <= b.
template <int kCap>
__device__ __forceinline__ int field_replica(const TiledFieldParamsT<kCap>& p) {
    if (kCap == 1) return 0;
    int lo = 0, hi = p.R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.rep[mid].blk_begin <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int S, int TX, int TY, int TZ, int kCap>
__global__ void __launch_bounds__(TX * TY) k_field_tiled(const __grid_constant__ TiledFieldParamsT<kCap> p) {
    griddep_wait();
    griddep_launch_dependents();
    constexpr int BX = TX + 4, BY = TY + 2, BZ = TZ + 2;
    constexpr int BOX = BX * BY * BZ;
    constexpr int NT = TX * TY;
    extern __shared__ __align__(128) long long box[];  // [S][BZ][BY][BX]
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int s_ok;

    const int lo = field_replica(p);  // replica of this block
    const TiledFieldRep& r = p.rep[lo];
    const MeshGeom& g = r.g;
    const int t = (int)blockIdx.x - r.blk_begin;
    const int x0 = (t % r.tiles_x) * TX;
    const int y0 = ((t / r.tiles_x) % r.tiles_y) * TY;
    const int z0 = (t / (r.tiles_x * r.tiles_y)) * TZ;
    const int ux = x0 - 2, vy = y0 - 1, wz = z0 - 1;  // box origin (unwrapped node indices)
    const bool interior = ux >= 0 && ux + BX <= g.mx && vy >= 0 && vy + BY <= g.my && wz >= 0 &&
                          wz + BZ <= g.mz;
    const int tid = threadIdx.x;

    if (r.use_tma) {
        const uint32_t b = smem_u32(&bar);
        if (tid == 0) {
            s_ok = 1;
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)(sizeof(long long) * BOX * S);
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b),
                         "r"(bytes)
                         : "memory");
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(box)),
                "l"(reinterpret_cast<uint64_t>(&r.tmap)), "r"(ux), "r"(vy), "r"(wz), "r"(0),
                "r"(b)
                : "memory");
        }
        if (!mbar_wait(b, 0)) {
            // give up on this tile: report, then wait (bounded) for the copy in flight
            atomicOr(p.flag, kFlagTimeout);
            s_ok = 0;
            mbar_wait(b, 0);
        }
        __syncthreads();
        if (!s_ok) return;
    }
    if (!r.use_tma || !interior) {
        // plain loads: every element, or only those the copy filled with zeros
        for (int e = tid; e < S * BOX; e += NT) {
            const int u = e % BX, v = (e / BX) % BY, w = (e / (BX * BY)) % BZ, k = e / BOX;
            int gx = ux + u, gy = vy + v, gz = wz + w;
            const bool inside = gx >= 0 && gx < g.mx && gy >= 0 && gy < g.my && gz >= 0 &&
                                gz < g.mz;
            if (r.use_tma && inside) continue;
            gx = wrap_near(gx, g.mx);
            gy = wrap_near(gy, g.my);
            gz = wrap_near(gz, g.mz);
            box[e] = __ldg(r.D + (size_t)k * g.nodes + ((size_t)gz * g.my + gy) * g.mx + gx);
        }
    }
    __syncthreads();

    const int tx = tid % TX, ty = tid / TX;
    const int px = x0 + tx, py = y0 + ty;
    if (px > g.mx || py > g.my) return;
    const FieldCoef& c = *r.coef;
    const int u = tx + 2, v = ty + 1;
#pragma unroll 1
    for (int tz = 0; tz < TZ; ++tz) {
        const int pz = z0 + tz;
        if (pz > g.mz) break;
        if (r.D_clear && px < g.mx && py < g.my && pz < g.mz) {
            const size_t node = ((size_t)pz * g.my + py) * g.mx + px;
#pragma unroll
            for (int k = 0; k < S; ++k) r.D_clear[(size_t)k * g.nodes + node] = 0ull;
        }
        const int w = tz + 1;
        float ddx[S], ddy[S], ddz[S], dc[S];
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const long long* bk = box + k * BOX;
            const int o = (w * BY + v) * BX + u;
            ddx[k] = (float)(bk[o + 1] - bk[o - 1]);
            ddy[k] = (float)(bk[o + BX] - bk[o - BX]);
            ddz[k] = (float)(bk[o + BX * BY] - bk[o - BX * BY]);
            dc[k] = (float)bk[o];
        }
        const size_t pnode = (size_t)pz * g.gxy + (size_t)py * g.gx + px;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            float gx = 0.f, gy = 0.f, gz = 0.f, vv = c.v0;
#pragma unroll
            for (int kp = 0; kp < S; ++kp) {
                gx = fmaf(c.gx[k][kp], ddx[kp], gx);
                gy = fmaf(c.gy[k][kp], ddy[kp], gy);
                gz = fmaf(c.gz[k][kp], ddz[kp], gz);
                vv = fmaf(c.v[k][kp], dc[kp], vv);
            }
            r.G[(size_t)k * g.gnodes + pnode] = make_float4(gx, gy, gz, vv);
        }
    }
}

// The untiled candidate: one thread per node of the ghosted array, neighbours
// loaded directly (through L1/L2), same arithmetic as the tiled kernel.
template <int S, int kCap>
__global__ void __launch_bounds__(256) k_field_plain(const __grid_constant__ TiledFieldParamsT<kCap> p) {
    griddep_wait();
    griddep_launch_dependents();
    const int lo = field_replica(p);
    const TiledFieldRep& r = p.rep[lo];
    const MeshGeom& g = r.g;
    const int pnode = ((int)blockIdx.x - r.blk_begin) * 256 + threadIdx.x;
    if (pnode >= g.gnodes) return;
    const int px = pnode % g.gx, py = (pnode / g.gx) % (g.my + 1), pz = pnode / g.gxy;
    const int x = px == g.mx ? 0 : px, y = py == g.my ? 0 : py, z = pz == g.mz ? 0 : pz;
    const int node = (z * g.my + y) * g.mx + x;
    if (r.D_clear && px < g.mx && py < g.my && pz < g.mz) {
#pragma unroll
        for (int k = 0; k < S; ++k) r.D_clear[(size_t)k * g.nodes + node] = 0ull;
    }
    const int xp = node + ((x + 1 == g.mx) ? 1 - g.mx : 1);
    const int xm = node + ((x == 0) ? g.mx - 1 : -1);
    const int sy = g.mx, sz = g.mx * g.my;
    const int yp = node + ((y + 1 == g.my) ? (1 - g.my) * sy : sy);
    const int ym = node + ((y == 0) ? (g.my - 1) * sy : -sy);
    const int zp = node + ((z + 1 == g.mz) ? (1 - g.mz) * sz : sz);
    const int zm = node + ((z == 0) ? (g.mz - 1) * sz : -sz);
    const FieldCoef& c = *r.coef;
    float ddx[S], ddy[S], ddz[S], dc[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const long long* Dk = r.D + (size_t)k * g.nodes;
        ddx[k] = (float)(__ldg(Dk + xp) - __ldg(Dk + xm));
        ddy[k] = (float)(__ldg(Dk + yp) - __ldg(Dk + ym));
        ddz[k] = (float)(__ldg(Dk + zp) - __ldg(Dk + zm));
        dc[k] = (float)__ldg(Dk + node);
    }
#pragma unroll
    for (int k = 0; k < S; ++k) {
        float gx = 0.f, gy = 0.f, gz = 0.f, vv = c.v0;
#pragma unroll
        for (int kp = 0; kp < S; ++kp) {
            gx = fmaf(c.gx[k][kp], ddx[kp], gx);
            gy = fmaf(c.gy[k][kp], ddy[kp], gy);
            gz = fmaf(c.gz[k][kp], ddz[kp], gz);
            vv = fmaf(c.v[k][kp], dc[kp], vv);
        }
        r.G[(size_t)k * g.gnodes + pnode] = make_float4(gx, gy, gz, vv);
    }
}

// Two x-adjacent real nodes (x, x + 1) per thread.  With an even x extent
// every pair starts on a 16-byte boundary and the centre, y +- 1 and z +- 1
// rows are read as int64 pairs (7 loads per species for two nodes); an odd
// extent uses scalar loads and a last pair of one node.  Each node writes its
// ghost copies itself (x = 0 also at x = Mx, and so on), so no ghosted-index
// arithmetic is needed.  Same arithmetic as the other candidates.
template <int S, int kCap>
__global__ void __launch_bounds__(256) k_field_pair(const __grid_constant__ TiledFieldParamsT<kCap> p) {
    griddep_wait();
    griddep_launch_dependents();
    const int lo = field_replica(p);
    const TiledFieldRep& r = p.rep[lo];
    const MeshGeom& g = r.g;
    const int hx = (g.mx + 1) >> 1;  // pairs per row
    const int t = ((int)blockIdx.x - r.blk_begin) * 256 + threadIdx.x;
    if (t >= hx * g.my * g.mz) return;
    const int x = 2 * (t % hx), y = (t / hx) % g.my, z = t / (hx * g.my);
    const bool two = x + 1 < g.mx;
    const int row = (z * g.my + y) * g.mx;
    const int ym = y == 0 ? g.my - 1 : y - 1, yp = y + 1 == g.my ? 0 : y + 1;
    const int zm = z == 0 ? g.mz - 1 : z - 1, zp = z + 1 == g.mz ? 0 : z + 1;
    const int rym = (z * g.my + ym) * g.mx, ryp = (z * g.my + yp) * g.mx;
    const int rzm = (zm * g.my + y) * g.mx, rzp = (zp * g.my + y) * g.mx;
    const int xl = x == 0 ? g.mx - 1 : x - 1;
    const int x1 = two ? x + 1 : x;  // the second node (a repeat of the first if absent)
    const int xr = x1 + 1 == g.mx ? 0 : x1 + 1;
    const bool vec = (g.mx & 1) == 0;
    float ddx[2][S], ddy[2][S], ddz[2][S], dc[2][S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const long long* Dk = r.D + (size_t)k * g.nodes;
        long long c0, c1, a0, a1, b0, b1, e0, e1, f0, f1;
        if (vec) {
            const longlong2 c = __ldg(reinterpret_cast<const longlong2*>(Dk + row + x));
            const longlong2 a = __ldg(reinterpret_cast<const longlong2*>(Dk + rym + x));
            const longlong2 b = __ldg(reinterpret_cast<const longlong2*>(Dk + ryp + x));
            const longlong2 e = __ldg(reinterpret_cast<const longlong2*>(Dk + rzm + x));
            const longlong2 f = __ldg(reinterpret_cast<const longlong2*>(Dk + rzp + x));
            c0 = c.x; c1 = c.y; a0 = a.x; a1 = a.y; b0 = b.x; b1 = b.y;
            e0 = e.x; e1 = e.y; f0 = f.x; f1 = f.y;
        } else {
            c0 = __ldg(Dk + row + x); c1 = __ldg(Dk + row + x1);
            a0 = __ldg(Dk + rym + x); a1 = __ldg(Dk + rym + x1);
            b0 = __ldg(Dk + ryp + x); b1 = __ldg(Dk + ryp + x1);
            e0 = __ldg(Dk + rzm + x); e1 = __ldg(Dk + rzm + x1);
            f0 = __ldg(Dk + rzp + x); f1 = __ldg(Dk + rzp + x1);
        }
        const long long l = __ldg(Dk + row + xl), rr = __ldg(Dk + row + xr);
        ddx[0][k] = (float)((two ? c1 : rr) - l);  // a lone node's right neighbour wraps
        ddy[0][k] = (float)(b0 - a0);
        ddz[0][k] = (float)(f0 - e0);
        dc[0][k] = (float)c0;
        ddx[1][k] = (float)(rr - c0);
        ddy[1][k] = (float)(b1 - a1);
        ddz[1][k] = (float)(f1 - e1);
        dc[1][k] = (float)c1;
        if (r.D_clear) {
            r.D_clear[(size_t)k * g.nodes + row + x] = 0ull;
            if (two) r.D_clear[(size_t)k * g.nodes + row + x1] = 0ull;
        }
    }
    const FieldCoef& c = *r.coef;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        if (j == 1 && !two) break;
        const int xx = x + j;
        // the node and its periodic ghost copies
        const int nxs = (xx == 0) ? 2 : 1, nys = (y == 0) ? 2 : 1, nzs = (z == 0) ? 2 : 1;
#pragma unroll
        for (int k = 0; k < S; ++k) {
            float gx = 0.f, gy = 0.f, gz = 0.f, vv = c.v0;
#pragma unroll
            for (int kp = 0; kp < S; ++kp) {
                gx = fmaf(c.gx[k][kp], ddx[j][kp], gx);
                gy = fmaf(c.gy[k][kp], ddy[j][kp], gy);
                gz = fmaf(c.gz[k][kp], ddz[j][kp], gz);
                vv = fmaf(c.v[k][kp], dc[j][kp], vv);
            }
            const float4 out = make_float4(gx, gy, gz, vv);
            float4* Gk = r.G + (size_t)k * g.gnodes;
            for (int iz = 0; iz < nzs; ++iz)
                for (int iy = 0; iy < nys; ++iy)
                    for (int ix = 0; ix < nxs; ++ix) {
                        const int px = ix ? g.mx : xx, py = iy ? g.my : y, pz = iz ? g.mz : z;
                        Gk[(size_t)pz * g.gxy + (size_t)py * g.gx + px] = out;
                    }
        }
    }
}

template <int S, int TX, int TY, int TZ, int kCap>
static void launch_tile(const TiledFieldParamsT<kCap>& p, cudaStream_t s) {
    const size_t smem = sizeof(long long) * (size_t)(TX + 4) * (TY + 2) * (TZ + 2) * S;
    static std::once_flag attr[64];
    once_per_device(attr, [smem] {
        cudaFuncSetAttribute(k_field_tiled<S, TX, TY, TZ, kCap>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (kCap == 1) launch_pdl(k_field_tiled<S, TX, TY, TZ, kCap>, p.blocks, TX * TY, smem, s, p);
    else k_field_tiled<S, TX, TY, TZ, kCap><<<p.blocks, TX * TY, smem, s>>>(p);
}

template <int S, int kCap>
static void launch_for_species(const TiledFieldParamsT<kCap>& p, int tile, cudaStream_t s) {
    switch (tile) {
        case 0: launch_tile<S, 32, 8, 4>(p, s); break;
        case 1: launch_tile<S, 32, 8, 8>(p, s); break;
        case 2: launch_tile<S, 16, 16, 4>(p, s); break;
        case 3: launch_tile<S, 64, 4, 4>(p, s); break;
        case 4: launch_tile<S, 16, 16, 8>(p, s); break;
        case 5: launch_tile<S, 32, 4, 8>(p, s); break;
        case kPairTile:
            if (kCap == 1) launch_pdl(k_field_pair<S, kCap>, p.blocks, 256, 0, s, p);
            else k_field_pair<S, kCap><<<p.blocks, 256, 0, s>>>(p);
            break;
        default:
            if (kCap == 1) launch_pdl(k_field_plain<S, kCap>, p.blocks, 256, 0, s, p);
            else k_field_plain<S, kCap><<<p.blocks, 256, 0, s>>>(p);
            break;
    }
}

template <int kCap>
static void launch_field_tiled_t(const TiledFieldParamsT<kCap>& p, int S, int tile,
                                 cudaStream_t s) {
    if (p.blocks <= 0) return;
    switch (S) {
        case 1: launch_for_species<1>(p, tile, s); break;
        case 2: launch_for_species<2>(p, tile, s); break;
        case 3: launch_for_species<3>(p, tile, s); break;
        default: launch_for_species<4>(p, tile, s); break;
    }
}

void launch_wait_selftest(int* flag, cudaStream_t s) { k_wait_selftest<<<1, 32, 0, s>>>(flag); }

void launch_field_tiled(const TiledFieldParams& p, int S, int tile, cudaStream_t s) {
    launch_field_tiled_t(p, S, tile, s);
}

void launch_field_tiled(const SingleFieldParams& p, int S, int tile, cudaStream_t s) {
    launch_field_tiled_t(p, S, tile, s);
}

// ------------------------------------------------------------------ tensor maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

bool encode_tiled_map(CUtensorMap* map, CUtensorMapDataType type, int rank, void* base,
                      const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return fn(map, type, (cuuint32_t)rank, base, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

// A tensor map over the int64 mesh D [S][Mz][My][Mx] with the box of `tile`.
// False when TMA cannot be used (odd Mx, unaligned base, no driver entry point).
bool make_mesh_tensor_map(CUtensorMap* map, const long long* D, const MeshGeom& g, int S,
                          int tile) {
    if (field_tile_is_plain(tile)) return false;
    if (g.mx % 2 != 0 || (reinterpret_cast<uintptr_t>(D) & 15u) != 0 || S > 4) return false;
    const int* t = kTileShapes[tile];
    const cuuint64_t dims[4] = {(cuuint64_t)g.mx, (cuuint64_t)g.my, (cuuint64_t)g.mz,
                                (cuuint64_t)S};
    const cuuint64_t strides[3] = {(cuuint64_t)g.mx * 8, (cuuint64_t)g.mx * g.my * 8,
                                   (cuuint64_t)g.mx * g.my * g.mz * 8};
    const cuuint32_t box[4] = {(cuuint32_t)(t[0] + 4), (cuuint32_t)(t[1] + 2),
                               (cuuint32_t)(t[2] + 2), (cuuint32_t)S};
    return encode_tiled_map(map, CU_TENSOR_MAP_DATA_TYPE_INT64, 4, const_cast<long long*>(D),
                            dims, strides, box);
}

void tile_grid(const MeshGeom& g, int tile, int* tiles_x, int* tiles_y, int* blocks) {
    const int* t = kTileShapes[tile];
    if (tile == kPairTile) {  // 256 node pairs of the real mesh per block
        *tiles_x = 0;
        *tiles_y = 0;
        *blocks = (((g.mx + 1) >> 1) * g.my * g.mz + 255) / 256;
        return;
    }
    if (t[0] == 0) {  // untiled: 256 nodes of the ghosted array per block
        *tiles_x = 0;
        *tiles_y = 0;
        *blocks = (g.gnodes + 255) / 256;
        return;
    }
    const int nx = (g.mx + 1 + t[0] - 1) / t[0];
    const int ny = (g.my + 1 + t[1] - 1) / t[1];
    const int nz = (g.mz + 1 + t[2] - 1) / t[2];
    *tiles_x = nx;
    *tiles_y = ny;
    *blocks = nx * ny * nz;
}

}  // namespace hpf
