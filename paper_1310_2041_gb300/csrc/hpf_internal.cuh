// hpf_internal.cuh -- shared declarations of the CUDA hPF-MD library.
//
// Device layout (all buffers owned by the context):
//   state   : SoA float arrays x, y, z, vx, vy, vz in storage order, two copies
//             (ping-pong) because the step kernel reads neighbours' old positions
//   meta    : uint32 per bead = tag (24 bits) | species (3 bits) << 24
//             | bonded-to-previous << 27 | bonded-to-next << 28
//   D       : int64 density [S][Mz][My][Mx], fixed point with 2^39 per bead
//   G       : float4 field  [S][Mz+1][My+1][Mx+1] = (dV/dx, dV/dy, dV/dz, V), with one
//             periodic ghost layer per axis so a cell's upper corner is always lo + 1
// Storage order keeps every chain contiguous (bonds only join storage
// neighbours); the sort permutes whole chains for locality.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <utility>

#include "hpf.h"

namespace hpf {

constexpr uint32_t kTagMask = 0x00FFFFFFu;
constexpr int kTypeShift = 24;
constexpr uint32_t kTypeMask = 0x7u;
constexpr uint32_t kBondPrev = 1u << 27;
constexpr uint32_t kBondNext = 1u << 28;
constexpr int kFrac = HPF_FRAC_BITS;
constexpr int kOne = 1 << kFrac;
constexpr float kCoordLimit = 262144.0f;  // |mesh coordinate| < 2^18 keeps 2^13 s in int32

// status bits raised by kernels into the context's device flag word
constexpr int kFlagNonFinite = 1;
constexpr int kFlagRange = 2;
constexpr int kFlagTimeout = 4;

struct MeshGeom {
    int mx, my, mz;
    int nodes;        // mx * my * mz
    int gx, gxy;      // field-array strides: mx + 1, (mx + 1)(my + 1)
    int gnodes;       // (mx + 1)(my + 1)(mz + 1)
    float inv_h[3];   // fl32(M / L): mesh coordinate s = fl32(x * inv_h)
    float inv_m[3];   // 1 / M, used only to wrap cell indices
};

struct StepConsts {
    float dt;
    float dt_m;       // dt / m
    float fric;       // gamma * m
    float sigma;      // sqrt(2 gamma m kT / dt)
    float two_k;      // 2 * bond_k
    float r0;
    uint32_t seed_lo, seed_hi;
    uint32_t rk0[10], rk1[10];  // Philox round keys: seed + r * (Weyl increments)
    int force_mode;             // field force: 0 interpolated gradient, 1 exact energy gradient,
                                // 2 staggered differences at the nearest vertex
    float two_ka;               // 2 * angle_k (0: no angle terms)
    float cos0;                 // cos of the equilibrium angle
    int angle_form;             // 0 cosine form, 1 harmonic form in theta
    float th0;                  // equilibrium angle of the harmonic form (radians)
    float p_coll;               // Andersen collision probability per step fl32(nu dt) (0: none)
    float sig_v;                // sqrt(kT / m): the Maxwell velocity scale
    float kd;                   // dihedral_k (0: no dihedral terms)
    int nd;                     // dihedral multiplicity n
    float cd, sd;               // cos and sin of the dihedral phase delta
    uint32_t tag_base;          // added to a bead's tag in its noise counter (parts of a system)
};

// Bonded terms the step kernels evaluate: 0 bonds, 1 bonds and angles,
// 2 bonds, angles and dihedrals (angle_k may be 0 there).
inline int bonded_level(const StepConsts& c) {
    return c.kd != 0.f ? 2 : (c.two_ka != 0.f ? 1 : 0);
}

// Thermostat of the step kernels: 0 none (NVE), 1 Langevin noise, 2 Andersen.
inline int step_thermostat(const StepConsts& c) {
    return c.sigma > 0.f ? 1 : (c.p_coll > 0.f ? 2 : 0);
}

// Coefficients of the field stencil: gradient of V_K from integer central
// differences of D_K', and V_K from D_K'.
struct FieldCoef {
    float gx[HPF_MAX_SPECIES][HPF_MAX_SPECIES];  // A_KK' c / (2 h_x)
    float gy[HPF_MAX_SPECIES][HPF_MAX_SPECIES];
    float gz[HPF_MAX_SPECIES][HPF_MAX_SPECIES];
    float v[HPF_MAX_SPECIES][HPF_MAX_SPECIES];   // A_KK' c
    float v0;                                    // -inv_kappa
    int S;
};

// Constants of the FP64 observables.
struct EnergyConsts {
    double half_dt_m;   // dt / (2m)
    double mass;
    double bond_k;
    double r0;
    float r0_hi, r0_lo;  // r0 as a float-float pair
    float bond_k_hi, bond_k_lo;  // bond_k as a float-float pair
    double kT;
    double inv_kappa;
    double phi_c;       // phi per fixed-point unit: 2^-39 / (rho0 h^3)
    double w_scale;     // rho0 h^3
    double chi[HPF_MAX_SPECIES][HPF_MAX_SPECIES];
    int S;
    int n;
    double angle_k, cos0;  // angle potential
    int angle_form;        // 0 cosine, 1 harmonic (theta0)
    double theta0;
    double dih_k;          // dihedral potential k [1 + cos(n phi - delta)]
    int dih_n;
    double dih_cd, dih_sd; // cos delta, sin delta
};

struct StateBuf {
    float* x;
    float* y;
    float* z;
    float* vx;
    float* vy;
    float* vz;
};

// Buffers of the chain sort (chain ids are fixed at state load, in tag order).
struct SortBufs {
    int* cstart;        // [C] storage index of each chain's first bead
    int* clen;          // [C]
    uint32_t* tag0;     // [C] tag of the first bead
    uint32_t* key;      // [C] sort key
    uint32_t* count;    // [K] bucket sizes
    uint32_t* binoff;   // [K] bucket offsets
    uint32_t* cursor;   // [K]
    int* order_tmp;     // [C]
    int* rank_of;       // [C] new position of chain c
    uint32_t* newstart; // [max(C, n)] new first-bead index per position (also a scan temp)
    int* chain_of_in;   // [n] chain of each bead, current order
    int* chain_of_out;  // [n]
    uint32_t* scratch;  // scan scratch
    // warp segments (whole chains, <= 64 beads each); seg_start == nullptr: not built
    int* seg_start;     // [C]
    int* seg_count;     // [C]
    int* seg_tmp;       // [2 C]
    uint32_t* chunk_nseg;  // [C / 256 + 1]
    uint32_t* chunk_off;   // [C / 256 + 1]
    int* n_seg;         // device scalar: number of segments
};

// Per-replica records of a batch, passed by value in the kernel parameter
// block (indexed by a warp-uniform replica id).
struct BatchStepRep {
    MeshGeom g;
    StepConsts c;
    StateBuf st[2];
    const uint32_t* meta;
    const int* seg_start;
    const int* seg_count;
    const int* n_seg;
    const float4* G;
    unsigned long long* D[2];
};

template <int kCap>
struct BatchStepParamsT {
    int R;
    int n_sub;
    int cur;       // state buffer read this launch (the other is written)
    int fuse;      // deposit the final positions into D[dnext]
    int dnext;
    long long step0;
    const long long* step_dev;  // if set, the step number is read here (graph replays)
    int* flag;
    BatchStepRep rep[kCap];
};
using BatchStepParams = BatchStepParamsT<HPF_MAX_REPLICAS>;
using SingleStepParams = BatchStepParamsT<1>;

struct BatchFieldRep {
    MeshGeom g;
    const long long* D;
    float4* G;
    unsigned long long* D_clear;   // mesh cleared by the same launch (NULL: none)
    int blk_begin;  // first block of this replica
};

struct BatchFieldParams {
    int R;
    int blocks;
    const FieldCoef* coef;  // [R] in device memory
    BatchFieldRep rep[HPF_MAX_REPLICAS];
};

// Tiled field stencil: one record per replica (a context is a batch of one).
struct TiledFieldRep {
    CUtensorMap tmap;  // over D (valid when use_tma)
    const FieldCoef* coef;  // this replica's stencil coefficients (device memory)
    MeshGeom g;
    const long long* D;
    float4* G;
    unsigned long long* D_clear;   // mesh cleared by the same launch (NULL: none)
    int use_tma;
    int tiles_x, tiles_y;
    int blk_begin;
};

// Capacity kCap replicas: a batch passes HPF_MAX_REPLICAS records, a single
// context one (a 64-record block is ~14 KB of kernel parameters per launch).
template <int kCap>
struct TiledFieldParamsT {
    int R;
    int blocks;
    int* flag;
    TiledFieldRep rep[kCap];
};
using TiledFieldParams = TiledFieldParamsT<HPF_MAX_REPLICAS>;
using SingleFieldParams = TiledFieldParamsT<1>;

// Run `f` once per device (ordinals taken modulo 64) for set-up that CUDA
// keeps per device, such as kernel attributes; thread-safe.
template <typename F>
inline void once_per_device(std::once_flag (&flags)[64], F&& f) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(flags[dev & 63], std::forward<F>(f));
}

// ------------------------------------------------------------------ dependent launch
//
// Programmatic dependent launch (sm_90+): a kernel launched with
// launch_pdl may be scheduled while its predecessor on the stream is still
// running, so launch latency overlaps the predecessor's tail.  Every such
// kernel executes griddep_wait() before its first global-memory access, which
// returns once the predecessor grid has completed and its writes are visible:
// the ordering is that of the plain stream.  griddep_launch_dependents() lets
// the next kernel be scheduled early (it waits in turn).  Both are no-ops for
// kernels launched without the attribute.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void griddep_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

// ------------------------------------------------------------------ device helpers

// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// with multipliers 0xD2511F53 and 0xCD9E8D57; the round keys (the key bumped
// by the Weyl increments 0x9E3779B9, 0xBB67AE85 per round) are precomputed.
__device__ __forceinline__ void philox4x32_10(uint32_t& c0, uint32_t& c1, uint32_t& c2,
                                              uint32_t& c3, const uint32_t* rk0,
                                              const uint32_t* rk1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)0xD2511F53u * c0;
        const unsigned long long p1 = (unsigned long long)0xCD9E8D57u * c2;
        c0 = (uint32_t)(p1 >> 32) ^ c1 ^ rk0[r];
        c1 = (uint32_t)p1;
        c2 = (uint32_t)(p0 >> 32) ^ c3 ^ rk1[r];
        c3 = (uint32_t)p0;
    }
}

// (2 (r >> 9) + 1) 2^-24: exact in FP32, strictly inside (0, 1).
__device__ __forceinline__ float open_uniform(uint32_t r) {
    return __uint2float_rn(2u * (r >> 9) + 1u) * 5.9604644775390625e-8f;
}

// ln u for a uniform u in (0, 1), with the relative accuracy that the
// Box-Muller radius sqrt(-2 ln u) needs as u -> 1.  With d = 1 - u (exact in
// FP32 for u >= 1/2): for d <= 2^-6, ln(1 - d) = -d (1 + d/2 + d^2/3) up to a
// relative d^3/4 <= 2^-20; otherwise the hardware logarithm (__logf: absolute
// error below 2^-21.4 on [1/2, 1), a few ulp below 1/2), which is below
// 2.3e-5 relative there since |ln u| >= 0.0157.  Branch-free (both forms are
// evaluated and one is selected).
__device__ __forceinline__ float log_unit(float u) {
    const float d = 1.0f - u;
    const float series = -d * fmaf(fmaf(d, 1.0f / 3.0f, 0.5f), d, 1.0f);
    const float hw = __logf(u);
    return d <= 0.015625f ? series : hw;
}

// Three standard normals of bead `tag` (its global tag is tag + c.tag_base)
// at step `step` (Box-Muller):
// x, y = sqrt(-2 ln u0) (cos, sin)(2 pi u1); z = sqrt(-2 ln u2) cos(2 pi u3).
// The angle is taken as 2 pi (u - 1/2) + pi, inside (-pi, pi) for the
// hardware sine and cosine.
__device__ __forceinline__ void gauss3(const StepConsts& c, uint32_t tag, long long step,
                                       float& gx, float& gy, float& gz) {
    uint32_t c0 = tag + c.tag_base, c1 = (uint32_t)step,
             c2 = (uint32_t)((unsigned long long)step >> 32), c3 = 0u;
    philox4x32_10(c0, c1, c2, c3, c.rk0, c.rk1);
    const float L0 = -2.0f * log_unit(open_uniform(c0));
    const float L2 = -2.0f * log_unit(open_uniform(c2));
    const float a = L0 * rsqrtf(L0);
    const float b = L2 * rsqrtf(L2);
    float s1, k1;
    __sincosf(6.28318530717958648f * (open_uniform(c1) - 0.5f), &s1, &k1);
    gx = -a * k1;
    gy = -a * s1;
    gz = -b * __cosf(6.28318530717958648f * (open_uniform(c3) - 0.5f));
}

// Andersen collision of bead `tag` at step `step`: the uniform of word 0 of
// Philox4x32-10(counter = (tag, step lo, step hi, 1)) below p_coll.  Both are
// exact in FP32, so the decision is the same as an FP64 comparison of them.
__device__ __forceinline__ bool andersen_collides(const StepConsts& c, uint32_t tag,
                                                  long long step) {
    uint32_t c0 = tag + c.tag_base, c1 = (uint32_t)step,
             c2 = (uint32_t)((unsigned long long)step >> 32), c3 = 1u;
    philox4x32_10(c0, c1, c2, c3, c.rk0, c.rk1);
    return open_uniform(c0) < c.p_coll;
}

// Mesh coordinate of one component.  t = floor(2^13 s) is exact in FP32, so
// cell = floor(s) = t >> 13 and q = t & 8191 = floor(2^13 frac(s)) exactly.
// f = s - floor(s) is the FP32 interpolation weight of the upper node.
struct AxisCoord {
    int lo, hi, q;
    float f;
};

__device__ __forceinline__ int wrap_cell(int c, int m, float inv_m) {
    int w = c - m * __float2int_rd(__int2float_rn(c) * inv_m);
    if (w < 0) w += m;
    else if (w >= m) w -= m;
    return w;
}

__device__ __forceinline__ AxisCoord axis_coord(float x, float inv_h, int m, float inv_m) {
    AxisCoord a;
    const float s = __fmul_rn(x, inv_h);
    const int t = __float2int_rd(__fmul_rn(s, 8192.0f));
    a.q = t & (kOne - 1);
    a.f = __fsub_rn(s, floorf(s));
    a.lo = wrap_cell(t >> kFrac, m, inv_m);
    a.hi = (a.lo + 1 == m) ? 0 : a.lo + 1;
    return a;
}

// Lower node and interpolation weight only (the field array's ghost layers
// make the upper node lo + 1).  floor(s) is an exact integer-valued float and
// floor((fl + 1/2) / M) = floor(fl / M) holds in FP32 for |fl| < 2^22 (the
// half-integer is never a multiple of M, and the relative error 2^-23 stays
// below the distance 1/(2M) to the nearest integer), so no fix-up is needed;
// the clamp only keeps out-of-range input inside the array.
__device__ __forceinline__ AxisCoord axis_gather(float x, float inv_h, float m, float inv_m) {
    AxisCoord a;
    const float s = __fmul_rn(x, inv_h);
    const float fl = floorf(s);
    a.f = __fsub_rn(s, fl);
    float w = __fmaf_rn(-m, floorf((fl + 0.5f) * inv_m), fl);
    w = fminf(fmaxf(w, 0.0f), m - 1.0f);
    a.lo = (int)w;
    a.hi = a.lo + 1;
    a.q = 0;
    return a;
}

__device__ __forceinline__ bool coord_in_range(float x, float inv_h) {
    const float s = __fmul_rn(x, inv_h);
    return fabsf(s) < kCoordLimit;
}

// Add one bead's eight fixed-point CIC weights to its species' mesh.
__device__ __forceinline__ void scatter_bead(unsigned long long* __restrict__ Dt, const MeshGeom& g,
                                             const AxisCoord& ax, const AxisCoord& ay,
                                             const AxisCoord& az) {
    const unsigned long long wx0 = (unsigned long long)(kOne - ax.q), wx1 = (unsigned long long)ax.q;
    const unsigned long long wy[2] = {(unsigned long long)(kOne - ay.q), (unsigned long long)ay.q};
    const unsigned long long wz[2] = {(unsigned long long)(kOne - az.q), (unsigned long long)az.q};
    const int ny[2] = {ay.lo, ay.hi}, nz[2] = {az.lo, az.hi};
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const unsigned long long wzy = wz[dz] * wy[dy];
            unsigned long long* row = Dt + (nz[dz] * g.my + ny[dy]) * g.mx;
            const unsigned long long a = wzy * wx0, b = wzy * wx1;
            if (a) atomicAdd(row + ax.lo, a);
            if (b) atomicAdd(row + ax.hi, b);
        }
}

// -trilinear interpolation of the nodal gradient of one species (ghosted
// field array: the eight corners are base + {0, 1} + {0, gx} + {0, gxy}).
__device__ __forceinline__ void gather_field(const float4* __restrict__ Gt, const MeshGeom& g,
                                             const AxisCoord& ax, const AxisCoord& ay,
                                             const AxisCoord& az, float& fx, float& fy,
                                             float& fz) {
    const float wx1 = ax.f, wx0 = 1.0f - ax.f;
    const float wy1 = ay.f, wy0 = 1.0f - ay.f;
    const float wz1 = az.f, wz0 = 1.0f - az.f;
    const int o00 = az.lo * g.gxy + ay.lo * g.gx + ax.lo;
    const int o01 = o00 + g.gx, o10 = o00 + g.gxy, o11 = o10 + g.gx;
    const float4 c000 = __ldg(Gt + o00), c001 = __ldg(Gt + o00 + 1);
    const float4 c010 = __ldg(Gt + o01), c011 = __ldg(Gt + o01 + 1);
    const float4 c100 = __ldg(Gt + o10), c101 = __ldg(Gt + o10 + 1);
    const float4 c110 = __ldg(Gt + o11), c111 = __ldg(Gt + o11 + 1);
    const float w00 = wz0 * wy0, w01 = wz0 * wy1, w10 = wz1 * wy0, w11 = wz1 * wy1;
    float gx = w00 * (wx0 * c000.x + wx1 * c001.x) + w01 * (wx0 * c010.x + wx1 * c011.x) +
               w10 * (wx0 * c100.x + wx1 * c101.x) + w11 * (wx0 * c110.x + wx1 * c111.x);
    float gy = w00 * (wx0 * c000.y + wx1 * c001.y) + w01 * (wx0 * c010.y + wx1 * c011.y) +
               w10 * (wx0 * c100.y + wx1 * c101.y) + w11 * (wx0 * c110.y + wx1 * c111.y);
    float gz = w00 * (wx0 * c000.z + wx1 * c001.z) + w01 * (wx0 * c010.z + wx1 * c011.z) +
               w10 * (wx0 * c100.z + wx1 * c101.z) + w11 * (wx0 * c110.z + wx1 * c111.z);
    fx -= gx;
    fy -= gy;
    fz -= gz;
}

// The exact derivative of the CIC field energy at a bead: minus the gradient
// of the trilinear interpolant of V_T (the .w of the ghosted field array),
// -sum over the 8 corners of V_c grad w_c with grad w = (+-1/h) per axis.
__device__ __forceinline__ void gather_field_exact(const float4* __restrict__ Gt,
                                                   const MeshGeom& g, const AxisCoord& ax,
                                                   const AxisCoord& ay, const AxisCoord& az,
                                                   float& fx, float& fy, float& fz) {
    const float wx1 = ax.f, wx0 = 1.0f - ax.f;
    const float wy1 = ay.f, wy0 = 1.0f - ay.f;
    const float wz1 = az.f, wz0 = 1.0f - az.f;
    const int o00 = az.lo * g.gxy + ay.lo * g.gx + ax.lo;
    const int o01 = o00 + g.gx, o10 = o00 + g.gxy, o11 = o10 + g.gx;
    const float v000 = __ldg(Gt + o00).w, v100 = __ldg(Gt + o00 + 1).w;
    const float v010 = __ldg(Gt + o01).w, v110 = __ldg(Gt + o01 + 1).w;
    const float v001 = __ldg(Gt + o10).w, v101 = __ldg(Gt + o10 + 1).w;
    const float v011 = __ldg(Gt + o11).w, v111 = __ldg(Gt + o11 + 1).w;
    // d/dfx, d/dfy, d/dfz of the interpolant
    const float dx = wz0 * (wy0 * (v100 - v000) + wy1 * (v110 - v010)) +
                     wz1 * (wy0 * (v101 - v001) + wy1 * (v111 - v011));
    const float dy = wz0 * (wx0 * (v010 - v000) + wx1 * (v110 - v100)) +
                     wz1 * (wx0 * (v011 - v001) + wx1 * (v111 - v101));
    const float dz = wy0 * (wx0 * (v001 - v000) + wx1 * (v101 - v100)) +
                     wy1 * (wx0 * (v011 - v010) + wx1 * (v111 - v110));
    fx = fmaf(-g.inv_h[0], dx, fx);
    fy = fmaf(-g.inv_h[1], dy, fy);
    fz = fmaf(-g.inv_h[2], dz, fz);
}

// Algorithm 1's staggered field force (kernels 3-4 read literally): along each
// axis the backward and forward differences of V at the vertex c nearest the
// bead are blended with the linear fractions 1/2 - d and 1/2 + d, d = s - c:
//   F_a = -(1/h_a) [g0 + d g1],  g0 = (V(c+1) - V(c-1)) / 2,  g1 = V(c+1) - 2 V(c) + V(c-1)
// (the derivative of the quadratic through the three values on the vertex's
// grid line).  stag_coefs and the final fma are shared by the direct gather
// and the per-bead cache of the step kernels, so both give the same bits.
__device__ __forceinline__ float stag_vertex(float s) { return floorf(s + 0.5f); }

// Periodic image of a vertex coordinate (an integer-valued float) in [0, m).
__device__ __forceinline__ float vertex_wrap(float k, float m, float inv_m) {
    const float w = __fmaf_rn(-m, floorf((k + 0.5f) * inv_m), k);
    return fminf(fmaxf(w, 0.0f), m - 1.0f);
}

__device__ __forceinline__ void stag_coefs(float vm, float vc, float vp, float& g0, float& g1) {
    g0 = 0.5f * (vp - vm);
    g1 = (vp - vc) - (vc - vm);
}

// The six coefficients (g0, g1 per axis) of the bead's nearest vertex
// (kx, ky, kz) from the V components of the ghosted field array.
__device__ __forceinline__ void stag_vertex_coefs(const float4* __restrict__ Gt, const MeshGeom& g,
                                                  float kx, float ky, float kz, float (&c)[6]) {
    const float wx = vertex_wrap(kx, (float)g.mx, g.inv_m[0]);
    const float wy = vertex_wrap(ky, (float)g.my, g.inv_m[1]);
    const float wz = vertex_wrap(kz, (float)g.mz, g.inv_m[2]);
    const int ix = (int)wx, iy = (int)wy, iz = (int)wz;
    const int o = iz * g.gxy + iy * g.gx + ix;
    // the upper neighbours may be ghost entries; the lower ones wrap
    const int oxm = ix == 0 ? o + (g.mx - 1) : o - 1;
    const int oym = iy == 0 ? o + (g.my - 1) * g.gx : o - g.gx;
    const int ozm = iz == 0 ? o + (g.mz - 1) * g.gxy : o - g.gxy;
    const float vc = __ldg(Gt + o).w;
    stag_coefs(__ldg(Gt + oxm).w, vc, __ldg(Gt + o + 1).w, c[0], c[1]);
    stag_coefs(__ldg(Gt + oym).w, vc, __ldg(Gt + o + g.gx).w, c[2], c[3]);
    stag_coefs(__ldg(Gt + ozm).w, vc, __ldg(Gt + o + g.gxy).w, c[4], c[5]);
}

__device__ __forceinline__ void stag_force(const float (&c)[6], float dx, float dy, float dz,
                                           const MeshGeom& g, float& fx, float& fy, float& fz) {
    fx = fmaf(-g.inv_h[0], fmaf(dx, c[1], c[0]), fx);
    fy = fmaf(-g.inv_h[1], fmaf(dy, c[3], c[2]), fy);
    fz = fmaf(-g.inv_h[2], fmaf(dz, c[5], c[4]), fz);
}

// The staggered field force at position (x, y, z), gathered directly.
__device__ __forceinline__ void gather_field_staggered(const float4* __restrict__ Gt,
                                                       const MeshGeom& g, float x, float y,
                                                       float z, float& fx, float& fy, float& fz) {
    const float sx = __fmul_rn(x, g.inv_h[0]), sy = __fmul_rn(y, g.inv_h[1]),
                sz = __fmul_rn(z, g.inv_h[2]);
    const float kx = stag_vertex(sx), ky = stag_vertex(sy), kz = stag_vertex(sz);
    float c[6];
    stag_vertex_coefs(Gt, g, kx, ky, kz, c);
    stag_force(c, __fsub_rn(sx, kx), __fsub_rn(sy, ky), __fsub_rn(sz, kz), g, fx, fy, fz);
}

// Field force of mode 0, 1 or 2 at (x, y, z), gathered directly.
__device__ __forceinline__ void gather_field_mode(const float4* __restrict__ Gt, const MeshGeom& g,
                                                  int mode, float x, float y, float z, float& fx,
                                                  float& fy, float& fz) {
    if (mode == 2) {
        gather_field_staggered(Gt, g, x, y, z, fx, fy, fz);
        return;
    }
    const AxisCoord ax = axis_gather(x, g.inv_h[0], (float)g.mx, g.inv_m[0]);
    const AxisCoord ay = axis_gather(y, g.inv_h[1], (float)g.my, g.inv_m[1]);
    const AxisCoord az = axis_gather(z, g.inv_h[2], (float)g.mz, g.inv_m[2]);
    if (mode == 1) gather_field_exact(Gt, g, ax, ay, az, fx, fy, fz);
    else gather_field(Gt, g, ax, ay, az, fx, fy, fz);
}

// ------------------------------------------------------------------ float-float sums

// Per-block partial sums of the observables' bead terms, in this order:
// |v_n|^2 (kinetic energy without m/2), bond energy, momentum x, y, z
// (without m); each a float-float pair (h, l).
constexpr int kBeadVals = 5;


// Knuth's two-sum: s + t == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    t = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Float-float sums (h, l): the partial sums of every observable are carried as
// pairs of FP32 numbers, added with two-sum and renormalised, so that the
// block and warp reductions run on the FP32 pipe (this GPU's FP64 rate is
// 1/64 of its FP32 rate) with about 2^-45 relative error per addition, and in
// a fixed tree, so that every bit is the same from run to run.
struct FF {
    float h, l;
};
__device__ __forceinline__ FF ff_norm(float s, float t) {
    const float h = __fadd_rn(s, t);
    return FF{h, __fsub_rn(t, __fsub_rn(h, s))};
}
__device__ __forceinline__ FF ff_plus(FF a, float x) {
    float s, t;
    two_sum(a.h, x, s, t);
    return ff_norm(s, __fadd_rn(t, a.l));
}
__device__ __forceinline__ FF ff_plus(FF a, FF b) {
    float s, t;
    two_sum(a.h, b.h, s, t);
    return ff_norm(s, __fadd_rn(t, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ FF ff_from_double(double v) {
    const float h = (float)v;
    return FF{h, (float)(v - (double)h)};
}
__device__ __forceinline__ double ff_to_double(FF v) { return (double)v.h + (double)v.l; }
__device__ __forceinline__ FF warp_sum_ff(FF v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = ff_plus(v, FF{__shfl_down_sync(0xffffffffu, v.h, o),
                          __shfl_down_sync(0xffffffffu, v.l, o)});
    return v;  // lane 0
}

// The bond energy k (|d| - r0)^2 of d = x_i - x_j in float-float arithmetic
// (pairs of FP32 numbers), added to the float-float sum (uh, ul): each
// component of d exactly by two-sum, |d|^2 with the exact error of each
// square (FMA) to about 2^-46, |d| from the correctly rounded square root plus
// its residual, |d| - r0 = a + b against r0 = r0_hi + r0_lo, renormalised
// by two-sum; then (a + b)^2 = a^2 + 2ab + b^2 with |b| <= ulp(a)/2 -- a^2
// exactly as p + pe,
// 2ab rounded (2^-24 of a term 2^-23 below a^2), b^2 (2^-48 of a^2)
// dropped -- times k = k_hi + k_lo, and a two-sum accumulation.  About
// 2^-45 relative per term, like an FP64 evaluation, with no FP64 instruction
// (this GPU's FP64 rate is 1/64 of its FP32 rate).
struct BondFF {
    float r0_hi, r0_lo;  // r0 as a float-float pair
    float k_hi, k_lo;    // the bond constant k as a float-float pair
};
__device__ __forceinline__ void bond_energy_ff(float xi, float yi, float zi, float xj, float yj,
                                               float zj, const BondFF& e, float& uh,
                                               float& ul) {
    float hx, lx, hy, ly, hz, lz;
    two_sum(xi, -xj, hx, lx);
    two_sum(yi, -yj, hy, ly);
    two_sum(zi, -zj, hz, lz);
    float H = 0.f, L = 0.f;
    const float hs[3] = {hx, hy, hz}, ls[3] = {lx, ly, lz};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float p = __fmul_rn(hs[c], hs[c]);
        const float pe = fmaf(hs[c], hs[c], -p);                        // exact error of h^2
        const float rest = fmaf(2.0f * hs[c], ls[c], fmaf(ls[c], ls[c], pe));  // 2hl + l^2 + pe
        float t;
        two_sum(H, p, H, t);
        L = __fadd_rn(L, __fadd_rn(t, rest));
    }
    const float H2 = __fadd_rn(H, L);
    const float L2 = __fsub_rn(L, __fsub_rn(H2, H));
    float a, b;
    if (H2 > 0.f) {
        const float r = sqrtf(H2);
        const float res = __fadd_rn(fmaf(-r, r, H2), L2);  // H2 - r^2 is exact
        const float r_lo = 0.5f * res * rsqrtf(H2);
        two_sum(r, -e.r0_hi, a, b);
        b = __fadd_rn(b, __fsub_rn(r_lo, e.r0_lo));
    } else {  // coincident beads: |d| - r0 = -r0
        a = -e.r0_hi;
        b = -e.r0_lo;
    }
    // renormalised, so that |b| <= ulp(a)/2 also when |d| is close to r0 (then
    // the two parts of the difference are of similar size)
    two_sum(a, b, a, b);
    const float p = __fmul_rn(a, a);
    const float pe = fmaf(a, a, -p);
    const float q = fmaf(2.0f * a, b, pe);
    const float u = __fmul_rn(e.k_hi, p);
    const float ue = fmaf(e.k_hi, p, -u);
    const float w = fmaf(e.k_hi, q, fmaf(e.k_lo, p, ue));
    float s, t;
    two_sum(uh, u, s, t);
    t = __fadd_rn(t, __fadd_rn(ul, w));
    uh = __fadd_rn(s, t);
    ul = __fsub_rn(t, __fsub_rn(uh, s));
}

__host__ __device__ __forceinline__ BondFF bond_ff(const EnergyConsts& e) {
    return BondFF{e.r0_hi, e.r0_lo, e.bond_k_hi, e.bond_k_lo};
}

// Harmonic bond U = k (r - r0)^2 seen from bead i: F_i += -2k (1 - r0 / r) d, d = x_i - x_j,
// with 1 / r from the hardware reciprocal square root (2 ulp: about 1e-6 of a
// typical bond force).
__device__ __forceinline__ void bond_force(float dx, float dy, float dz, float two_k, float r0,
                                           float& fx, float& fy, float& fz) {
    // r^2 is clamped so that a masked bond (two_k = 0, zero vector) adds exactly zero
    const float r2 = fmaxf(dx * dx + dy * dy + dz * dz, 1e-30f);
    const float ir = rsqrtf(r2);
    const float s = -two_k * fmaf(-r0, ir, 1.0f);
    fx += s * dx;
    fy += s * dy;
    fz += s * dz;
}

// Angle at a middle bead j with u = x_a - x_j, w = x_b - x_j: forces on the
// end beads a and b (the middle bead takes minus their sum), g dc/dx with
// c = cos theta, dc/dx_a = w / (|u||w|) - c u / |u|^2 and dc/dx_b symmetric.
// Cosine form U = k (c - cos0)^2: g = -2k (c - cos0).  Harmonic form
// U = k (theta - theta0)^2, theta = atan2(|u x w|, u.w): dtheta/dx =
// -(1 / sin theta) dc/dx, so g = 2k (theta - theta0) / sin theta.  Lengths and
// sin theta are clamped, so every intermediate stays finite even for zero
// vectors (lanes without beads) and two_ka = 0 gives exactly zero.
__device__ __forceinline__ void angle_force(float ux, float uy, float uz, float wx, float wy,
                                            float wz, float two_ka, const StepConsts& sc,
                                            float& fax, float& fay, float& faz, float& fbx,
                                            float& fby, float& fbz) {
    const float uu = fmaxf(ux * ux + uy * uy + uz * uz, 1e-30f);
    const float ww = fmaxf(wx * wx + wy * wy + wz * wz, 1e-30f);
    const float uw = ux * wx + uy * wy + uz * wz;
    const float ru = rsqrtf(uu), rw = rsqrtf(ww);  // 1/|u|, 1/|w|: no divisions below
    const float inv = ru * rw;
    const float c = uw * inv;
    float g;
    if (sc.angle_form == 1) {
        const float qx = uy * wz - uz * wy, qy = uz * wx - ux * wz, qz = ux * wy - uy * wx;
        const float qq = fmaxf(qx * qx + qy * qy + qz * qz, 1e-30f);  // |u x w|^2
        const float rq = rsqrtf(qq);
        const float th = atan2f(qq * rq, uw);
        // 1 / sin theta = |u||w| / |u x w|
        g = two_ka * (th - sc.th0) * rq * ((uu * ru) * (ww * rw));
    } else {
        g = -two_ka * (c - sc.cos0);
    }
    const float ca = c * (ru * ru), cb = c * (rw * rw);
    fax = g * (wx * inv - ca * ux);
    fay = g * (wy * inv - ca * uy);
    faz = g * (wz * inv - ca * uz);
    fbx = g * (ux * inv - cb * wx);
    fby = g * (uy * inv - cb * wy);
    fbz = g * (uz * inv - cb * wz);
}

// The three angles bead i belongs to (centred at i - 1, i and i + 1), read
// from global memory in storage order (chains are contiguous there).
__device__ __forceinline__ void angle_forces_of(const StateBuf& st, const uint32_t* __restrict__ meta,
                                                int i, uint32_t m, const StepConsts& c, float& fx,
                                                float& fy, float& fz) {
    const bool hp = (m & kBondPrev) != 0, hn = (m & kBondNext) != 0;
    const float x = st.x[i], y = st.y[i], z = st.z[i];
    float ax, ay, az, bx, by, bz;
    if (hp && hn) {
        angle_force(st.x[i - 1] - x, st.y[i - 1] - y, st.z[i - 1] - z, st.x[i + 1] - x,
                    st.y[i + 1] - y, st.z[i + 1] - z, c.two_ka, c, ax, ay, az, bx, by, bz);
        fx -= ax + bx;
        fy -= ay + by;
        fz -= az + bz;
    }
    if (hp && (meta[i - 1] & kBondPrev)) {
        const float xp = st.x[i - 1], yp = st.y[i - 1], zp = st.z[i - 1];
        angle_force(st.x[i - 2] - xp, st.y[i - 2] - yp, st.z[i - 2] - zp, x - xp, y - yp, z - zp,
                    c.two_ka, c, ax, ay, az, bx, by, bz);
        fx += bx;
        fy += by;
        fz += bz;
    }
    if (hn && (meta[i + 1] & kBondNext)) {
        const float xn = st.x[i + 1], yn = st.y[i + 1], zn = st.z[i + 1];
        angle_force(x - xn, y - yn, z - zn, st.x[i + 2] - xn, st.y[i + 2] - yn, st.z[i + 2] - zn,
                    c.two_ka, c, ax, ay, az, bx, by, bz);
        fx += ax;
        fy += ay;
        fz += az;
    }
}

__device__ __forceinline__ float3 f3_sub(float3 a, float3 b) {
    return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float3 f3_cross(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float f3_dot(float3 a, float3 b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Dihedral U = k [1 + cos(n phi - delta)] of the bonded quadruplet 0-1-2-3
// from its bond vectors b1 = x1 - x0, b2 = x2 - x1, b3 = x3 - x2.  With
// A = b1 x b2 and B = b2 x b3: cos phi = A.B / (|A||B|), sin phi =
// |b2| b1.B / (|A||B|) (trans pi, cis 0), and cos(n phi), sin(n phi) are the
// n-th power of cos phi + i sin phi, so no angle is formed.  With
// g = dU/dphi = -k n sin(n phi - delta) the end beads take F0 = g |b2| A / |A|^2
// and F3 = -g |b2| B / |B|^2, the middle ones F1 = S - F0 and F2 = -(F3 + S),
// S = pa F0 - pb F3, pa = -b1.b2 / |b2|^2, pb = -b3.b2 / |b2|^2 (no net force
// or torque).  Squared norms are clamped, so for any finite vectors every
// intermediate stays finite (|cos phi|, |sin phi| <= 1 up to rounding) and a
// masked quadruplet (kd = 0) gives exactly zero.
__device__ __forceinline__ void dihedral_force(float3 b1, float3 b2, float3 b3, float kd,
                                               const StepConsts& c, float3& f0, float3& f1,
                                               float3& f2, float3& f3) {
    const float3 A = f3_cross(b1, b2), B = f3_cross(b2, b3);
    const float AA = fmaxf(f3_dot(A, A), 1e-30f), BB = fmaxf(f3_dot(B, B), 1e-30f);
    const float b22 = fmaxf(f3_dot(b2, b2), 1e-30f);
    const float ib = rsqrtf(b22);
    const float L = b22 * ib;  // |b2|
    const float rA = rsqrtf(AA), rB = rsqrtf(BB);  // no divisions below
    const float inv = rA * rB;
    const float cp = f3_dot(A, B) * inv, sp = L * f3_dot(b1, B) * inv;
    float cn = cp, sn = sp;
    for (int k = 1; k < c.nd; ++k) {
        const float t = fmaf(cn, cp, -sn * sp);
        sn = fmaf(sn, cp, cn * sp);
        cn = t;
    }
    const float g = -kd * (float)c.nd * fmaf(sn, c.cd, -cn * c.sd);
    const float a0 = g * L * (rA * rA), a3 = -g * L * (rB * rB);
    f0 = make_float3(a0 * A.x, a0 * A.y, a0 * A.z);
    f3 = make_float3(a3 * B.x, a3 * B.y, a3 * B.z);
    const float ib2 = ib * ib;
    const float pa = -f3_dot(b1, b2) * ib2, pb = -f3_dot(b3, b2) * ib2;
    const float3 S = make_float3(fmaf(pa, f0.x, -pb * f3.x), fmaf(pa, f0.y, -pb * f3.y),
                                 fmaf(pa, f0.z, -pb * f3.z));
    f1 = f3_sub(S, f0);
    f2 = make_float3(-(f3.x + S.x), -(f3.y + S.y), -(f3.z + S.z));
}

// How many consecutive bonds lead from bead i backwards (back) and forwards
// (fwd) along its chain, each capped at 3; chains are contiguous in storage.
__device__ __forceinline__ void chain_reach(const uint32_t* __restrict__ meta, int i, uint32_t m,
                                            int& back, int& fwd) {
    back = 0;
    fwd = 0;
    if (m & kBondPrev) {
        back = 1;
        if (meta[i - 1] & kBondPrev) {
            back = 2;
            if (meta[i - 2] & kBondPrev) back = 3;
        }
    }
    if (m & kBondNext) {
        fwd = 1;
        if (meta[i + 1] & kBondNext) {
            fwd = 2;
            if (meta[i + 2] & kBondNext) fwd = 3;
        }
    }
}

// Dihedral forces on one bead from the (up to four) quadruplets it belongs
// to, which start 3, 2, 1 and 0 beads before it; back / fwd as chain_reach,
// pos(d) the position of the bead d places along the chain (-back <= d <= fwd).
template <class Pos>
__device__ __forceinline__ void dihedral_forces_of(Pos pos, int back, int fwd, const StepConsts& c,
                                                   float& fx, float& fy, float& fz) {
    float3 P[7];
#pragma unroll
    for (int d = -3; d <= 3; ++d)
        P[d + 3] = (d >= -back && d <= fwd) ? pos(d) : make_float3(0.f, 0.f, 0.f);
#pragma unroll
    for (int q = 0; q < 4; ++q) {  // the quadruplet starting q beads back: this bead is its q-th
        if (back >= q && fwd >= 3 - q) {
            float3 f[4];
            dihedral_force(f3_sub(P[4 - q], P[3 - q]), f3_sub(P[5 - q], P[4 - q]),
                           f3_sub(P[6 - q], P[5 - q]), c.kd, c, f[0], f[1], f[2], f[3]);
            fx += f[q].x;
            fy += f[q].y;
            fz += f[q].z;
        }
    }
}

// Bonded forces of one warp segment of whole chains: lane l holds beads 2l
// and 2l + 1 at (x0, y0, z0) and (x1, y1, z1); p0, n0: bead 2l is bonded to
// its previous / next bead, n1: bead 2l + 1 to its next.  Returns the summed
// bond forces on the lane's two beads, with kBonded >= 1 the angle forces
// and with kBonded == 2 the dihedral forces.
template <int kBonded>
__device__ __forceinline__ void warp_bonded_forces(float x0, float y0, float z0, float x1, float y1,
                                                   float z1, bool p0, bool n0, bool n1,
                                                   const StepConsts& c, int lane, float& w0x,
                                                   float& w0y, float& w0z, float& w1x,
                                                   float& w1y, float& w1z) {
    // every bond is evaluated once: bond (2l, 2l + 1) inside the lane, bond
    // (2l + 1, 2l + 2) with the next lane's first bead, whose share (the
    // opposite force) goes back up one lane
    const float dx = __shfl_down_sync(0xffffffffu, x0, 1);
    const float dy = __shfl_down_sync(0xffffffffu, y0, 1);
    const float dz = __shfl_down_sync(0xffffffffu, z0, 1);
    float ax = 0.f, ay = 0.f, az = 0.f;  // on bead 2l from bead 2l + 1
    bond_force(x0 - x1, y0 - y1, z0 - z1, n0 ? c.two_k : 0.0f, c.r0, ax, ay, az);
    float nx = 0.f, ny = 0.f, nz = 0.f;  // on bead 2l + 1 from bead 2l + 2
    bond_force(x1 - dx, y1 - dy, z1 - dz, n1 ? c.two_k : 0.0f, c.r0, nx, ny, nz);
    const float ux = __shfl_up_sync(0xffffffffu, nx, 1);  // previous lane's share
    const float uy = __shfl_up_sync(0xffffffffu, ny, 1);
    const float uz = __shfl_up_sync(0xffffffffu, nz, 1);
    // angles, each evaluated once by the lane of its middle bead: at bead 2l
    // (ends 2l - 1, 2l + 1) and at bead 2l + 1 (ends 2l, 2l + 2); the shares
    // of the end beads held by the neighbouring lanes go there by one shuffle
    float q0x = 0.f, q0y = 0.f, q0z = 0.f, q1x = 0.f, q1y = 0.f, q1z = 0.f;
    if (kBonded >= 1) {
        const float px = __shfl_up_sync(0xffffffffu, x1, 1);  // bead 2l - 1
        const float py = __shfl_up_sync(0xffffffffu, y1, 1);
        const float pz = __shfl_up_sync(0xffffffffu, z1, 1);
        float fpx, fpy, fpz, f1x, f1y, f1z, f0x, f0y, f0z, fdx, fdy, fdz;
        angle_force(px - x0, py - y0, pz - z0, x1 - x0, y1 - y0, z1 - z0,
                    (p0 && n0) ? c.two_ka : 0.0f, c, fpx, fpy, fpz, f1x, f1y, f1z);
        angle_force(x0 - x1, y0 - y1, z0 - z1, dx - x1, dy - y1, dz - z1,
                    (n0 && n1) ? c.two_ka : 0.0f, c, f0x, f0y, f0z, fdx, fdy, fdz);
        // from lane l - 1: its share on bead 2l; from lane l + 1: its share on bead 2l + 1
        const float r0x = __shfl_up_sync(0xffffffffu, fdx, 1);
        const float r0y = __shfl_up_sync(0xffffffffu, fdy, 1);
        const float r0z = __shfl_up_sync(0xffffffffu, fdz, 1);
        const float r1x = __shfl_down_sync(0xffffffffu, fpx, 1);
        const float r1y = __shfl_down_sync(0xffffffffu, fpy, 1);
        const float r1z = __shfl_down_sync(0xffffffffu, fpz, 1);
        const bool first = lane == 0, last = lane == 31;
        q0x = f0x - (fpx + f1x) + (first ? 0.f : r0x);
        q0y = f0y - (fpy + f1y) + (first ? 0.f : r0y);
        q0z = f0z - (fpz + f1z) + (first ? 0.f : r0z);
        q1x = f1x - (f0x + fdx) + (last ? 0.f : r1x);
        q1y = f1y - (f0y + fdy) + (last ? 0.f : r1y);
        q1z = f1z - (f0z + fdz) + (last ? 0.f : r1z);
    }
    w0x = (p0 ? ax - ux : ax) + q0x;
    w0y = (p0 ? ay - uy : ay) + q0y;
    w0z = (p0 ? az - uz : az) + q0z;
    w1x = (nx - ax) + q1x;
    w1y = (ny - ay) + q1y;
    w1z = (nz - az) + q1z;
    if (kBonded == 2) {
        // dihedrals, each evaluated once by the lane of its first bead: Q0 =
        // (2l .. 2l + 3) and Q1 = (2l + 1 .. 2l + 4).  Their shares on beads
        // 2l + 2 and 2l + 3 go up one lane, Q1's share on bead 2l + 4 two
        // lanes.  The last bead of a segment has no next bond, so no valid
        // quadruplet reaches past lane 31.
        const float3 r0 = make_float3(x0, y0, z0), r1 = make_float3(x1, y1, z1);
        const float3 r2 = make_float3(dx, dy, dz);  // bead 2l + 2
        const float3 r3 = make_float3(__shfl_down_sync(0xffffffffu, x1, 1),
                                      __shfl_down_sync(0xffffffffu, y1, 1),
                                      __shfl_down_sync(0xffffffffu, z1, 1));
        const float3 r4 = make_float3(__shfl_down_sync(0xffffffffu, x0, 2),
                                      __shfl_down_sync(0xffffffffu, y0, 2),
                                      __shfl_down_sync(0xffffffffu, z0, 2));
        const bool n2 = __shfl_down_sync(0xffffffffu, (int)n0, 1) != 0;  // bond 2l+2 -> 2l+3
        const bool n3 = __shfl_down_sync(0xffffffffu, (int)n1, 1) != 0;  // bond 2l+3 -> 2l+4
        const float3 b01 = f3_sub(r1, r0), b12 = f3_sub(r2, r1), b23 = f3_sub(r3, r2),
                     b34 = f3_sub(r4, r3);
        float3 e0, e1, e2, e3, h1, h2, h3, h4;
        dihedral_force(b01, b12, b23, (n0 && n1 && n2) ? c.kd : 0.0f, c, e0, e1, e2, e3);
        dihedral_force(b12, b23, b34, (n1 && n2 && n3) ? c.kd : 0.0f, c, h1, h2, h3, h4);
        const float u0x = e2.x + h2.x, u0y = e2.y + h2.y, u0z = e2.z + h2.z;  // to lane l+1, bead 0
        const float u1x = e3.x + h3.x, u1y = e3.y + h3.y, u1z = e3.z + h3.z;  // to lane l+1, bead 1
        const float v0x = __shfl_up_sync(0xffffffffu, u0x, 1);
        const float v0y = __shfl_up_sync(0xffffffffu, u0y, 1);
        const float v0z = __shfl_up_sync(0xffffffffu, u0z, 1);
        const float v1x = __shfl_up_sync(0xffffffffu, u1x, 1);
        const float v1y = __shfl_up_sync(0xffffffffu, u1y, 1);
        const float v1z = __shfl_up_sync(0xffffffffu, u1z, 1);
        const float v2x = __shfl_up_sync(0xffffffffu, h4.x, 2);
        const float v2y = __shfl_up_sync(0xffffffffu, h4.y, 2);
        const float v2z = __shfl_up_sync(0xffffffffu, h4.z, 2);
        const bool up1 = lane >= 1, up2 = lane >= 2;
        w0x += e0.x + (up1 ? v0x : 0.f) + (up2 ? v2x : 0.f);
        w0y += e0.y + (up1 ? v0y : 0.f) + (up2 ? v2y : 0.f);
        w0z += e0.z + (up1 ? v0z : 0.f) + (up2 ? v2z : 0.f);
        w1x += (e1.x + h1.x) + (up1 ? v1x : 0.f);
        w1y += (e1.y + h1.y) + (up1 ? v1y : 0.f);
        w1z += (e1.z + h1.z) + (up1 ? v1z : 0.f);
    }
}

// ------------------------------------------------------------------ launchers

// Mesh, box, species, rho0, kT, 1/kappa and chi of a parameter block:
// HPF_OK or HPF_ERR_INVALID.
hpf_status validate_field_params(const hpf_params* p);

void launch_stage_state(const float* pos, const float* vel, const int32_t* type, int n, int S,
                        StateBuf st, uint32_t* meta, int* err, cudaStream_t s);
void launch_mark_bonds(const int32_t* bonds, long long nb, int n, uint32_t* meta, int* err,
                       cudaStream_t s);
void launch_scatter(StateBuf st, const uint32_t* meta, int n, MeshGeom g,
                    unsigned long long* D, cudaStream_t s);
void launch_field(const long long* D, MeshGeom g, const FieldCoef& coef, float4* G,
                  unsigned long long* D_clear, cudaStream_t s);
void launch_unpad_field(const float4* G, MeshGeom g, int S, float4* out, cudaStream_t s);
void launch_forces(StateBuf st, const uint32_t* meta, int n, MeshGeom g, const float4* G,
                   StepConsts c, int which, float* F_tag, cudaStream_t s);
void launch_step(StateBuf in, StateBuf out, const uint32_t* meta, int n, int n_sub,
                 long long step0, MeshGeom g, const float4* G, StepConsts c,
                 unsigned long long* D_next, int* flag, cudaStream_t s);
void launch_energy(StateBuf st, const uint32_t* meta, int n, MeshGeom g, const float4* G,
                   StepConsts c, long long step, const long long* D, const EnergyConsts& e,
                   double* partials, double* out6, cudaStream_t s);
void launch_order(const uint32_t* meta, int n, int32_t* order, cudaStream_t s);
void launch_advance_counter(long long* step, long long by, cudaStream_t s);
void launch_set_counter(long long* step, long long v, cudaStream_t s);
void launch_unpermute(StateBuf st, const uint32_t* meta, int n, float* pos_tag, float* vel_tag,
                      int* flag, cudaStream_t s);
void launch_repermute(const float* pos_tag, const float* vel_tag, const uint32_t* meta, int n,
                      StateBuf st, const MeshGeom& g, unsigned long long* D, int* flag,
                      cudaStream_t s);

long long sort_key_space(const MeshGeom& g);
long long scan_scratch_words(long long L);
int scan_exclusive(const uint32_t* in, uint32_t* out, long long L, uint32_t* scratch,
                   cudaStream_t s);
int launch_chain_build_heads(const uint32_t* meta, int n, uint32_t* hd, uint32_t* scratch,
                             cudaStream_t s);
int launch_chain_build(const uint32_t* meta, const uint32_t* hx, int n, int C, int* cstart,
                       uint32_t* tag0, int* chain_of, int* clen, int* max_len, cudaStream_t s);
int launch_sort(const SortBufs& b, StateBuf in, StateBuf out, const uint32_t* meta_in,
                uint32_t* meta_out, int n, int C, MeshGeom g, cudaStream_t s);

int step_halo_max();
void launch_step_warp_batch(const BatchStepParams& p, int max_seg_total, int therm,
                            cudaStream_t s);
// A single context's launch that also writes the observables' bead partials
// of its final state (kBeadVals float-float pairs per CTA); returns the CTA
// count.  Bonds only, force_mode 0, therm 0 or 1.
int launch_step_warp_obs(const SingleStepParams& p, int max_seg, int therm, float2* part,
                         float half_dt_m, const BondFF& bond, cudaStream_t s);
int step_warp_grid_cap();  // CTAs of the persistent step grid on this device
void launch_step_warp_single(const SingleStepParams& p, int max_seg, int therm, cudaStream_t s);
// A learned window: the field (1 - j/K) G + j/K G2 at window step j (j0 at the
// launch's first sub-step, inv_k = 1/K); a single context, force_mode 0.
void launch_step_warp_lerp(const SingleStepParams& p, const float4* G2, int j0, float inv_k,
                           int max_seg, int therm, cudaStream_t s);
void launch_field_batch(const BatchFieldParams& p, int S, cudaStream_t s);
int field_tile_candidates();
bool field_tile_is_plain(int id);
void field_tile_shape(int id, int out[3]);
void launch_field_tiled(const TiledFieldParams& p, int S, int tile, cudaStream_t s);
void launch_wait_selftest(int* flag, cudaStream_t s);
void launch_field_tiled(const SingleFieldParams& p, int S, int tile, cudaStream_t s);
// cuTensorMapEncodeTiled through the runtime's driver entry point: unit element
// strides, no interleave, no swizzle, 128-byte L2 promotion, zero fill out of
// range.  False when the entry point is missing or the encoding is refused.
bool encode_tiled_map(CUtensorMap* map, CUtensorMapDataType type, int rank, void* base,
                      const cuuint64_t* dims, const cuuint64_t* strides, const cuuint32_t* box);
bool make_mesh_tensor_map(CUtensorMap* map, const long long* D, const MeshGeom& g, int S,
                          int tile);
void tile_grid(const MeshGeom& g, int tile, int* tiles_x, int* tiles_y, int* blocks);
int energy_partials_needed(int n, int nodes, int S);
int energy_launches(int n, int S);  // kernels launch_energy issues
void launch_energy_nodes_only(int n, MeshGeom g, const long long* D, const EnergyConsts& e,
                              const float2* bead_part, int nb_bead, double* partials,
                              double* out6, cudaStream_t s);

// learned density propagator (the network lives in k_prop.cu)
bool prop_mesh_is(const hpf_prop* p, const MeshGeom& g);
// flag: device status word for a tensor-core wait that gives up (kFlagTimeout)
void prop_predict(hpf_prop* p, const float* x, float* dphi, cudaStream_t s, int* flag);
void launch_mesh_to_phi(const unsigned long long* D, long long n, double phi_c, float* phi,
                        cudaStream_t s);
void launch_smooth_phi(const float* in, float* out, float* tmp, int mx, int my, int mz, int C,
                       int passes, cudaStream_t s);
void launch_mesh_predict(const unsigned long long* D_base, const float* dphi, long long n,
                         double frac_over_phi_c, unsigned long long* D_out, cudaStream_t s);
// acc[0] = sum (Fa - Fb)^2, acc[1] = sum Fb^2 over n floats, deterministic;
// acc holds 2 + 2 force_error_partials() doubles (the tail is scratch)
void launch_force_error(const float* Fa, const float* Fb, long long n, double* acc,
                        cudaStream_t s);
int force_error_partials();

}  // namespace hpf
