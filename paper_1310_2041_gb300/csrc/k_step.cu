// k_step.cu -- field gather, bonds, Langevin velocity-Verlet (the fused field-period kernels).
#include "hpf_internal.cuh"

namespace hpf {

constexpr int kStepBlock = 512;
constexpr int kHaloMax = 16;  // most steps fused into one launch

int step_halo_max() { return kHaloMax; }

// ------------------------------------------------------------------ A4 + A5 forces
//
// Conservative force at the current positions, written in tag order.
__global__ void __launch_bounds__(256) k_forces(StateBuf st, const uint32_t* __restrict__ meta,
                                                int n, MeshGeom g, const float4* __restrict__ G,
                                                StepConsts c, int which,
                                                float* __restrict__ F_tag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = st.x[i], y = st.y[i], z = st.z[i];
    const uint32_t m = meta[i];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (which & HPF_FORCE_BOND) {
        if (m & kBondPrev)
            bond_force(x - st.x[i - 1], y - st.y[i - 1], z - st.z[i - 1], c.two_k, c.r0, fx, fy, fz);
        if (m & kBondNext)
            bond_force(x - st.x[i + 1], y - st.y[i + 1], z - st.z[i + 1], c.two_k, c.r0, fx, fy, fz);
        if (c.two_ka != 0.f) angle_forces_of(st, meta, i, m, c, fx, fy, fz);
        if (c.kd != 0.f) {
            int back, fwd;
            chain_reach(meta, i, m, back, fwd);
            dihedral_forces_of([&](int d) { return make_float3(st.x[i + d], st.y[i + d], st.z[i + d]); },
                               back, fwd, c, fx, fy, fz);
        }
    }
    if (which & HPF_FORCE_FIELD) {
        const int T = (m >> kTypeShift) & kTypeMask;
        gather_field_mode(G + (size_t)T * g.gnodes, g, c.force_mode, x, y, z, fx, fy, fz);
    }
    const uint32_t tag = m & kTagMask;
    F_tag[3 * tag] = fx;
    F_tag[3 * tag + 1] = fy;
    F_tag[3 * tag + 2] = fz;
}

void launch_forces(StateBuf st, const uint32_t* meta, int n, MeshGeom g, const float4* G,
                   StepConsts c, int which, float* F_tag, cudaStream_t s) {
    if (n <= 0) return;
    k_forces<<<(n + 255) / 256, 256, 0, s>>>(st, meta, n, g, G, c, which, F_tag);
}

// ------------------------------------------------------------------ A6 fused steps
//
// One CTA advances a window of kStepBlock consecutive beads (whole chains or
// not) by n_sub steps without leaving the chip: positions live in registers,
// bonded neighbours are exchanged through shared memory, and the frozen field
// is sampled through a per-bead cache.  A bead's update after k steps depends
// on beads up to k places away along its chain, so the outer `halo` beads on
// each side are recomputed redundantly (bit-identically, the noise is keyed by
// tag and step) and only the inner kStepBlock - 2 halo beads are written back.
//
// Field cache: inside one cell the interpolated gradient is the trilinear
// polynomial c0 + c1 fx + c2 fy + c3 fz + c4 fx fy + c5 fx fz + c6 fy fz
// + c7 fx fy fz of the cell offset f (per component).  A bead keeps the 24
// coefficients of its current cell in shared memory (six float4 planes, one
// slot per thread, conflict-free) and rebuilds them from the eight corners
// only when it enters another cell -- about once every 40 steps at kT = 1,
// h = 1, dt = 0.01 -- so most sub-steps read six shared float4s instead of
// gathering eight corners from L1/L2.
constexpr int kCachePlanes = 6;
constexpr size_t kStepSmem = sizeof(float4) * kCachePlanes * kStepBlock +
                             sizeof(float) * 3 * 2 * kStepBlock;

// Ghosted-array index of the lower corner of cell (flx, fly, flz) (periodic
// image; see axis_gather for why no fix-up is needed).
__device__ __forceinline__ int cell_base(const MeshGeom& g, float flx, float fly, float flz) {
    const float fmx = (float)g.mx, fmy = (float)g.my, fmz = (float)g.mz;
    float wx = __fmaf_rn(-fmx, floorf((flx + 0.5f) * g.inv_m[0]), flx);
    float wy = __fmaf_rn(-fmy, floorf((fly + 0.5f) * g.inv_m[1]), fly);
    float wz = __fmaf_rn(-fmz, floorf((flz + 0.5f) * g.inv_m[2]), flz);
    wx = fminf(fmaxf(wx, 0.0f), fmx - 1.0f);
    wy = fminf(fmaxf(wy, 0.0f), fmy - 1.0f);
    wz = fminf(fmaxf(wz, 0.0f), fmz - 1.0f);
    return (int)wz * g.gxy + (int)wy * g.gx + (int)wx;
}

// The eight corners (x, y, z offsets in {0, 1}) of cell (flx, fly, flz).
struct Corners {
    float4 g000, g100, g010, g110, g001, g101, g011, g111;
};

__device__ __forceinline__ Corners load_corners(const float4* __restrict__ Gt, const MeshGeom& g,
                                                float flx, float fly, float flz) {
    const int o00 = cell_base(g, flx, fly, flz);
    const int o01 = o00 + g.gx, o10 = o00 + g.gxy, o11 = o10 + g.gx;
    Corners k;
    k.g000 = __ldg(Gt + o00);
    k.g100 = __ldg(Gt + o00 + 1);
    k.g010 = __ldg(Gt + o01);
    k.g110 = __ldg(Gt + o01 + 1);
    k.g001 = __ldg(Gt + o10);
    k.g101 = __ldg(Gt + o10 + 1);
    k.g011 = __ldg(Gt + o11);
    k.g111 = __ldg(Gt + o11 + 1);
    return k;
}

// The cell polynomial's coefficients from its corners into cache slot t
// (component-major: planes 2j, 2j + 1 hold c0..c7 of component j; kForce 1:
// planes 0 and 1 hold the polynomial of V).
template <int kForce>
__device__ __forceinline__ void store_cell_coefs(const Corners& k, float4* __restrict__ cache, int t,
                                                 int stride) {
#define HPF_COEF(comp, j)                                                                        \
    {                                                                                            \
        const float a0 = k.g000.comp, a1 = k.g100.comp - k.g000.comp;                            \
        const float a2 = k.g010.comp - k.g000.comp, a3 = k.g001.comp - k.g000.comp;              \
        const float a4 = (k.g110.comp - k.g100.comp) - a2;                                       \
        const float a5 = (k.g101.comp - k.g100.comp) - a3;                                       \
        const float a6 = (k.g011.comp - k.g010.comp) - a3;                                       \
        const float a7 = ((k.g111.comp - k.g110.comp) - (k.g101.comp - k.g100.comp)) - a6;       \
        cache[(2 * j) * stride + t] = make_float4(a0, a1, a2, a3);                               \
        cache[(2 * j + 1) * stride + t] = make_float4(a4, a5, a6, a7);                           \
    }
    if (kForce == 1) {
        HPF_COEF(w, 0)
    } else {
        HPF_COEF(x, 0)
        HPF_COEF(y, 1)
        HPF_COEF(z, 2)
    }
#undef HPF_COEF
}

// kForce 1: planes 0 and 1 hold the trilinear polynomial of V instead (the
// exact-energy-gradient force differentiates it).  kForce 2: the key is the
// nearest vertex and planes 0 and 1 hold its six staggered coefficients.
template <int kForce>
__device__ __forceinline__ void fill_cell_cache(const float4* __restrict__ Gt, const MeshGeom& g,
                                                float flx, float fly, float flz,
                                                float4* __restrict__ cache, int t,
                                                int stride = kStepBlock) {
    if (kForce == 2) {
        float c[6];
        stag_vertex_coefs(Gt, g, flx, fly, flz, c);
        cache[t] = make_float4(c[0], c[1], c[2], c[3]);
        cache[stride + t] = make_float4(c[4], c[5], 0.f, 0.f);
        return;
    }
    store_cell_coefs<kForce>(load_corners(Gt, g, flx, fly, flz), cache, t, stride);
}

// The cache key of a mesh coordinate: its cell (floor), or its nearest
// vertex for the staggered force.
template <int kForce>
__device__ __forceinline__ float cache_key(float s) {
    return kForce == 2 ? stag_vertex(s) : floorf(s);
}

// -(trilinear polynomial) of the cached cell at offset (fx, fy, fz).
__device__ __forceinline__ float cell_poly(const float4 lo, const float4 hi, float fx, float fy,
                                           float fz) {
    // lo = (c0, c1, c2, c3), hi = (c4, c5, c6, c7)
    float a = fmaf(fz, hi.w, hi.x);
    a = fmaf(fy, a, lo.y);
    a = fmaf(fz, hi.y, a);
    const float b = fmaf(fz, hi.z, lo.z);
    float v = fmaf(fx, a, lo.x);
    v = fmaf(fy, b, v);
    return fmaf(fz, lo.w, v);
}

template <int kForce>
__device__ __forceinline__ void eval_cell_cache(const float4* __restrict__ cache, int t, float fx,
                                                float fy, float fz, float& Fx, float& Fy,
                                                float& Fz, const MeshGeom& g,
                                                int stride = kStepBlock) {
    if (kForce == 2) {
        const float4 lo = cache[t], hi = cache[stride + t];
        const float c[6] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y};
        stag_force(c, fx, fy, fz, g, Fx, Fy, Fz);
    } else if (kForce == 1) {
        // V = a0 + a1 fx + a2 fy + a3 fz + a4 fx fy + a5 fx fz + a6 fy fz + a7 fx fy fz;
        // F = -(1/h) dV/df per axis
        const float4 lo = cache[t], hi = cache[stride + t];
        const float dx = fmaf(fz, fmaf(fy, hi.w, hi.y), fmaf(fy, hi.x, lo.y));
        const float dy = fmaf(fz, fmaf(fx, hi.w, hi.z), fmaf(fx, hi.x, lo.z));
        const float dz = fmaf(fy, fmaf(fx, hi.w, hi.z), fmaf(fx, hi.y, lo.w));
        Fx = fmaf(-g.inv_h[0], dx, Fx);
        Fy = fmaf(-g.inv_h[1], dy, Fy);
        Fz = fmaf(-g.inv_h[2], dz, Fz);
    } else {
        Fx -= cell_poly(cache[0 * stride + t], cache[1 * stride + t], fx, fy, fz);
        Fy -= cell_poly(cache[2 * stride + t], cache[3 * stride + t], fx, fy, fz);
        Fz -= cell_poly(cache[4 * stride + t], cache[5 * stride + t], fx, fy, fz);
    }
}

// A warp reads shared positions of its own lanes and of the edge lanes of the
// two adjacent warps only, so each sub-step synchronises adjacent warp pairs
// (named barrier w + 1 joins warps w and w + 1) instead of the whole CTA.
// Every warp waits on its left pair first, then its right pair, so the waits
// form no cycle.  With two position buffers a warp can run at most one
// sub-step ahead of a neighbour, which has by then finished reading the buffer
// it is about to overwrite.
static_assert(kStepBlock / 32 <= 16, "named barriers 1..15 cover at most 16 warps");
__device__ __forceinline__ void neighbour_sync(int w) {
    constexpr int kWarps = kStepBlock / 32;
    if (w > 0) asm volatile("bar.sync %0, 64;" ::"r"(w) : "memory");
    if (w + 1 < kWarps) asm volatile("bar.sync %0, 64;" ::"r"(w + 1) : "memory");
}

template <int kTherm, int kForce, int kBonded>
__global__ void __launch_bounds__(kStepBlock, 2) k_step(StateBuf in, StateBuf out,
                                                        const uint32_t* __restrict__ meta, int n,
                                                        int halo, int n_sub, long long step0,
                                                        MeshGeom g, const float4* __restrict__ G,
                                                        StepConsts c,
                                                        unsigned long long* __restrict__ D_next,
                                                        int* __restrict__ flag) {
    extern __shared__ float4 smem4[];
    float4* cache = smem4;                                   // [kCachePlanes][kStepBlock]
    float* sx = reinterpret_cast<float*>(smem4 + kCachePlanes * kStepBlock);  // [2][block]
    float* sy = sx + 2 * kStepBlock;
    float* sz = sy + 2 * kStepBlock;
    const int t = threadIdx.x;
    const int payload = kStepBlock - 2 * halo;
    const long long i = (long long)blockIdx.x * payload - halo + t;
    const bool live = (i >= 0 && i < n);
    float x = 0.f, y = 0.f, z = 0.f, vx = 0.f, vy = 0.f, vz = 0.f;
    uint32_t m = 0;
    if (live) {
        x = in.x[i];
        y = in.y[i];
        z = in.z[i];
        vx = in.vx[i];
        vy = in.vy[i];
        vz = in.vz[i];
        m = meta[i];
    }
    // out-of-range threads only fill their shared-memory slot
    const bool has_prev = live && (m & kBondPrev) && t > 0;
    const bool has_next = live && (m & kBondNext) && t + 1 < kStepBlock;
    // bond flags of the whole window, for the angles centred at the neighbours
    // and the dihedrals through them
    __shared__ unsigned char s_bonds[kStepBlock];
    int back = 0, fwd = 0;  // consecutive bonds backwards / forwards inside the window (<= 3)
    if (kBonded >= 1) {
        s_bonds[t] = (unsigned char)((has_prev ? 1 : 0) | (has_next ? 2 : 0));
        __syncthreads();
    }
    if (kBonded == 2) {
        if (has_prev) {
            back = 1;
            if (s_bonds[t - 1] & 1) {
                back = 2;
                if (s_bonds[t - 2] & 1) back = 3;
            }
        }
        if (has_next) {
            fwd = 1;
            if (s_bonds[t + 1] & 2) {
                fwd = 2;
                if (s_bonds[t + 2] & 2) fwd = 3;
            }
        }
    }
    const uint32_t tag = m & kTagMask;
    const float4* __restrict__ Gt = G + (size_t)((m >> kTypeShift) & kTypeMask) * g.gnodes;
    float cfx = __int_as_float(0x7fc00000), cfy = cfx, cfz = cfx;  // cached cell: none
    for (int k = 0; k < n_sub; ++k) {
        const int b = k & 1;
        sx[b * kStepBlock + t] = x;
        sy[b * kStepBlock + t] = y;
        sz[b * kStepBlock + t] = z;
        neighbour_sync(t >> 5);
        const float s0 = __fmul_rn(x, g.inv_h[0]), s1 = __fmul_rn(y, g.inv_h[1]),
                    s2 = __fmul_rn(z, g.inv_h[2]);
        const float flx = cache_key<kForce>(s0), fly = cache_key<kForce>(s1),
                    flz = cache_key<kForce>(s2);
        if (flx != cfx || fly != cfy || flz != cfz) {
            fill_cell_cache<kForce>(Gt, g, flx, fly, flz, cache, t);
            cfx = flx;
            cfy = fly;
            cfz = flz;
        }
        float fx = -c.fric * vx, fy = -c.fric * vy, fz = -c.fric * vz;
        eval_cell_cache<kForce>(cache, t, __fsub_rn(s0, flx), __fsub_rn(s1, fly),
                                __fsub_rn(s2, flz), fx, fy, fz, g);
        if (kTherm == 1) {
            float nx, ny, nz;
            gauss3(c, tag, step0 + k, nx, ny, nz);
            fx = fmaf(c.sigma, nx, fx);
            fy = fmaf(c.sigma, ny, fy);
            fz = fmaf(c.sigma, nz, fz);
        }
        const int tp = has_prev ? t - 1 : t, tn = has_next ? t + 1 : t;
        bond_force(x - sx[b * kStepBlock + tp], y - sy[b * kStepBlock + tp],
                   z - sz[b * kStepBlock + tp], has_prev ? c.two_k : 0.0f, c.r0, fx, fy, fz);
        bond_force(x - sx[b * kStepBlock + tn], y - sy[b * kStepBlock + tn],
                   z - sz[b * kStepBlock + tn], has_next ? c.two_k : 0.0f, c.r0, fx, fy, fz);
        if (kBonded >= 1) {
            // the three angles this bead belongs to: centred at t - 1, t and t + 1
            const int tp2 = (has_prev && t >= 2) ? t - 2 : t;
            const int tn2 = (has_next && t + 2 < kStepBlock) ? t + 2 : t;
            const bool left = has_prev && t >= 2 && (s_bonds[t - 1] & 1);
            const bool right = has_next && t + 2 < kStepBlock && (s_bonds[t + 1] & 2);
            const float xp = sx[b * kStepBlock + tp], yp = sy[b * kStepBlock + tp],
                        zp = sz[b * kStepBlock + tp];
            const float xn = sx[b * kStepBlock + tn], yn = sy[b * kStepBlock + tn],
                        zn = sz[b * kStepBlock + tn];
            float ax, ay, az, bx, by, bz;
            // centred at t: this bead takes minus both end shares
            angle_force(xp - x, yp - y, zp - z, xn - x, yn - y, zn - z,
                        (has_prev && has_next) ? c.two_ka : 0.0f, c, ax, ay, az, bx, by,
                        bz);
            fx -= ax + bx;
            fy -= ay + by;
            fz -= az + bz;
            // centred at t - 1 (ends t - 2 and t): this bead is end b
            angle_force(sx[b * kStepBlock + tp2] - xp, sy[b * kStepBlock + tp2] - yp,
                        sz[b * kStepBlock + tp2] - zp, x - xp, y - yp, z - zp,
                        left ? c.two_ka : 0.0f, c, ax, ay, az, bx, by, bz);
            fx += bx;
            fy += by;
            fz += bz;
            // centred at t + 1 (ends t and t + 2): this bead is end a
            angle_force(x - xn, y - yn, z - zn, sx[b * kStepBlock + tn2] - xn,
                        sy[b * kStepBlock + tn2] - yn, sz[b * kStepBlock + tn2] - zn,
                        right ? c.two_ka : 0.0f, c, ax, ay, az, bx, by, bz);
            fx += ax;
            fy += ay;
            fz += az;
        }
        if (kBonded == 2) {
            const int o = b * kStepBlock + t;
            dihedral_forces_of(
                [&](int d) { return make_float3(sx[o + d], sy[o + d], sz[o + d]); }, back, fwd, c,
                fx, fy, fz);
        }
        if (kTherm == 2 && andersen_collides(c, tag, step0 + k)) {
            // the on-step velocity redrawn, then the second half kick
            float nx, ny, nz;
            gauss3(c, tag, step0 + k, nx, ny, nz);
            const float h = 0.5f * c.dt_m;
            vx = fmaf(h, fx, c.sig_v * nx);
            vy = fmaf(h, fy, c.sig_v * ny);
            vz = fmaf(h, fz, c.sig_v * nz);
        } else {
            vx = fmaf(c.dt_m, fx, vx);
            vy = fmaf(c.dt_m, fy, vy);
            vz = fmaf(c.dt_m, fz, vz);
        }
        x = fmaf(c.dt, vx, x);
        y = fmaf(c.dt, vy, y);
        z = fmaf(c.dt, vz, z);
    }
    if (live && t >= halo && t < kStepBlock - halo) {
        out.x[i] = x;
        out.y[i] = y;
        out.z[i] = z;
        out.vx[i] = vx;
        out.vy[i] = vy;
        out.vz[i] = vz;
        const bool finite = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) &&
                            isfinite(vy) && isfinite(vz);
        if (!finite) atomicOr(flag, kFlagNonFinite);
        else if (!(coord_in_range(x, g.inv_h[0]) && coord_in_range(y, g.inv_h[1]) &&
                   coord_in_range(z, g.inv_h[2])))
            atomicOr(flag, kFlagRange);
        if (D_next) {
            // this launch ends on a refresh step: deposit the final positions
            const AxisCoord ax = axis_coord(x, g.inv_h[0], g.mx, g.inv_m[0]);
            const AxisCoord ay = axis_coord(y, g.inv_h[1], g.my, g.inv_m[1]);
            const AxisCoord az = axis_coord(z, g.inv_h[2], g.mz, g.inv_m[2]);
            scatter_bead(D_next + (size_t)((m >> kTypeShift) & kTypeMask) * g.nodes, g, ax, ay,
                         az);
        }
    }
}

template <int kTherm, int kForce, int kBonded>
static void launch_step_t(StateBuf in, StateBuf out, const uint32_t* meta, int n, int n_sub,
                          long long step0, MeshGeom g, const float4* G, StepConsts c,
                          unsigned long long* D_next, int* flag, cudaStream_t s) {
    static std::once_flag attr[64];
    once_per_device(attr, [] {
        cudaFuncSetAttribute(k_step<kTherm, kForce, kBonded>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStepSmem);
    });
    // a bead's update after k sub-steps depends on beads up to k (bonds), 2k
    // (angles) or 3k (dihedrals) places away along its chain
    const int halo = (kBonded + 1) * n_sub;
    const int payload = kStepBlock - 2 * halo;
    const int blocks = (n + payload - 1) / payload;
    k_step<kTherm, kForce, kBonded><<<blocks, kStepBlock, kStepSmem, s>>>(
        in, out, meta, n, halo, n_sub, step0, g, G, c, D_next, flag);
}

template <int kTherm, int kForce>
static void launch_step_a(StateBuf in, StateBuf out, const uint32_t* meta, int n, int n_sub,
                          long long step0, MeshGeom g, const float4* G, StepConsts c,
                          unsigned long long* D_next, int* flag, cudaStream_t s) {
    const int bonded = bonded_level(c);
    if (bonded == 2)
        launch_step_t<kTherm, kForce, 2>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);
    else if (bonded == 1)
        launch_step_t<kTherm, kForce, 1>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);
    else
        launch_step_t<kTherm, kForce, 0>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);
}

void launch_step(StateBuf in, StateBuf out, const uint32_t* meta, int n, int n_sub,
                 long long step0, MeshGeom g, const float4* G, StepConsts c,
                 unsigned long long* D_next, int* flag, cudaStream_t s) {
    if (n <= 0 || n_sub <= 0) return;
    const int therm = step_thermostat(c);
#define HPF_HALO(T)                                                                        \
    if (c.force_mode == 2)                                                                   \
        launch_step_a<T, 2>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);       \
    else if (c.force_mode == 1)                                                              \
        launch_step_a<T, 1>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);       \
    else                                                                                     \
        launch_step_a<T, 0>(in, out, meta, n, n_sub, step0, g, G, c, D_next, flag, s);
    if (therm == 1) {
        HPF_HALO(1)
    } else if (therm == 2) {
        HPF_HALO(2)
    } else {
        HPF_HALO(0)
    }
#undef HPF_HALO
}

// ------------------------------------------------------------------ A6, warp form
//
// When every chain has at most 64 beads the sort also packs consecutive whole
// chains into segments of at most 64 beads, and one warp advances one segment
// for all n_sub steps on its own: lane l holds beads 2l and 2l + 1, so a
// bead's chain neighbours are either its partner in the same lane or the
// neighbouring lane's bead, exchanged with register shuffles.  No halo, no
// shared positions and no barrier: warps never wait for one another.  The
// field is sampled through the same per-bead cell cache as above (two slots
// per thread).  A persistent grid walks the segment list, whose length is
// read on the device so a re-sort needs no host synchronisation.
constexpr int kWarpBlock = 256;
constexpr size_t kWarpSmem = sizeof(float4) * kCachePlanes * 2 * kWarpBlock;

struct Bead {
    float x, y, z, vx, vy, vz;
    uint32_t m;
    float cfx, cfy, cfz;  // cached cell (floor of the mesh coordinate), NaN: none
};

// The bead's cell: refill its cache of the cell polynomial when the bead
// has entered another cell; returns the offsets inside the cell.
template <int kForce, int kLerp = 0>
__device__ __forceinline__ void cell_check(Bead& b, const float4* __restrict__ G, const MeshGeom& g,
                                           float4* __restrict__ cache, int slot, float& f0,
                                           float& f1, float& f2,
                                           const float4* __restrict__ G2 = nullptr) {
    const float s0 = __fmul_rn(b.x, g.inv_h[0]), s1 = __fmul_rn(b.y, g.inv_h[1]),
                s2 = __fmul_rn(b.z, g.inv_h[2]);
    const float flx = cache_key<kForce>(s0), fly = cache_key<kForce>(s1),
                flz = cache_key<kForce>(s2);
    if (flx != b.cfx || fly != b.cfy || flz != b.cfz) {
        const size_t off = (size_t)((b.m >> kTypeShift) & kTypeMask) * g.gnodes;
        if (kLerp) {
            // the window's second field: its polynomial in planes 6..11
            store_cell_coefs<0>(load_corners(G2 + off, g, flx, fly, flz),
                                cache + kCachePlanes * 2 * kWarpBlock, slot, 2 * kWarpBlock);
        }
        fill_cell_cache<kForce>(G + off, g, flx,
                                fly, flz, cache, slot, 2 * kWarpBlock);
        b.cfx = flx;
        b.cfy = fly;
        b.cfz = flz;
    }
    f0 = __fsub_rn(s0, flx);
    f1 = __fsub_rn(s1, fly);
    f2 = __fsub_rn(s2, flz);
}

// Force on one bead: field (cached cell polynomial at offsets f), friction,
// noise (nx, ny, nz) and the bond force (bx, by, bz) already summed over its
// chain neighbours.
template <int kTherm, int kForce, int kLerp = 0>
__device__ __forceinline__ void bead_force(const Bead& b, float f0, float f1, float f2, float nx,
                                           float ny, float nz, float bx, float by, float bz,
                                           const StepConsts& c, const MeshGeom& g,
                                           const float4* __restrict__ cache, int slot, float a,
                                           float& fx, float& fy, float& fz) {
    fx = -c.fric * b.vx;
    fy = -c.fric * b.vy;
    fz = -c.fric * b.vz;
    if (kLerp) {
        // the field (1 - a) G0 + a G2: P0 + a (P2 - P0) of the two cached polynomials
        constexpr int st = 2 * kWarpBlock;
        const float4* c2 = cache + kCachePlanes * st;
        const float p0x = cell_poly(cache[0 * st + slot], cache[1 * st + slot], f0, f1, f2);
        const float p0y = cell_poly(cache[2 * st + slot], cache[3 * st + slot], f0, f1, f2);
        const float p0z = cell_poly(cache[4 * st + slot], cache[5 * st + slot], f0, f1, f2);
        const float p2x = cell_poly(c2[0 * st + slot], c2[1 * st + slot], f0, f1, f2);
        const float p2y = cell_poly(c2[2 * st + slot], c2[3 * st + slot], f0, f1, f2);
        const float p2z = cell_poly(c2[4 * st + slot], c2[5 * st + slot], f0, f1, f2);
        fx -= fmaf(a, p2x - p0x, p0x);
        fy -= fmaf(a, p2y - p0y, p0y);
        fz -= fmaf(a, p2z - p0z, p0z);
    } else {
        eval_cell_cache<kForce>(cache, slot, f0, f1, f2, fx, fy, fz, g, 2 * kWarpBlock);
    }
    if (kTherm == 1) {
        fx = fmaf(c.sigma, nx, fx);
        fy = fmaf(c.sigma, ny, fy);
        fz = fmaf(c.sigma, nz, fz);
    }
    fx += bx;
    fy += by;
    fz += bz;
}

// Kick of one bead by that force.  Andersen (kTherm 2): a colliding bead's
// on-step velocity is sqrt(kT/m) (nx, ny, nz) before the second half kick.
template <int kTherm, int kForce, int kLerp = 0>
__device__ __forceinline__ void kick_bead(Bead& b, float f0, float f1, float f2, float nx,
                                          float ny, float nz, float bx, float by, float bz,
                                          const StepConsts& c, const MeshGeom& g,
                                          const float4* __restrict__ cache, int slot,
                                          bool coll, float a = 0.f) {
    float fx, fy, fz;
    bead_force<kTherm, kForce, kLerp>(b, f0, f1, f2, nx, ny, nz, bx, by, bz, c, g, cache, slot, a,
                                      fx, fy, fz);
    if (kTherm == 2 && coll) {
        const float h = 0.5f * c.dt_m;
        b.vx = fmaf(h, fx, c.sig_v * nx);
        b.vy = fmaf(h, fy, c.sig_v * ny);
        b.vz = fmaf(h, fz, c.sig_v * nz);
    } else {
        b.vx = fmaf(c.dt_m, fx, b.vx);
        b.vy = fmaf(c.dt_m, fy, b.vy);
        b.vz = fmaf(c.dt_m, fz, b.vz);
    }
}

__device__ __forceinline__ void finish_bead(const Bead& b, long long i, StateBuf out,
                                            const MeshGeom& g, unsigned long long* D_next,
                                            int* flag) {
    out.x[i] = b.x;
    out.y[i] = b.y;
    out.z[i] = b.z;
    out.vx[i] = b.vx;
    out.vy[i] = b.vy;
    out.vz[i] = b.vz;
    const bool finite = isfinite(b.x) && isfinite(b.y) && isfinite(b.z) && isfinite(b.vx) &&
                        isfinite(b.vy) && isfinite(b.vz);
    if (!finite) atomicOr(flag, kFlagNonFinite);
    else if (!(coord_in_range(b.x, g.inv_h[0]) && coord_in_range(b.y, g.inv_h[1]) &&
               coord_in_range(b.z, g.inv_h[2])))
        atomicOr(flag, kFlagRange);
    if (D_next) {
        const AxisCoord ax = axis_coord(b.x, g.inv_h[0], g.mx, g.inv_m[0]);
        const AxisCoord ay = axis_coord(b.y, g.inv_h[1], g.my, g.inv_m[1]);
        const AxisCoord az = axis_coord(b.z, g.inv_h[2], g.mz, g.inv_m[2]);
        scatter_bead(D_next + (size_t)((b.m >> kTypeShift) & kTypeMask) * g.nodes, g, ax, ay, az);
    }
}

// The observables' bead terms of a segment's final state (what the next
// sub-step's force evaluation would form, never applied): F_n at the final
// positions with step `step`'s noise, the on-step velocity
// v_n = v + dt/(2m) F_n, |v_n|^2 and v_n added to the thread's float-float
// sums, and the energy of each bond once (the bond to the next bead: b0's to
// b1, b1's to the next lane's b0).  Bonds only, interpolated-gradient force,
// no Andersen redraw.
struct ObsArgs {
    float2* part;     // [gridDim.x][kBeadVals] float-float block partials
    float half_dt_m;  // dt / (2m)
    BondFF bond;
};

template <int kTherm>
__device__ __forceinline__ void observe_segment(Bead& b0, Bead& b1, bool a0, bool a1, bool p0,
                                                bool n0, bool n1, long long step,
                                                const MeshGeom& g, const float4* __restrict__ G,
                                                const StepConsts& c, float4* wcache, int tid,
                                                const ObsArgs& o, FF* acc) {
    const int lane = tid & 31;
    float w0x, w0y, w0z, w1x, w1y, w1z;
    warp_bonded_forces<0>(b0.x, b0.y, b0.z, b1.x, b1.y, b1.z, p0, n0, n1, c, lane, w0x, w0y, w0z,
                          w1x, w1y, w1z);
    float f00, f01, f02, f10, f11, f12;
    cell_check<0>(b0, G, g, wcache, tid, f00, f01, f02);
    cell_check<0>(b1, G, g, wcache, kWarpBlock + tid, f10, f11, f12);
    float g0x = 0.f, g0y = 0.f, g0z = 0.f, g1x = 0.f, g1y = 0.f, g1z = 0.f;
    if (kTherm == 1) {
        gauss3(c, b0.m & kTagMask, step, g0x, g0y, g0z);
        gauss3(c, b1.m & kTagMask, step, g1x, g1y, g1z);
    }
    float F0x, F0y, F0z, F1x, F1y, F1z;
    bead_force<kTherm, 0>(b0, f00, f01, f02, g0x, g0y, g0z, w0x, w0y, w0z, c, g, wcache, tid, 0.f,
                          F0x, F0y, F0z);
    bead_force<kTherm, 0>(b1, f10, f11, f12, g1x, g1y, g1z, w1x, w1y, w1z, c, g, wcache,
                          kWarpBlock + tid, 0.f, F1x, F1y, F1z);
    // the next lane's first bead (every lane takes part in the shuffles)
    const float qx = __shfl_down_sync(0xffffffffu, b0.x, 1);
    const float qy = __shfl_down_sync(0xffffffffu, b0.y, 1);
    const float qz = __shfl_down_sync(0xffffffffu, b0.z, 1);
    float uh = acc[1].h, ul = acc[1].l;
    if (n0) bond_energy_ff(b0.x, b0.y, b0.z, b1.x, b1.y, b1.z, o.bond, uh, ul);
    if (n1) bond_energy_ff(b1.x, b1.y, b1.z, qx, qy, qz, o.bond, uh, ul);
    acc[1] = FF{uh, ul};
    const float hf = o.half_dt_m;
    if (a0) {
        const float ux = fmaf(hf, F0x, b0.vx), uy = fmaf(hf, F0y, b0.vy), uz = fmaf(hf, F0z, b0.vz);
        acc[0] = ff_plus(acc[0], fmaf(ux, ux, fmaf(uy, uy, __fmul_rn(uz, uz))));
        acc[2] = ff_plus(acc[2], ux);
        acc[3] = ff_plus(acc[3], uy);
        acc[4] = ff_plus(acc[4], uz);
    }
    if (a1) {
        const float ux = fmaf(hf, F1x, b1.vx), uy = fmaf(hf, F1y, b1.vy), uz = fmaf(hf, F1z, b1.vz);
        acc[0] = ff_plus(acc[0], fmaf(ux, ux, fmaf(uy, uy, __fmul_rn(uz, uz))));
        acc[2] = ff_plus(acc[2], ux);
        acc[3] = ff_plus(acc[3], uy);
        acc[4] = ff_plus(acc[4], uz);
    }
}

// One warp advances one segment (whole chains, base .. base + cnt) by n_sub steps.
// kObs: also the observables' terms of the final state (observe_segment).
template <int kTherm, int kForce, int kBonded, int kLerp = 0, int kObs = 0>
__device__ __forceinline__ void advance_segment(const StateBuf& in, const StateBuf& out,
                                                const uint32_t* __restrict__ meta, int base,
                                                int cnt, int n_sub, long long step0,
                                                const MeshGeom& g, const float4* __restrict__ G,
                                                const StepConsts& c,
                                                unsigned long long* __restrict__ D_next,
                                                int* __restrict__ flag, float4* wcache, int tid,
                                                const float4* __restrict__ G2 = nullptr,
                                                int lerp_j0 = 0, float lerp_inv_k = 0.f,
                                                const ObsArgs* obs = nullptr,
                                                FF* obs_acc = nullptr) {
    const int lane = tid & 31;
    const float nan = __int_as_float(0x7fc00000);
    const int j0 = 2 * lane, j1 = j0 + 1;
    const bool a0 = j0 < cnt, a1 = j1 < cnt;
    Bead b0{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u, nan, nan, nan};
    Bead b1 = b0;
    if (a0) {
        const long long i = (long long)base + j0;
        b0.x = in.x[i]; b0.y = in.y[i]; b0.z = in.z[i];
        b0.vx = in.vx[i]; b0.vy = in.vy[i]; b0.vz = in.vz[i];
        b0.m = meta[i];
    }
    if (a1) {
        const long long i = (long long)base + j1;
        b1.x = in.x[i]; b1.y = in.y[i]; b1.z = in.z[i];
        b1.vx = in.vx[i]; b1.vy = in.vy[i]; b1.vz = in.vz[i];
        b1.m = meta[i];
    }
    // whole chains: every flagged neighbour is inside the segment
    const bool p0 = (b0.m & kBondPrev) != 0, n0 = (b0.m & kBondNext) != 0;
    const bool n1 = (b1.m & kBondNext) != 0;  // b1's previous bond is b0's next
    for (int k = 0; k < n_sub; ++k) {
        float w0x, w0y, w0z, w1x, w1y, w1z;  // bonded forces on the lane's two beads
        warp_bonded_forces<kBonded>(b0.x, b0.y, b0.z, b1.x, b1.y, b1.z, p0, n0, n1, c, lane, w0x,
                                    w0y, w0z, w1x, w1y, w1z);
        // the two beads' phases side by side, so their independent work interleaves
        float f00, f01, f02, f10, f11, f12;
        cell_check<kForce, kLerp>(b0, G, g, wcache, tid, f00, f01, f02, G2);
        cell_check<kForce, kLerp>(b1, G, g, wcache, kWarpBlock + tid, f10, f11, f12, G2);
        float g0x = 0.f, g0y = 0.f, g0z = 0.f, g1x = 0.f, g1y = 0.f, g1z = 0.f;
        bool coll0 = false, coll1 = false;
        if (kTherm == 1) {
            gauss3(c, b0.m & kTagMask, step0 + k, g0x, g0y, g0z);
            gauss3(c, b1.m & kTagMask, step0 + k, g1x, g1y, g1z);
        }
        if (kTherm == 2) {
            coll0 = andersen_collides(c, b0.m & kTagMask, step0 + k);
            coll1 = andersen_collides(c, b1.m & kTagMask, step0 + k);
            if (coll0) gauss3(c, b0.m & kTagMask, step0 + k, g0x, g0y, g0z);
            if (coll1) gauss3(c, b1.m & kTagMask, step0 + k, g1x, g1y, g1z);
        }
        // window fraction of this sub-step (the learned field's interpolation)
        const float a = kLerp ? (float)(lerp_j0 + k) * lerp_inv_k : 0.f;
        kick_bead<kTherm, kForce, kLerp>(b0, f00, f01, f02, g0x, g0y, g0z, w0x, w0y, w0z, c, g,
                                         wcache, tid, coll0, a);
        kick_bead<kTherm, kForce, kLerp>(b1, f10, f11, f12, g1x, g1y, g1z, w1x, w1y, w1z, c, g,
                                         wcache, kWarpBlock + tid, coll1, a);
        b0.x = fmaf(c.dt, b0.vx, b0.x);
        b0.y = fmaf(c.dt, b0.vy, b0.y);
        b0.z = fmaf(c.dt, b0.vz, b0.z);
        b1.x = fmaf(c.dt, b1.vx, b1.x);
        b1.y = fmaf(c.dt, b1.vy, b1.y);
        b1.z = fmaf(c.dt, b1.vz, b1.z);
    }
    if constexpr (kObs != 0)
        observe_segment<kTherm>(b0, b1, a0, a1, p0, n0, n1, step0 + n_sub, g, G, c, wcache, tid,
                                *obs, obs_acc);
    if (a0) finish_bead(b0, (long long)base + j0, out, g, D_next, flag);
    if (a1) finish_bead(b1, (long long)base + j1, out, g, D_next, flag);
}

// All replicas of a batch in one persistent launch (a single context is a
// batch of one): the warps walk the concatenated segment lists; each
// segment's replica (warp-uniform) selects its record in the kernel parameter
// block.
template <int kTherm, int kCap, int kForce, int kBonded>
__global__ void __launch_bounds__(kWarpBlock, 2) k_step_warp_batch(
    const __grid_constant__ BatchStepParamsT<kCap> p) {
    griddep_wait();
    griddep_launch_dependents();
    extern __shared__ float4 wcache[];
    __shared__ int s_off[kCap + 1];
    const int tid = threadIdx.x;
    if (tid == 0) {
        int acc = 0;
        for (int r = 0; r < p.R; ++r) {
            s_off[r] = acc;
            acc += *p.rep[r].n_seg;
        }
        s_off[p.R] = acc;
    }
    __syncthreads();
    const int total = s_off[p.R];
    const int warps_total = gridDim.x * (kWarpBlock / 32);
    const long long step0 = p.step_dev ? *p.step_dev : p.step0;
    for (int w = blockIdx.x * (kWarpBlock / 32) + (tid >> 5); w < total; w += warps_total) {
        int lo = 0;  // replica r with s_off[r] <= w < s_off[r + 1]
        if (kCap > 1) {
            int hi = p.R - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= w) lo = mid;
                else hi = mid - 1;
            }
        }
        const BatchStepRep& rp = p.rep[kCap > 1 ? lo : 0];
        const int s = w - s_off[lo];
        advance_segment<kTherm, kForce, kBonded>(rp.st[p.cur], rp.st[p.cur ^ 1], rp.meta,
                                                 rp.seg_start[s],
                                rp.seg_count[s], p.n_sub, step0, rp.g, rp.G, rp.c,
                                p.fuse ? rp.D[p.dnext] : nullptr, p.flag, wcache, tid);
    }
}

// A single context's launch that also forms the observables' bead terms of
// its final state (bonds only, interpolated-gradient force, Langevin or no
// thermostat): each thread's float-float sums over its segments, then the
// block's, one partial per CTA for k_energy_final.
template <int kTherm>
__global__ void __launch_bounds__(kWarpBlock, 2) k_step_warp_obs(
    const __grid_constant__ SingleStepParams p, const ObsArgs o) {
    griddep_wait();
    griddep_launch_dependents();
    extern __shared__ float4 wcache[];
    __shared__ FF sh[kBeadVals][kWarpBlock / 32];
    const int tid = threadIdx.x;
    const BatchStepRep& rp = p.rep[0];
    const int total = *rp.n_seg;
    const int warps_total = gridDim.x * (kWarpBlock / 32);
    const long long step0 = p.step0;
    FF acc[kBeadVals];
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) acc[k] = FF{0.f, 0.f};
    for (int w = blockIdx.x * (kWarpBlock / 32) + (tid >> 5); w < total; w += warps_total)
        advance_segment<kTherm, 0, 0, 0, 1>(rp.st[p.cur], rp.st[p.cur ^ 1], rp.meta,
                                            rp.seg_start[w], rp.seg_count[w], p.n_sub, step0,
                                            rp.g, rp.G, rp.c, p.fuse ? rp.D[p.dnext] : nullptr,
                                            p.flag, wcache, tid, nullptr, 0, 0.f, &o, acc);
    const int wi = tid >> 5;
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) {
        acc[k] = warp_sum_ff(acc[k]);
        if ((tid & 31) == 0) sh[k][wi] = acc[k];
    }
    __syncthreads();
    if (tid < kBeadVals) {
        FF r = sh[tid][0];
#pragma unroll
        for (int j = 1; j < kWarpBlock / 32; ++j) r = ff_plus(r, sh[tid][j]);
        o.part[(size_t)blockIdx.x * kBeadVals + tid] = make_float2(r.h, r.l);
    }
}

// A learned window in one launch (a single context, interpolated-gradient
// force): the field at window step j is (1 - j/K) G0 + (j/K) G2, G0 the field
// of the true density at the window start and G2 that of the predicted
// density at its end -- the field of D(t) + (j/K) dphi, since the field is
// linear in the density.  Each bead caches both cells' polynomials (twelve
// planes); the launch's first sub-step is window step j0.
constexpr size_t kWarpSmemLerp = 2 * sizeof(float4) * kCachePlanes * 2 * kWarpBlock;

template <int kTherm, int kBonded>
__global__ void __launch_bounds__(kWarpBlock, 2) k_step_warp_lerp(
    const __grid_constant__ SingleStepParams p, const float4* __restrict__ G2, int j0,
    float inv_k) {
    griddep_wait();
    griddep_launch_dependents();
    extern __shared__ float4 wcache[];
    const int tid = threadIdx.x;
    const BatchStepRep& rp = p.rep[0];
    const int total = *rp.n_seg;
    const int warps_total = gridDim.x * (kWarpBlock / 32);
    for (int w = blockIdx.x * (kWarpBlock / 32) + (tid >> 5); w < total; w += warps_total)
        advance_segment<kTherm, 0, kBonded, 1>(rp.st[p.cur], rp.st[p.cur ^ 1], rp.meta,
                                               rp.seg_start[w], rp.seg_count[w], p.n_sub,
                                               p.step0, rp.g, rp.G, rp.c,
                                               p.fuse ? rp.D[p.dnext] : nullptr, p.flag, wcache,
                                               tid, G2, j0, inv_k);
}

template <int kTherm, int kBonded>
static void launch_lerp_k(const SingleStepParams& p, const float4* G2, int j0, float inv_k,
                          int blocks, cudaStream_t s) {
    static std::once_flag once[64];
    once_per_device(once, [] {
        cudaFuncSetAttribute(k_step_warp_lerp<kTherm, kBonded>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpSmemLerp);
    });
    launch_pdl(k_step_warp_lerp<kTherm, kBonded>, blocks, kWarpBlock, kWarpSmemLerp, s, p, G2, j0,
               inv_k);
}

template <int kCap, int kTherm, int kForce>
static void warp_attrs_f() {
    cudaFuncSetAttribute(k_step_warp_batch<kTherm, kCap, kForce, 0>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpSmem);
    cudaFuncSetAttribute(k_step_warp_batch<kTherm, kCap, kForce, 1>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpSmem);
    cudaFuncSetAttribute(k_step_warp_batch<kTherm, kCap, kForce, 2>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWarpSmem);
}

template <int kCap, int kTherm>
static void warp_attrs_n() {
    warp_attrs_f<kCap, kTherm, 0>();
    warp_attrs_f<kCap, kTherm, 1>();
    warp_attrs_f<kCap, kTherm, 2>();
}

template <int kCap>
static void warp_attrs() {
    warp_attrs_n<kCap, 0>();
    warp_attrs_n<kCap, 1>();
    warp_attrs_n<kCap, 2>();
}

// The persistent grid of the current device (its SM count times the
// resident CTAs per SM), with the kernels' attributes set on first use.
static int warp_grid_cap() {
    static std::once_flag once[64];
    static int cap[64];
    int dev = 0;
    cudaGetDevice(&dev);
    once_per_device(once, [dev] {
        warp_attrs<HPF_MAX_REPLICAS>();
        warp_attrs<1>();
        cudaFuncSetAttribute(k_step_warp_obs<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kWarpSmem);
        cudaFuncSetAttribute(k_step_warp_obs<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kWarpSmem);
        int sms = 0, per_sm = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, k_step_warp_batch<1, HPF_MAX_REPLICAS, 0, 0>, kWarpBlock,
            kWarpSmem);
        cudaGetLastError();
        cap[dev & 63] = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    });
    return cap[dev & 63];
}

// A context's launches use dependent launch; a batch's are captured into
// graphs and launched plainly.
template <int kCap>
static void launch_warp_k(void (*k)(const BatchStepParamsT<kCap>), const BatchStepParamsT<kCap>& p,
                          int blocks, cudaStream_t s) {
    if (kCap == 1) launch_pdl(k, blocks, kWarpBlock, kWarpSmem, s, p);
    else k<<<blocks, kWarpBlock, kWarpSmem, s>>>(p);
}

template <int kCap, int kTherm, int kForce>
static void launch_warp_f(const BatchStepParamsT<kCap>& p, int blocks, int bonded,
                          cudaStream_t s) {
    if (bonded == 2) launch_warp_k(k_step_warp_batch<kTherm, kCap, kForce, 2>, p, blocks, s);
    else if (bonded == 1) launch_warp_k(k_step_warp_batch<kTherm, kCap, kForce, 1>, p, blocks, s);
    else launch_warp_k(k_step_warp_batch<kTherm, kCap, kForce, 0>, p, blocks, s);
}

template <int kCap, int kTherm>
static void launch_warp_n(const BatchStepParamsT<kCap>& p, int blocks, int force, int bonded,
                          cudaStream_t s) {
    if (force == 2) launch_warp_f<kCap, kTherm, 2>(p, blocks, bonded, s);
    else if (force == 1) launch_warp_f<kCap, kTherm, 1>(p, blocks, bonded, s);
    else launch_warp_f<kCap, kTherm, 0>(p, blocks, bonded, s);
}

template <int kCap>
static void launch_warp(const BatchStepParamsT<kCap>& p, int blocks, int therm, int force,
                        cudaStream_t s) {
    const int bonded = bonded_level(p.rep[0].c);  // all replicas alike (checked at init)
    if (therm == 1) launch_warp_n<kCap, 1>(p, blocks, force, bonded, s);
    else if (therm == 2) launch_warp_n<kCap, 2>(p, blocks, force, bonded, s);
    else launch_warp_n<kCap, 0>(p, blocks, force, bonded, s);
}

void launch_step_warp_batch(const BatchStepParams& p, int max_seg_total, int therm,
                            cudaStream_t s) {
    if (max_seg_total <= 0 || p.n_sub <= 0) return;
    const int cap = warp_grid_cap();
    const int need = (max_seg_total + kWarpBlock / 32 - 1) / (kWarpBlock / 32);
    const int blocks = need < cap ? need : cap;
    launch_warp(p, blocks, therm, p.rep[0].c.force_mode, s);  // replicas share the force mode
}

void launch_step_warp_lerp(const SingleStepParams& p, const float4* G2, int j0, float inv_k,
                           int max_seg, int therm, cudaStream_t s) {
    if (max_seg <= 0 || p.n_sub <= 0) return;
    const int cap = warp_grid_cap();
    const int need = (max_seg + kWarpBlock / 32 - 1) / (kWarpBlock / 32);
    const int blocks = need < cap ? need : cap;
    const int bonded = bonded_level(p.rep[0].c);
    if (therm == 1) {
        if (bonded == 2) launch_lerp_k<1, 2>(p, G2, j0, inv_k, blocks, s);
        else if (bonded == 1) launch_lerp_k<1, 1>(p, G2, j0, inv_k, blocks, s);
        else launch_lerp_k<1, 0>(p, G2, j0, inv_k, blocks, s);
    } else if (therm == 2) {
        if (bonded == 2) launch_lerp_k<2, 2>(p, G2, j0, inv_k, blocks, s);
        else if (bonded == 1) launch_lerp_k<2, 1>(p, G2, j0, inv_k, blocks, s);
        else launch_lerp_k<2, 0>(p, G2, j0, inv_k, blocks, s);
    } else {
        if (bonded == 2) launch_lerp_k<0, 2>(p, G2, j0, inv_k, blocks, s);
        else if (bonded == 1) launch_lerp_k<0, 1>(p, G2, j0, inv_k, blocks, s);
        else launch_lerp_k<0, 0>(p, G2, j0, inv_k, blocks, s);
    }
}

int step_warp_grid_cap() { return warp_grid_cap(); }

int launch_step_warp_obs(const SingleStepParams& p, int max_seg, int therm, float2* part,
                         float half_dt_m, const BondFF& bond, cudaStream_t s) {
    if (max_seg <= 0 || p.n_sub <= 0) return 0;
    const int cap = warp_grid_cap();
    const int need = (max_seg + kWarpBlock / 32 - 1) / (kWarpBlock / 32);
    const int blocks = need < cap ? need : cap;
    const ObsArgs o{part, half_dt_m, bond};
    if (therm == 1) launch_pdl(k_step_warp_obs<1>, blocks, kWarpBlock, kWarpSmem, s, p, o);
    else launch_pdl(k_step_warp_obs<0>, blocks, kWarpBlock, kWarpSmem, s, p, o);
    return blocks;
}

void launch_step_warp_single(const SingleStepParams& p, int max_seg, int therm,
                             cudaStream_t s) {
    if (max_seg <= 0 || p.n_sub <= 0) return;
    const int cap = warp_grid_cap();
    const int need = (max_seg + kWarpBlock / 32 - 1) / (kWarpBlock / 32);
    const int blocks = need < cap ? need : cap;
    launch_warp(p, blocks, therm, p.rep[0].c.force_mode, s);
}


}  // namespace hpf
