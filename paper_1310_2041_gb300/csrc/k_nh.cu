// k_nh.cu -- Nose-Hoover NVT steps (the thermostat the section "MD methods and
// algorithms" names for the canonical ensemble; Hoover's equations
// dv/dt = F/m - xi v, dxi/dt = (2K/(g kT) - 1) / tau^2, deta/dt = xi).
//
// Every step couples all beads through the kinetic energy K, so a step
// cannot run on chip for a whole field period like the Langevin kernel.  The
// step is split where K is needed:
//   force_kick : F_n at the current positions; v^E = v + dt/(2m) F_n; the
//                kinetic energy of v^E is summed (FP64, per-block partials in a
//                fixed order) and the last block to finish applies the two
//                thermostat half steps T(dt/2) (the end of step n - 1, the
//                start of step n), writing the velocity scales s1, s2 and xi, eta;
//   kick_drift : v = s2 (s1 v^E) + dt/(2m) F_n (F_n recomputed from the same
//                positions and field, so the bits agree); x += dt v.
// One launch does kick_drift of step n and force_kick of step n + 1 when no
// field refresh lies between them; a refresh splits them (kick_drift, which
// also deposits the positions into the next density mesh, then the refresh,
// then force_kick).  Beads are advanced in place, one warp per segment of
// whole chains (two beads per lane, bonded neighbours by shuffles), so the
// result does not depend on how the steps are split into calls.
#include "hpf_internal.cuh"

namespace hpf {

namespace {

constexpr int kNhBlock = 256;

struct NhBead {
    float x, y, z, vx, vy, vz;
    uint32_t m;
};

template <bool kExact>
__device__ __forceinline__ void field_force_at(const NhBead& b, const MeshGeom& g,
                                               const float4* __restrict__ G, float& fx, float& fy,
                                               float& fz) {
    const float4* Gt = G + (size_t)((b.m >> kTypeShift) & kTypeMask) * g.gnodes;
    const AxisCoord ax = axis_gather(b.x, g.inv_h[0], (float)g.mx, g.inv_m[0]);
    const AxisCoord ay = axis_gather(b.y, g.inv_h[1], (float)g.my, g.inv_m[1]);
    const AxisCoord az = axis_gather(b.z, g.inv_h[2], (float)g.mz, g.inv_m[2]);
    if (kExact) gather_field_exact(Gt, g, ax, ay, az, fx, fy, fz);
    else gather_field(Gt, g, ax, ay, az, fx, fy, fz);
}

// Conservative forces on the lane's two beads (bonded terms by shuffles: the
// whole warp must call this).
template <bool kExact, bool kAngles>
__device__ __forceinline__ void pair_forces(const NhBead& b0, const NhBead& b1, bool p0, bool n0,
                                            bool n1, const NhParams& p, int lane, float* F) {
    warp_bonded_forces<kAngles>(b0.x, b0.y, b0.z, b1.x, b1.y, b1.z, p0, n0, n1, p.c, lane, F[0],
                                F[1], F[2], F[3], F[4], F[5]);
    field_force_at<kExact>(b0, p.g, p.G, F[0], F[1], F[2]);
    field_force_at<kExact>(b1, p.g, p.G, F[3], F[4], F[5]);
}

__device__ __forceinline__ double nh_rate(const NhConsts& t, double K) {
    return t.dof_kT > 0.0 ? (2.0 * K / t.dof_kT - 1.0) * t.inv_tau2 : 0.0;
}

// One thermostat half step T(h) (h = dt/2): xi += (h/2) G(K); s = exp(-xi h);
// K *= s^2; eta += xi h; xi += (h/2) G(K).  Returns s.
__device__ __forceinline__ double nh_half(const NhConsts& t, double& xi, double& eta, double& K) {
    xi += 0.5 * t.h * nh_rate(t, K);
    const double s = exp(-xi * t.h);
    K *= s * s;
    eta += xi * t.h;
    xi += 0.5 * t.h * nh_rate(t, K);
    return s;
}

template <bool kExact, bool kAngles>
__global__ void __launch_bounds__(kNhBlock) k_nh_step(const __grid_constant__ NhParams p) {
    __shared__ double s_ke[kNhBlock / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31;
    const float hdt_m = 0.5f * p.c.dt_m;
    float s1 = 1.0f, s2 = 1.0f;
    if (p.kick_drift) {
        s1 = p.nh->s1;
        s2 = p.nh->s2;
    }
    double ke = 0.0;  // sum of |v^E|^2 over this thread's beads
    const int n_seg = *p.n_seg;
    const int warps_total = gridDim.x * (kNhBlock / 32);
    for (int w = blockIdx.x * (kNhBlock / 32) + (tid >> 5); w < n_seg; w += warps_total) {
        const int base = p.seg_start[w], cnt = p.seg_count[w];
        const int j0 = 2 * lane, j1 = j0 + 1;
        const bool a0 = j0 < cnt, a1 = j1 < cnt;
        NhBead b0{0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u}, b1 = b0;
        if (a0) {
            const long long i = (long long)base + j0;
            b0 = NhBead{p.st.x[i], p.st.y[i], p.st.z[i], p.st.vx[i], p.st.vy[i], p.st.vz[i],
                        p.meta[i]};
        }
        if (a1) {
            const long long i = (long long)base + j1;
            b1 = NhBead{p.st.x[i], p.st.y[i], p.st.z[i], p.st.vx[i], p.st.vy[i], p.st.vz[i],
                        p.meta[i]};
        }
        const bool p0 = (b0.m & kBondPrev) != 0, n0 = (b0.m & kBondNext) != 0;
        const bool n1 = (b1.m & kBondNext) != 0;
        float F[6];
        if (p.kick_drift) {
            pair_forces<kExact, kAngles>(b0, b1, p0, n0, n1, p, lane, F);
            b0.vx = fmaf(hdt_m, F[0], s2 * (s1 * b0.vx));
            b0.vy = fmaf(hdt_m, F[1], s2 * (s1 * b0.vy));
            b0.vz = fmaf(hdt_m, F[2], s2 * (s1 * b0.vz));
            b1.vx = fmaf(hdt_m, F[3], s2 * (s1 * b1.vx));
            b1.vy = fmaf(hdt_m, F[4], s2 * (s1 * b1.vy));
            b1.vz = fmaf(hdt_m, F[5], s2 * (s1 * b1.vz));
            b0.x = fmaf(p.c.dt, b0.vx, b0.x);
            b0.y = fmaf(p.c.dt, b0.vy, b0.y);
            b0.z = fmaf(p.c.dt, b0.vz, b0.z);
            b1.x = fmaf(p.c.dt, b1.vx, b1.x);
            b1.y = fmaf(p.c.dt, b1.vy, b1.y);
            b1.z = fmaf(p.c.dt, b1.vz, b1.z);
        }
        if (p.force_kick) {
            pair_forces<kExact, kAngles>(b0, b1, p0, n0, n1, p, lane, F);
            b0.vx = fmaf(hdt_m, F[0], b0.vx);
            b0.vy = fmaf(hdt_m, F[1], b0.vy);
            b0.vz = fmaf(hdt_m, F[2], b0.vz);
            b1.vx = fmaf(hdt_m, F[3], b1.vx);
            b1.vy = fmaf(hdt_m, F[4], b1.vy);
            b1.vz = fmaf(hdt_m, F[5], b1.vz);
            if (a0) ke += (double)fmaf(b0.vx, b0.vx, fmaf(b0.vy, b0.vy, b0.vz * b0.vz));
            if (a1) ke += (double)fmaf(b1.vx, b1.vx, fmaf(b1.vy, b1.vy, b1.vz * b1.vz));
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            if (!(k ? a1 : a0)) continue;
            const NhBead& b = k ? b1 : b0;
            const long long i = (long long)base + (k ? j1 : j0);
            p.st.x[i] = b.x;
            p.st.y[i] = b.y;
            p.st.z[i] = b.z;
            p.st.vx[i] = b.vx;
            p.st.vy[i] = b.vy;
            p.st.vz[i] = b.vz;
            const bool finite = isfinite(b.x) && isfinite(b.y) && isfinite(b.z) &&
                                isfinite(b.vx) && isfinite(b.vy) && isfinite(b.vz);
            if (!finite) atomicOr(p.flag, kFlagNonFinite);
            else if (!(coord_in_range(b.x, p.g.inv_h[0]) && coord_in_range(b.y, p.g.inv_h[1]) &&
                       coord_in_range(b.z, p.g.inv_h[2])))
                atomicOr(p.flag, kFlagRange);
            else if (p.D_next) {
                const AxisCoord ax = axis_coord(b.x, p.g.inv_h[0], p.g.mx, p.g.inv_m[0]);
                const AxisCoord ay = axis_coord(b.y, p.g.inv_h[1], p.g.my, p.g.inv_m[1]);
                const AxisCoord az = axis_coord(b.z, p.g.inv_h[2], p.g.mz, p.g.inv_m[2]);
                scatter_bead(p.D_next + (size_t)((b.m >> kTypeShift) & kTypeMask) * p.g.nodes,
                             p.g, ax, ay, az);
            }
        }
    }
    if (!p.force_kick) return;
    // the kinetic-energy sum: warp, block, then the blocks' partials in order
    for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
    if (lane == 0) s_ke[tid >> 5] = ke;
    __syncthreads();
    if (tid == 0) {
        double b = 0.0;
        for (int k = 0; k < kNhBlock / 32; ++k) b += s_ke[k];
        p.nh->part[blockIdx.x] = b;
        __threadfence();
        s_last = atomicAdd(&p.nh->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last || tid != 0) return;
    __threadfence();
    double sum = 0.0;
    for (int k = 0; k < (int)gridDim.x; ++k) sum += __ldcg(&p.nh->part[k]);
    double K = 0.5 * p.t.mass * sum;
    double xi = p.nh->xi, eta = p.nh->eta;
    p.nh->ke = K;
    const double a = nh_half(p.t, xi, eta, K);  // the end of step n - 1
    const double b = nh_half(p.t, xi, eta, K);  // the start of step n
    p.nh->s1 = (float)a;
    p.nh->s2 = (float)b;
    p.nh->xi = xi;
    p.nh->eta = eta;
    p.nh->ticket = 0u;
}

template <bool kExact>
void launch_nh_e(const NhParams& p, int blocks, bool angles, cudaStream_t s) {
    if (angles) k_nh_step<kExact, true><<<blocks, kNhBlock, 0, s>>>(p);
    else k_nh_step<kExact, false><<<blocks, kNhBlock, 0, s>>>(p);
}

}  // namespace

int nh_grid(int max_seg) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_nh_step<false, false>, kNhBlock, 0);
    cudaGetLastError();
    int cap = (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (cap > kNhMaxBlocks) cap = kNhMaxBlocks;
    const int need = (max_seg + kNhBlock / 32 - 1) / (kNhBlock / 32);
    const int blocks = need < cap ? need : cap;
    return blocks > 0 ? blocks : 1;
}

void launch_nh_step(const NhParams& p, int blocks, cudaStream_t s) {
    const bool angles = p.c.two_ka != 0.f;
    if (p.c.exact) launch_nh_e<true>(p, blocks, angles, s);
    else launch_nh_e<false>(p, blocks, angles, s);
}

}  // namespace hpf
