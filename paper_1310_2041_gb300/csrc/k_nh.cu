// k_nh.cu -- Nose-Hoover NVT steps (the thermostat the section "MD methods and
// algorithms" names for the canonical ensemble; Hoover's equations
// dv/dt = F/m - xi v, dxi/dt = (2K/(g kT) - 1) / tau^2, deta/dt = xi).
//
// Every step couples all beads through the kinetic energy K, so a step
// cannot run on chip for a whole field period like the Langevin kernel.  The
// step is split where K is needed:
//   force_kick : F_n at the current positions (stored for the next launch);
//                v^E = v + dt/(2m) F_n; the kinetic energy of v^E is summed
//                (float-float pairs of FP32 numbers through the thread, warp
//                and block, block partials added in a fixed order) and the last
//                block to finish applies the two thermostat half steps T(dt/2)
//                (the end of step n - 1, the start of step n), writing the
//                velocity scales s1, s2 and xi, eta;
//   kick_drift : v = s2 (s1 v^E) + dt/(2m) F_n with the stored F_n; x += dt v.
// One launch does kick_drift of step n and force_kick of step n + 1 when no
// field refresh lies between them; a refresh splits them (kick_drift, which
// also deposits the positions into the next density mesh, then the refresh,
// then force_kick).
//
// A fixed grid (at most kNhGrid blocks, set by n alone, so the summation
// order is the same on every GPU) whose threads loop over the beads; the
// state and the stored force are read from one buffer and written to the
// other.  A bead's bonded force after the drift
// needs its chain neighbours' new positions (two beads each way with angles,
// three with dihedrals);
// each thread recomputes those drifts from the neighbours' old state with the
// same arithmetic as the neighbours' own threads, so no grid synchronisation
// is needed and every bit agrees.  Any chain length works.
#include "nh_internal.cuh"

namespace hpf {

namespace {

constexpr int kNhBlock = 256;
constexpr int kNhGrid = 1024;  // at most this many blocks, each thread loops over beads

struct Drift {
    float s1, s2, hdt_m, dt;
    bool on;  // kick_drift launch
};

// Position (and velocity) of bead j after this launch's kick and drift (or
// the stored one when the launch does not drift).
__device__ __forceinline__ void moved(const NhParams& p, const Drift& d, int j, float& x, float& y,
                                      float& z, float& vx, float& vy, float& vz) {
    x = p.in.x[j];
    y = p.in.y[j];
    z = p.in.z[j];
    vx = p.in.vx[j];
    vy = p.in.vy[j];
    vz = p.in.vz[j];
    if (d.on) {
        vx = fmaf(d.hdt_m, p.Fin[0][j], d.s2 * (d.s1 * vx));
        vy = fmaf(d.hdt_m, p.Fin[1][j], d.s2 * (d.s1 * vy));
        vz = fmaf(d.hdt_m, p.Fin[2][j], d.s2 * (d.s1 * vz));
        x = fmaf(d.dt, vx, x);
        y = fmaf(d.dt, vy, y);
        z = fmaf(d.dt, vz, z);
    }
}

__device__ __forceinline__ void moved_pos(const NhParams& p, const Drift& d, int j, float& x,
                                          float& y, float& z) {
    float vx, vy, vz;
    moved(p, d, j, x, y, z, vx, vy, vz);
}

// Bonded force on bead i at (x, y, z): its bonds, with kBonded >= 1 the three
// angles it belongs to (centred at i - 1, i and i + 1) and with kBonded == 2
// the four dihedrals (starting at i - 3 .. i).
template <int kBonded>
__device__ __forceinline__ void bonded_of(const NhParams& p, const Drift& d, int i, uint32_t m,
                                          float x, float y, float z, float& fx, float& fy,
                                          float& fz) {
    const bool hp = (m & kBondPrev) != 0, hn = (m & kBondNext) != 0;
    float xp = 0.f, yp = 0.f, zp = 0.f, xn = 0.f, yn = 0.f, zn = 0.f;
    if (hp) {
        moved_pos(p, d, i - 1, xp, yp, zp);
        bond_force(x - xp, y - yp, z - zp, p.c.two_k, p.c.r0, fx, fy, fz);
    }
    if (hn) {
        moved_pos(p, d, i + 1, xn, yn, zn);
        bond_force(x - xn, y - yn, z - zn, p.c.two_k, p.c.r0, fx, fy, fz);
    }
    if (kBonded == 0) return;
    float ax, ay, az, bx, by, bz;
    if (hp && hn) {
        angle_force(xp - x, yp - y, zp - z, xn - x, yn - y, zn - z, p.c.two_ka, p.c, ax, ay,
                    az, bx, by, bz);
        fx -= ax + bx;
        fy -= ay + by;
        fz -= az + bz;
    }
    if (hp && (p.meta[i - 1] & kBondPrev)) {
        float xq, yq, zq;
        moved_pos(p, d, i - 2, xq, yq, zq);
        angle_force(xq - xp, yq - yp, zq - zp, x - xp, y - yp, z - zp, p.c.two_ka, p.c, ax,
                    ay, az, bx, by, bz);
        fx += bx;
        fy += by;
        fz += bz;
    }
    if (hn && (p.meta[i + 1] & kBondNext)) {
        float xq, yq, zq;
        moved_pos(p, d, i + 2, xq, yq, zq);
        angle_force(x - xn, y - yn, z - zn, xq - xn, yq - yn, zq - zn, p.c.two_ka, p.c, ax,
                    ay, az, bx, by, bz);
        fx += ax;
        fy += ay;
        fz += az;
    }
    if (kBonded == 2) {
        int back, fwd;
        chain_reach(p.meta, i, m, back, fwd);
        dihedral_forces_of(
            [&](int dd) {
                float3 r = make_float3(x, y, z);
                if (dd != 0) moved_pos(p, d, i + dd, r.x, r.y, r.z);
                return r;
            },
            back, fwd, p.c, fx, fy, fz);
    }
}

__device__ __forceinline__ double nh_rate(const NhConsts& t, double K) {
    return t.dof_kT > 0.0 ? fma(K, t.two_over_dof_kT, -1.0) * t.inv_tau2 : 0.0;
}

// One thermostat half step T(h) (h = dt/2): xi += (h/2) G(K); s = exp(-xi h);
// K *= s^2; eta += xi h; xi += (h/2) G(K).  Returns s.  The scale is taken in
// FP32 (it multiplies FP32 velocities); this GPU's FP64 rate is low and the
// step waits for this one thread.
__device__ __forceinline__ double nh_half(const NhConsts& t, double& xi, double& eta, double& K) {
    xi += 0.5 * t.h * nh_rate(t, K);
    const double s = (double)expf((float)(-xi * t.h));
    K *= s * s;
    eta += xi * t.h;
    xi += 0.5 * t.h * nh_rate(t, K);
    return s;
}

template <int kForce, int kBonded>
__global__ void __launch_bounds__(kNhBlock) k_nh_step(const __grid_constant__ NhParams p) {
    // dependent launch: the previous launch's state, force and velocity
    // scales are read only after it has completed
    griddep_wait();
    griddep_launch_dependents();
    __shared__ FF s_ke[kNhBlock / 32];
    __shared__ bool s_last;
    const int tid = threadIdx.x, lane = tid & 31;
    Drift d;
    d.on = p.kick_drift != 0;
    d.s1 = d.on ? p.nh->s1 : 1.0f;
    d.s2 = d.on ? p.nh->s2 : 1.0f;
    d.hdt_m = 0.5f * p.c.dt_m;
    d.dt = p.c.dt;
    FF ke{0.f, 0.f};  // this thread's beads, float-float (FP32 pipe) up to the last block
#pragma unroll 2
    for (int i = blockIdx.x * kNhBlock + tid; i < p.n; i += gridDim.x * kNhBlock) {
        const uint32_t m = p.meta[i];
        float x, y, z, vx, vy, vz;
        moved(p, d, i, x, y, z, vx, vy, vz);
        if (p.force_kick) {
            float fx = 0.f, fy = 0.f, fz = 0.f;
            bonded_of<kBonded>(p, d, i, m, x, y, z, fx, fy, fz);
            const float4* Gt = p.G + (size_t)((m >> kTypeShift) & kTypeMask) * p.g.gnodes;
            gather_field_mode(Gt, p.g, kForce, x, y, z, fx, fy, fz);
            p.Fout[0][i] = fx;
            p.Fout[1][i] = fy;
            p.Fout[2][i] = fz;
            vx = fmaf(d.hdt_m, fx, vx);
            vy = fmaf(d.hdt_m, fy, vy);
            vz = fmaf(d.hdt_m, fz, vz);
            ke = ff_plus(ke, fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
        }
        p.out.x[i] = x;
        p.out.y[i] = y;
        p.out.z[i] = z;
        p.out.vx[i] = vx;
        p.out.vy[i] = vy;
        p.out.vz[i] = vz;
        const bool finite = isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) &&
                            isfinite(vy) && isfinite(vz);
        if (!finite) atomicOr(p.flag, kFlagNonFinite);
        else if (!(coord_in_range(x, p.g.inv_h[0]) && coord_in_range(y, p.g.inv_h[1]) &&
                   coord_in_range(z, p.g.inv_h[2])))
            atomicOr(p.flag, kFlagRange);
        else if (p.D_next) {
            const AxisCoord ax = axis_coord(x, p.g.inv_h[0], p.g.mx, p.g.inv_m[0]);
            const AxisCoord ay = axis_coord(y, p.g.inv_h[1], p.g.my, p.g.inv_m[1]);
            const AxisCoord az = axis_coord(z, p.g.inv_h[2], p.g.mz, p.g.inv_m[2]);
            scatter_bead(p.D_next + (size_t)((m >> kTypeShift) & kTypeMask) * p.g.nodes, p.g,
                         ax, ay, az);
        }
    }
    if (!p.force_kick) return;
    // the kinetic-energy sum in float-float on the FP32 pipe (this GPU's FP64
    // rate is 1/64 of its FP32 rate): warp, block, then the blocks' partials
    // in a fixed order
    ke = warp_sum_ff(ke);
    if (lane == 0) s_ke[tid >> 5] = ke;
    __syncthreads();
    if (tid == 0) {
        FF b = s_ke[0];
        for (int k = 1; k < kNhBlock / 32; ++k) b = ff_plus(b, s_ke[k]);
        p.part[blockIdx.x] = make_float2(b.h, b.l);
        __threadfence();
        s_last = atomicAdd(&p.nh->ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // the last block sums the partials in a fixed order (strided per thread,
    // then the same shuffle tree and warp order as above)
    __threadfence();
    FF v{0.f, 0.f};
    for (int k = tid; k < (int)gridDim.x; k += kNhBlock) {
        const float2 q = __ldcg(&p.part[k]);
        v = ff_plus(v, FF{q.x, q.y});
    }
    v = warp_sum_ff(v);
    __syncthreads();
    if (lane == 0) s_ke[tid >> 5] = v;
    __syncthreads();
    if (tid != 0) return;
    FF tot = s_ke[0];
    for (int k = 1; k < kNhBlock / 32; ++k) tot = ff_plus(tot, s_ke[k]);
    const double sum = ff_to_double(tot);
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

template <int kForce>
void launch_nh_e(const NhParams& p, int bonded, cudaStream_t s) {
    const int blocks = nh_blocks(p.n);
    if (bonded == 2) launch_pdl(k_nh_step<kForce, 2>, blocks, kNhBlock, 0, s, p);
    else if (bonded == 1) launch_pdl(k_nh_step<kForce, 1>, blocks, kNhBlock, 0, s, p);
    else launch_pdl(k_nh_step<kForce, 0>, blocks, kNhBlock, 0, s, p);
}

}  // namespace

int nh_blocks(int n) {
    // a fixed grid (it depends only on n): the summation order of the kinetic
    // energy is the same on every GPU
    const int b = (n + kNhBlock - 1) / kNhBlock;
    return b < kNhGrid ? b : kNhGrid;
}

void launch_nh_step(const NhParams& p, cudaStream_t s) {
    if (p.n <= 0) return;
    const int bonded = bonded_level(p.c);
    if (p.c.force_mode == 2) launch_nh_e<2>(p, bonded, s);
    else if (p.c.force_mode == 1) launch_nh_e<1>(p, bonded, s);
    else launch_nh_e<0>(p, bonded, s);
}

}  // namespace hpf
