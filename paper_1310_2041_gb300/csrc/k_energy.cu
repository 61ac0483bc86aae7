// k_energy.cu -- the FP64 observables (kinetic, bonded and field energy,
// momentum, temperature) of the current step, reduced in a fixed order.
#include "hpf_internal.cuh"

namespace hpf {

// ------------------------------------------------------------------ A7 FP64 observables

constexpr int kRedBlock = 256;
constexpr int kBeadVals = 5;  // kinetic, bond, px, py, pz

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    return r;  // valid in thread 0
}

// |d| in FP64 from an FP32 reciprocal-square-root seed and one Newton step
// y <- y (3 - r2 y^2) / 2 (relative error ~1.5 e0^2 ~ 3e-14 for the FP32
// seed's e0 ~ 1.4e-7); r2 = 0 gives 0.
__device__ __forceinline__ double norm_fp64(double r2) {
    if (!(r2 > 0.0)) return 0.0;
    double y = (double)rsqrtf((float)r2);
    y = y * fma(-0.5 * r2, y * y, 1.5);
    return r2 * y;
}

// Dihedral energy k [1 + cos(n phi - delta)] of the quadruplet i .. i + 3 in
// FP64 from the FP32 positions: cos phi = A.B / (|A||B|), sin phi =
// |b2| b1.B / (|A||B|) with A = b1 x b2, B = b2 x b3, and cos(n phi),
// sin(n phi) by the n-th power of cos phi + i sin phi.
__device__ __forceinline__ double dihedral_energy_fp64(const StateBuf& st, int i,
                                                       const EnergyConsts& e) {
    double b[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        b[k][0] = (double)st.x[i + k + 1] - st.x[i + k];
        b[k][1] = (double)st.y[i + k + 1] - st.y[i + k];
        b[k][2] = (double)st.z[i + k + 1] - st.z[i + k];
    }
    double A[3], B[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int u = (a + 1) % 3, v = (a + 2) % 3;
        A[a] = b[0][u] * b[1][v] - b[0][v] * b[1][u];
        B[a] = b[1][u] * b[2][v] - b[1][v] * b[2][u];
    }
    const double AA = A[0] * A[0] + A[1] * A[1] + A[2] * A[2];
    const double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    const double L = norm_fp64(b[1][0] * b[1][0] + b[1][1] * b[1][1] + b[1][2] * b[1][2]);
    const double den = norm_fp64(AA) * norm_fp64(BB);
    const double cp = (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) / den;
    const double sp = L * (b[0][0] * B[0] + b[0][1] * B[1] + b[0][2] * B[2]) / den;
    double cn = cp, sn = sp;
    for (int k = 1; k < e.dih_n; ++k) {
        const double t = cn * cp - sn * sp;
        sn = sn * cp + cn * sp;
        cn = t;
    }
    return e.dih_k * (1.0 + cn * e.dih_cd + sn * e.dih_sd);
}

// Per bead: F_n exactly as the step kernel forms it, the on-step velocity
// v_n = v + dt/(2m) F_n, then kinetic energy, momentum and the bond energy of
// the bond to the next bead (each bond once).  The bond and angle energies
// are formed in FP64 from the FP32 positions (exact differences); v_n and its
// squares are FP32 (the FP32 force already limits them to ~1e-7) and are
// summed in FP32 over each thread's few beads (at most 8 on average), FP64
// from the block sums on: this GPU's FP64 rate is low.
__global__ void __launch_bounds__(kRedBlock) k_energy_beads(StateBuf st,
                                                            const uint32_t* __restrict__ meta,
                                                            int n, MeshGeom g,
                                                            const float4* __restrict__ G,
                                                            StepConsts c, long long step,
                                                            EnergyConsts e,
                                                            double* __restrict__ partials) {
    __shared__ double sh[kRedBlock / 32];
    double ub = 0.0;
    float kf = 0.f, pfx = 0.f, pfy = 0.f, pfz = 0.f;  // this thread's few beads
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float x = st.x[i], y = st.y[i], z = st.z[i];
        const float vx = st.vx[i], vy = st.vy[i], vz = st.vz[i];
        const uint32_t m = meta[i];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        if (m & kBondPrev)
            bond_force(x - st.x[i - 1], y - st.y[i - 1], z - st.z[i - 1], c.two_k, c.r0, fx, fy, fz);
        if (m & kBondNext) {
            const float xj = st.x[i + 1], yj = st.y[i + 1], zj = st.z[i + 1];
            bond_force(x - xj, y - yj, z - zj, c.two_k, c.r0, fx, fy, fz);
            const double dx = (double)x - xj, dy = (double)y - yj, dz = (double)z - zj;
            const double dr = norm_fp64(dx * dx + dy * dy + dz * dz) - e.r0;
            ub += e.bond_k * dr * dr;
        }
        if (c.two_ka != 0.f) {
            angle_forces_of(st, meta, i, m, c, fx, fy, fz);
            if ((m & kBondPrev) && (m & kBondNext)) {
                // the angle centred here, once, in FP64 from the FP32 positions
                const double ux = (double)st.x[i - 1] - x, uy = (double)st.y[i - 1] - y,
                             uz = (double)st.z[i - 1] - z;
                const double wx = (double)st.x[i + 1] - x, wy = (double)st.y[i + 1] - y,
                             wz = (double)st.z[i + 1] - z;
                const double uu = ux * ux + uy * uy + uz * uz, ww = wx * wx + wy * wy + wz * wz;
                const double uw = ux * wx + uy * wy + uz * wz;
                if (e.angle_form == 1) {
                    // harmonic: theta = atan2(|u x w|, u.w)
                    const double qx = uy * wz - uz * wy, qy = uz * wx - ux * wz,
                                 qz = ux * wy - uy * wx;
                    const double d = atan2(norm_fp64(qx * qx + qy * qy + qz * qz), uw) - e.theta0;
                    ub += e.angle_k * d * d;
                } else {
                    const double cth = uw / norm_fp64(uu * ww);
                    ub += e.angle_k * (cth - e.cos0) * (cth - e.cos0);
                }
            }
        }
        if (c.kd != 0.f) {
            int back, fwd;
            chain_reach(meta, i, m, back, fwd);
            dihedral_forces_of(
                [&](int d) { return make_float3(st.x[i + d], st.y[i + d], st.z[i + d]); }, back,
                fwd, c, fx, fy, fz);
            if (fwd == 3) ub += dihedral_energy_fp64(st, i, e);  // the one starting here, once
        }
        const float4* Gt = G + (size_t)((m >> kTypeShift) & kTypeMask) * g.gnodes;
        gather_field_mode(Gt, g, c.force_mode, x, y, z, fx, fy, fz);
        if (c.sigma > 0.f) {
            float nx, ny, nz;
            gauss3(c, m & kTagMask, step, nx, ny, nz);
            fx += c.sigma * nx;
            fy += c.sigma * ny;
            fz += c.sigma * nz;
        }
        fx -= c.fric * vx;
        fy -= c.fric * vy;
        fz -= c.fric * vz;
        const float hf = (float)e.half_dt_m;
        float ux = fmaf(hf, fx, vx), uy = fmaf(hf, fy, vy), uz = fmaf(hf, fz, vz);
        if (c.p_coll > 0.f && andersen_collides(c, m & kTagMask, step)) {
            // Andersen: this step's collision redraws the on-step velocity
            float nx, ny, nz;
            gauss3(c, m & kTagMask, step, nx, ny, nz);
            ux = c.sig_v * nx;
            uy = c.sig_v * ny;
            uz = c.sig_v * nz;
        }
        kf = fmaf(ux, ux, fmaf(uy, uy, fmaf(uz, uz, kf)));
        pfx += ux;
        pfy += uy;
        pfz += uz;
    }
    const double vals[kBeadVals] = {0.5 * e.mass * (double)kf, ub, e.mass * (double)pfx,
                                    e.mass * (double)pfy, e.mass * (double)pfz};
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) {
        const double s = block_sum(vals[k], sh);
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * kBeadVals + k] = s;
    }
}

// Per node: the field-energy density of the mesh D (FP64 from exact integers).
// Instantiated per species count: this GPU's FP64 rate is low, and loops to
// the species bound would issue predicated FP64 work for absent species.
template <int kS>
__global__ void __launch_bounds__(kRedBlock) k_energy_nodes(const long long* __restrict__ D,
                                                            int nodes, EnergyConsts e,
                                                            double* __restrict__ partials) {
    __shared__ double sh[kRedBlock / 32];
    double w = 0.0;
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nodes;
         node += gridDim.x * blockDim.x) {
        double phi[kS];
        double tot = 0.0;
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            phi[k] = e.phi_c * (double)D[(size_t)k * nodes + node];
            tot += phi[k];
        }
        double q = 0.0;
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            double row = 0.0;
#pragma unroll
            for (int kp = 0; kp < kS; ++kp) row += e.chi[k][kp] * phi[kp];
            q += phi[k] * row;
        }
        w += 0.5 * e.kT * q + 0.5 * e.inv_kappa * (tot - 1.0) * (tot - 1.0);
    }
    const double s = block_sum(w, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Fixed-order final sums -> out6 = {KE, U_bond, W, total, |P|, T}.
__global__ void __launch_bounds__(kRedBlock) k_energy_final(const double* __restrict__ bead_part,
                                                            int nb, const double* __restrict__ node_part,
                                                            int nn, EnergyConsts e,
                                                            double* __restrict__ out6) {
    __shared__ double sh[kRedBlock / 32];
    double acc[kBeadVals + 1];
    for (int k = 0; k < kBeadVals; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += bead_part[(size_t)b * kBeadVals + k];
        acc[k] = block_sum(v, sh);
    }
    double v = 0.0;
    for (int b = threadIdx.x; b < nn; b += blockDim.x) v += node_part[b];
    acc[kBeadVals] = block_sum(v, sh);
    if (threadIdx.x == 0) {
        const double ke = acc[0], ub = acc[1], w = acc[5] * e.w_scale;
        out6[0] = ke;
        out6[1] = ub;
        out6[2] = w;
        out6[3] = ke + ub + w;
        out6[4] = sqrt(acc[2] * acc[2] + acc[3] * acc[3] + acc[4] * acc[4]);
        out6[5] = e.n > 0 ? 2.0 * ke / (3.0 * (double)e.n) : 0.0;
    }
}

static int energy_blocks(int count);

int energy_partials_needed(int n, int nodes) {
    return energy_blocks(n) * kBeadVals + energy_blocks(nodes) + 1;
}

// Blocks of the energy reductions: each thread takes a grid-stride share (at
// most 8 beads or nodes per thread on average), independent of the device so
// the summation order, and with it every FP64 bit, is the same on any GPU.
static int energy_blocks(int count) {
    const int per_block = kRedBlock * 8;
    return (count + per_block - 1) / per_block;
}

void launch_energy(StateBuf st, const uint32_t* meta, int n, MeshGeom g, const float4* G,
                   StepConsts c, long long step, const long long* D, const EnergyConsts& e,
                   double* partials, double* out6, cudaStream_t s) {
    const int nb = energy_blocks(n);
    const int nn = energy_blocks(g.nodes);
    double* bead_part = partials;
    double* node_part = partials + (size_t)nb * kBeadVals;
    if (nb > 0) k_energy_beads<<<nb, kRedBlock, 0, s>>>(st, meta, n, g, G, c, step, e, bead_part);
    switch (e.S) {
#define HPF_NODES(k) \
    case k: k_energy_nodes<k><<<nn, kRedBlock, 0, s>>>(D, g.nodes, e, node_part); break;
        HPF_NODES(1) HPF_NODES(2) HPF_NODES(3) HPF_NODES(4)
        HPF_NODES(5) HPF_NODES(6) HPF_NODES(7) HPF_NODES(8)
#undef HPF_NODES
    }
    k_energy_final<<<1, kRedBlock, 0, s>>>(bead_part, nb, node_part, nn, e, out6);
}

}  // namespace hpf
