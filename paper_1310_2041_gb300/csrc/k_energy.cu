// k_energy.cu -- the FP64 observables (kinetic, bonded and field energy,
// momentum, temperature) of the current step, reduced in a fixed order.
#include "hpf_internal.cuh"

namespace hpf {

// ------------------------------------------------------------------ A7 FP64 observables

constexpr int kRedBlock = 256;
constexpr int kBeadVals = 5;  // kinetic, bond, px, py, pz
constexpr int kBeadsPerThread = 8;  // grid-stride share of a thread (on average)
constexpr int kNodesPerThread = 8;

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

// Knuth's two-sum: s + t == a + b exactly (round-to-nearest, no contraction).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
    s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    t = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
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
__device__ __forceinline__ void bond_energy_ff(float xi, float yi, float zi, float xj, float yj,
                                               float zj, const EnergyConsts& e, float& uh,
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
    const float u = __fmul_rn(e.bond_k_hi, p);
    const float ue = fmaf(e.bond_k_hi, p, -u);
    const float w = fmaf(e.bond_k_hi, q, fmaf(e.bond_k_lo, p, ue));
    float s, t;
    two_sum(uh, u, s, t);
    t = __fadd_rn(t, __fadd_rn(ul, w));
    uh = __fadd_rn(s, t);
    ul = __fsub_rn(t, __fsub_rn(uh, s));
}

// Exact unsigned 128-bit sums (the field energy's node sums).
struct U128 {
    unsigned long long lo, hi;
};
__device__ __forceinline__ void u128_add(U128& a, const U128& b) {
    const unsigned long long lo = a.lo + b.lo;
    a.hi += b.hi + (lo < a.lo ? 1ull : 0ull);
    a.lo = lo;
}
__device__ __forceinline__ U128 u128_mul(unsigned long long a, unsigned long long b) {
    return U128{a * b, __umul64hi(a, b)};
}
__device__ __forceinline__ double u128_to_double(const U128& v) {
    return (double)v.hi * 18446744073709551616.0 + (double)v.lo;
}
__device__ __forceinline__ U128 block_sum_u128(U128 v, U128* sh) {
    for (int o = 16; o > 0; o >>= 1)
        u128_add(v, U128{__shfl_down_sync(0xffffffffu, v.lo, o),
                         __shfl_down_sync(0xffffffffu, v.hi, o)});
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    U128 r{0ull, 0ull};
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) u128_add(r, sh[k]);
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
// the bond to the next bead (each bond once).  The bond energy is formed in
// float-float (bond_energy_ff), the angle and dihedral energies in FP64, all
// from the FP32 positions with exact differences; v_n and its
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
    double ub = 0.0;          // angle and dihedral energies (FP64)
    float uh = 0.f, ul = 0.f;  // bond energy, float-float
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
            bond_energy_ff(x, y, z, xj, yj, zj, e, uh, ul);
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
    ub += (double)uh + (double)ul;
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
// The field energy from exact integer sums.  With phi_K = phi_c D_K (D the
// int64 fixed-point density, non-negative) and T = sum_K D_K per node,
//   W / (rho0 h^3) = 1/2 kT phi_c^2 sum_KK' chi_KK' S_KK'
//                  + 1/2 inv_kappa (phi_c^2 sum T^2 - 2 phi_c sum T + nodes),
// S_KK' = sum over nodes of D_K D_K'.  Every product is below 2^126 and so is
// every sum (at most (sum D_K)(sum D_K') < 2^126), so the node sums are exact
// unsigned 128-bit integers, independent of order; FP64 enters only in the
// final combination.  Per block: the kS (kS + 1) / 2 pair sums (K <= K'),
// sum T^2 and sum T, each as (lo, hi).
template <int kS>
__global__ void __launch_bounds__(kRedBlock) k_energy_nodes(const long long* __restrict__ D,
                                                            int nodes,
                                                            unsigned long long* __restrict__ part) {
    constexpr int kP = kS * (kS + 1) / 2;
    __shared__ U128 sh[kRedBlock / 32];
    U128 acc[kP + 2];
#pragma unroll
    for (int q = 0; q < kP + 2; ++q) acc[q] = U128{0ull, 0ull};
    for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < nodes;
         node += gridDim.x * blockDim.x) {
        unsigned long long d[kS];
        unsigned long long T = 0ull;
#pragma unroll
        for (int k = 0; k < kS; ++k) {
            d[k] = (unsigned long long)D[(size_t)k * nodes + node];
            T += d[k];
        }
        int q = 0;
#pragma unroll
        for (int k = 0; k < kS; ++k)
#pragma unroll
            for (int kp = k; kp < kS; ++kp) u128_add(acc[q++], u128_mul(d[k], d[kp]));
        u128_add(acc[kP], u128_mul(T, T));
        u128_add(acc[kP + 1], U128{T, 0ull});
    }
#pragma unroll
    for (int q = 0; q < kP + 2; ++q) {
        const U128 v = block_sum_u128(acc[q], sh);
        if (threadIdx.x == 0) {
            part[((size_t)blockIdx.x * (kP + 2) + q) * 2] = v.lo;
            part[((size_t)blockIdx.x * (kP + 2) + q) * 2 + 1] = v.hi;
        }
    }
}

__global__ void __launch_bounds__(kRedBlock) k_energy_final(const double* __restrict__ bead_part,
                                                            int nb,
                                                            const unsigned long long* __restrict__ node_part,
                                                            int nn, int nodes, EnergyConsts e,
                                                            double* __restrict__ out6) {
    __shared__ double sh[kRedBlock / 32];
    __shared__ U128 shu[kRedBlock / 32];
    __shared__ double s_field;
    double acc[kBeadVals];
    for (int k = 0; k < kBeadVals; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += bead_part[(size_t)b * kBeadVals + k];
        acc[k] = block_sum(v, sh);
    }
    // the field energy's exact sums, then their combination
    const int nq = e.S * (e.S + 1) / 2 + 2;
    double q_chi = 0.0, t2 = 0.0, t1 = 0.0;
    int k = 0, kp = 0;
    for (int q = 0; q < nq; ++q) {
        U128 v{0ull, 0ull};
        for (int b = threadIdx.x; b < nn; b += blockDim.x)
            u128_add(v, U128{node_part[((size_t)b * nq + q) * 2],
                             node_part[((size_t)b * nq + q) * 2 + 1]});
        const U128 tot = block_sum_u128(v, shu);
        if (threadIdx.x == 0) {
            const double val = u128_to_double(tot);
            if (q < nq - 2) {
                q_chi += (k == kp ? 1.0 : 2.0) * e.chi[k][kp] * val;
                if (++kp == e.S) kp = ++k;
            } else if (q == nq - 2) {
                t2 = val;
            } else {
                t1 = val;
            }
        }
    }
    if (threadIdx.x == 0) {
        const double pc = e.phi_c;
        s_field = e.w_scale * (0.5 * e.kT * pc * pc * q_chi +
                               0.5 * e.inv_kappa * (pc * pc * t2 - 2.0 * pc * t1 + (double)nodes));
        const double ke = acc[0], ub = acc[1], w = s_field;
        out6[0] = ke;
        out6[1] = ub;
        out6[2] = w;
        out6[3] = ke + ub + w;
        out6[4] = sqrt(acc[2] * acc[2] + acc[3] * acc[3] + acc[4] * acc[4]);
        out6[5] = e.n > 0 ? 2.0 * ke / (3.0 * (double)e.n) : 0.0;
    }
}

static int energy_blocks(int count, int per_thread);

int energy_partials_needed(int n, int nodes, int S) {
    // bead partials (doubles), then per node block (S (S + 1) / 2 + 2) sums of two words
    return energy_blocks(n, kBeadsPerThread) * kBeadVals +
           energy_blocks(nodes, kNodesPerThread) * 2 * (S * (S + 1) / 2 + 2) + 1;
}

// Blocks of the energy reductions: each thread takes a grid-stride share (at
// most 8 beads or nodes per thread on average), independent of the device so
// the summation order, and with it every FP64 bit, is the same on any GPU.
static int energy_blocks(int count, int per_thread) {
    const int per_block = kRedBlock * per_thread;
    return (count + per_block - 1) / per_block;
}

void launch_energy(StateBuf st, const uint32_t* meta, int n, MeshGeom g, const float4* G,
                   StepConsts c, long long step, const long long* D, const EnergyConsts& e,
                   double* partials, double* out6, cudaStream_t s) {
    const int nb = energy_blocks(n, kBeadsPerThread);
    const int nn = energy_blocks(g.nodes, kNodesPerThread);
    double* bead_part = partials;
    unsigned long long* node_part =
        reinterpret_cast<unsigned long long*>(partials + (size_t)nb * kBeadVals);
    if (nb > 0) k_energy_beads<<<nb, kRedBlock, 0, s>>>(st, meta, n, g, G, c, step, e, bead_part);
    switch (e.S) {
#define HPF_NODES(k) \
    case k: k_energy_nodes<k><<<nn, kRedBlock, 0, s>>>(D, g.nodes, node_part); break;
        HPF_NODES(1) HPF_NODES(2) HPF_NODES(3) HPF_NODES(4)
        HPF_NODES(5) HPF_NODES(6) HPF_NODES(7) HPF_NODES(8)
#undef HPF_NODES
    }
    k_energy_final<<<1, kRedBlock, 0, s>>>(bead_part, nb, node_part, nn, g.nodes, e, out6);
}

}  // namespace hpf
