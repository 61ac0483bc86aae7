// k_energy.cu -- the FP64 observables (kinetic, bonded and field energy,
// momentum, temperature) of the current step, reduced in a fixed order.
#include "hpf_internal.cuh"

namespace hpf {

// ------------------------------------------------------------------ A7 FP64 observables

constexpr int kRedBlock = 256;    // the bead and node kernels
constexpr int kFinalBlock = 1024;  // the one block that combines their partials
// Grid-stride shares (on average) of a bead or node thread: small, so that a
// million beads make about 2000 blocks, which the SMs take in several waves
// with little left over for the last one (at 8 beads a thread the 489 blocks
// of a million beads came to just over one wave of three blocks per SM).
constexpr int kBeadsPerThread = 2;
constexpr int kNodesPerThread = 2;

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
__device__ __forceinline__ U128 warp_sum_u128(U128 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        u128_add(v, U128{__shfl_down_sync(0xffffffffu, v.lo, o),
                         __shfl_down_sync(0xffffffffu, v.hi, o)});
    return v;  // lane 0
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

// Per bead: F_n with the terms the step kernel's kick uses (bonds, the field
// by a direct trilinear gather, friction, step n's noise), the on-step velocity
// v_n = v + dt/(2m) F_n, then kinetic energy, momentum and the bond energy of
// the bond to the next bead (each bond once).  The bond energy is formed in
// float-float (bond_energy_ff), the angle and dihedral energies in FP64, all
// from the FP32 positions with exact differences; v_n and |v_n|^2 are FP32
// (the FP32 force already limits them to ~1e-7) and are summed in float-float
// over the thread's beads, its warp and its block, into one float-float
// partial per observable and block (kinetic energy without the factor m/2 and
// momentum without m, both applied in FP64 in k_energy_final).
// Block blk of nb bead blocks (grid-stride over the beads within them).
__device__ __forceinline__ void energy_beads_block(const StateBuf& st,
                                                   const uint32_t* __restrict__ meta, int n,
                                                   const MeshGeom& g,
                                                   const float4* __restrict__ G,
                                                   const StepConsts& c, long long step,
                                                   const EnergyConsts& e,
                                                   float2* __restrict__ partials, int blk, int nb,
                                                   FF (*sh)[kRedBlock / 32]) {
    double ub = 0.0;           // angle and dihedral energies (FP64)
    float uh = 0.f, ul = 0.f;  // bond energy, float-float
    FF kf{0.f, 0.f}, pfx{0.f, 0.f}, pfy{0.f, 0.f}, pfz{0.f, 0.f};
    for (int i = blk * kRedBlock + threadIdx.x; i < n; i += nb * kRedBlock) {
        const float x = st.x[i], y = st.y[i], z = st.z[i];
        const float vx = st.vx[i], vy = st.vy[i], vz = st.vz[i];
        const uint32_t m = meta[i];
        float fx = 0.f, fy = 0.f, fz = 0.f;
        if (m & kBondPrev)
            bond_force(x - st.x[i - 1], y - st.y[i - 1], z - st.z[i - 1], c.two_k, c.r0, fx, fy, fz);
        if (m & kBondNext) {
            const float xj = st.x[i + 1], yj = st.y[i + 1], zj = st.z[i + 1];
            bond_force(x - xj, y - yj, z - zj, c.two_k, c.r0, fx, fy, fz);
            bond_energy_ff(x, y, z, xj, yj, zj, bond_ff(e), uh, ul);
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
        kf = ff_plus(kf, fmaf(ux, ux, fmaf(uy, uy, __fmul_rn(uz, uz))));
        pfx = ff_plus(pfx, ux);
        pfy = ff_plus(pfy, uy);
        pfz = ff_plus(pfz, uz);
    }
    FF v[kBeadVals] = {kf, ff_norm(uh, ul), pfx, pfy, pfz};
    if (c.two_ka != 0.f || c.kd != 0.f) v[1] = ff_plus(v[1], ff_from_double(ub));
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) {
        v[k] = warp_sum_ff(v[k]);
        if ((threadIdx.x & 31) == 0) sh[k][w] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < kBeadVals) {
        FF r = sh[threadIdx.x][0];
#pragma unroll
        for (int j = 1; j < kRedBlock / 32; ++j) r = ff_plus(r, sh[threadIdx.x][j]);
        partials[(size_t)blk * kBeadVals + threadIdx.x] = make_float2(r.h, r.l);
    }
}

// Per node: the exact integer sums behind the field energy, instantiated per
// species count (the kS (kS + 1) / 2 + 2 sums are register arrays).
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
__device__ __forceinline__ void energy_nodes_block(const long long* __restrict__ D, int nodes,
                                                   unsigned long long* __restrict__ part, int blk,
                                                   int nn, U128 (*sh)[kRedBlock / 32]) {
    constexpr int kP = kS * (kS + 1) / 2;
    constexpr int kQ = kP + 2;
    U128 acc[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) acc[q] = U128{0ull, 0ull};
    for (int node = blk * kRedBlock + threadIdx.x; node < nodes; node += nn * kRedBlock) {
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
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        acc[q] = warp_sum_u128(acc[q]);
        if ((threadIdx.x & 31) == 0) sh[q][w] = acc[q];
    }
    __syncthreads();
    if (threadIdx.x < kQ) {
        U128 r = sh[threadIdx.x][0];
#pragma unroll
        for (int j = 1; j < kRedBlock / 32; ++j) u128_add(r, sh[threadIdx.x][j]);
        part[((size_t)blk * kQ + threadIdx.x) * 2] = r.lo;
        part[((size_t)blk * kQ + threadIdx.x) * 2 + 1] = r.hi;
    }
}

// The node sums alone (many species: their accumulators would not fit the
// register budget of the combined kernel below).
template <int kS>
__global__ void __launch_bounds__(kRedBlock) k_energy_nodes(const long long* __restrict__ D,
                                                            int nodes,
                                                            unsigned long long* __restrict__ part) {
    __shared__ U128 sh[kS * (kS + 1) / 2 + 2][kRedBlock / 32];
    energy_nodes_block<kS>(D, nodes, part, blockIdx.x, gridDim.x, sh);
    griddep_launch_dependents();
}

// One launch for the bead and node sums: blocks 0 .. nn - 1 take the nodes
// (kN species; 0: none), the rest the beads, so the two run side by side.
template <int kN>
__global__ void __launch_bounds__(kRedBlock, 4) k_energy_main(StateBuf st,
                                                              const uint32_t* __restrict__ meta,
                                                              int n, MeshGeom g,
                                                              const float4* __restrict__ G,
                                                              StepConsts c, long long step,
                                                              EnergyConsts e,
                                                              float2* __restrict__ bead_part,
                                                              int nb, const long long* __restrict__ D,
                                                              unsigned long long* __restrict__ node_part,
                                                              int nn) {
    constexpr int kQ = kN * (kN + 1) / 2 + 2;
    constexpr int kBytes = (int)sizeof(U128) * kQ > (int)sizeof(FF) * kBeadVals
                               ? (int)sizeof(U128) * kQ
                               : (int)sizeof(FF) * kBeadVals;
    __shared__ __align__(16) unsigned char sm[kBytes * (kRedBlock / 32)];
    int blk = (int)blockIdx.x;
    if constexpr (kN > 0) {
        if (blk < nn) {
            energy_nodes_block<kN>(D, g.nodes, node_part, blk, nn,
                                   reinterpret_cast<U128(*)[kRedBlock / 32]>(sm));
            griddep_launch_dependents();
            return;
        }
        blk -= nn;
    }
    energy_beads_block(st, meta, n, g, G, c, step, e, bead_part, blk, nb,
                       reinterpret_cast<FF(*)[kRedBlock / 32]>(sm));
    // the combining kernel may be scheduled once every block is here
    griddep_launch_dependents();
}

// One block: the bead partials (float-float) and the node partials (exact
// 128-bit) summed over the blocks in a fixed order -- each thread a strided
// share of the blocks, its loads all in flight together, then its warp, then
// one lane per value over the warps -- and combined in FP64.
template <int kS>
__global__ void __launch_bounds__(kFinalBlock) k_energy_final(const float2* __restrict__ bead_part,
                                                              int nb,
                                                              const unsigned long long* __restrict__ node_part,
                                                              int nn, int nodes, EnergyConsts e,
                                                              double* __restrict__ out6) {
    constexpr int kP = kS * (kS + 1) / 2;
    constexpr int kQ = kP + 2;
    constexpr int kW = kFinalBlock / 32;
    __shared__ FF shf[kBeadVals][kW];
    __shared__ U128 shu[kQ][kW];
    __shared__ double res[kBeadVals + kQ];
    griddep_wait();  // launched programmatically after the partial sums
    FF acc[kBeadVals];
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) acc[k] = FF{0.f, 0.f};
    for (int b = threadIdx.x; b < nb; b += kFinalBlock) {
        float2 p[kBeadVals];
#pragma unroll
        for (int k = 0; k < kBeadVals; ++k) p[k] = bead_part[(size_t)b * kBeadVals + k];
#pragma unroll
        for (int k = 0; k < kBeadVals; ++k) acc[k] = ff_plus(acc[k], FF{p[k].x, p[k].y});
    }
    U128 qa[kQ];
#pragma unroll
    for (int q = 0; q < kQ; ++q) qa[q] = U128{0ull, 0ull};
    for (int b = threadIdx.x; b < nn; b += kFinalBlock) {
        U128 p[kQ];
#pragma unroll
        for (int q = 0; q < kQ; ++q)
            p[q] = U128{node_part[((size_t)b * kQ + q) * 2], node_part[((size_t)b * kQ + q) * 2 + 1]};
#pragma unroll
        for (int q = 0; q < kQ; ++q) u128_add(qa[q], p[q]);
    }
    const int w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kBeadVals; ++k) {
        acc[k] = warp_sum_ff(acc[k]);
        if ((threadIdx.x & 31) == 0) shf[k][w] = acc[k];
    }
#pragma unroll
    for (int q = 0; q < kQ; ++q) {
        qa[q] = warp_sum_u128(qa[q]);
        if ((threadIdx.x & 31) == 0) shu[q][w] = qa[q];
    }
    __syncthreads();
    const int t = threadIdx.x;
    if (t < kBeadVals) {
        FF r = shf[t][0];
        for (int j = 1; j < kW; ++j) r = ff_plus(r, shf[t][j]);
        res[t] = ff_to_double(r);
    } else if (t >= 32 && t < 32 + kQ) {  // another warp, so that both run at once
        U128 r = shu[t - 32][0];
        for (int j = 1; j < kW; ++j) u128_add(r, shu[t - 32][j]);
        res[kBeadVals + t - 32] = u128_to_double(r);
    }
    __syncthreads();
    if (t == 0) {
        double q_chi = 0.0;
        int q = 0;
        for (int k = 0; k < kS; ++k)
            for (int kp = k; kp < kS; ++kp, ++q)
                q_chi += (k == kp ? 1.0 : 2.0) * e.chi[k][kp] * res[kBeadVals + q];
        const double t2 = res[kBeadVals + kP], t1 = res[kBeadVals + kP + 1];
        const double pc = e.phi_c;
        const double w_f = e.w_scale * (0.5 * e.kT * pc * pc * q_chi +
                                        0.5 * e.inv_kappa * (pc * pc * t2 - 2.0 * pc * t1 +
                                                             (double)nodes));
        const double ke = 0.5 * e.mass * res[0], ub = res[1];
        const double px = e.mass * res[2], py = e.mass * res[3], pz = e.mass * res[4];
        out6[0] = ke;
        out6[1] = ub;
        out6[2] = w_f;
        out6[3] = ke + ub + w_f;
        out6[4] = sqrt(px * px + py * py + pz * pz);
        out6[5] = e.n > 0 ? 2.0 * ke / (3.0 * (double)e.n) : 0.0;
    }
}

static int energy_blocks(int count, int per_thread);

int energy_launches(int n, int S) { return S <= 3 ? 2 : (n > 0 ? 3 : 2); }

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
    // bead partials: kBeadVals float-float pairs (one double's room each) per block
    float2* bead_part = reinterpret_cast<float2*>(partials);
    unsigned long long* node_part =
        reinterpret_cast<unsigned long long*>(partials + (size_t)nb * kBeadVals);
    // up to three species: node and bead sums in one launch; more species:
    // the node sums in a launch of their own, after the beads
    if (e.S <= 3) {
        switch (e.S) {
#define HPF_MAIN(k)                                                                              \
    case k:                                                                                      \
        k_energy_main<k><<<nn + nb, kRedBlock, 0, s>>>(st, meta, n, g, G, c, step, e, bead_part, \
                                                       nb, D, node_part, nn);                    \
        break;
            HPF_MAIN(1) HPF_MAIN(2) HPF_MAIN(3)
#undef HPF_MAIN
        }
    } else {
        if (nb > 0)
            k_energy_main<0><<<nb, kRedBlock, 0, s>>>(st, meta, n, g, G, c, step, e, bead_part, nb,
                                                      D, node_part, 0);
        switch (e.S) {
#define HPF_NODES(k)                                                                     \
    case k: k_energy_nodes<k><<<nn, kRedBlock, 0, s>>>(D, g.nodes, node_part); break;
            HPF_NODES(4) HPF_NODES(5) HPF_NODES(6) HPF_NODES(7) HPF_NODES(8)
#undef HPF_NODES
        }
    }
    switch (e.S) {
#define HPF_FINAL(k)                                                                        \
    case k:                                                                                 \
        launch_pdl(k_energy_final<k>, dim3(1), dim3(kFinalBlock), 0, s, (const float2*)bead_part, \
                   nb, (const unsigned long long*)node_part, nn, g.nodes, e, out6);         \
        break;
        HPF_FINAL(1) HPF_FINAL(2) HPF_FINAL(3) HPF_FINAL(4)
        HPF_FINAL(5) HPF_FINAL(6) HPF_FINAL(7) HPF_FINAL(8)
#undef HPF_FINAL
    }
}

// The node sums and the combination, with bead partials formed elsewhere
// (nb_bead CTAs' worth, by the step launch that ended at this state).
void launch_energy_nodes_only(int n, MeshGeom g, const long long* D, const EnergyConsts& e,
                              const float2* bead_part, int nb_bead, double* partials,
                              double* out6, cudaStream_t s) {
    const int nb = energy_blocks(n, kBeadsPerThread);
    const int nn = energy_blocks(g.nodes, kNodesPerThread);
    unsigned long long* node_part =
        reinterpret_cast<unsigned long long*>(partials + (size_t)nb * kBeadVals);
    switch (e.S) {
#define HPF_ONLY(k)                                                                         \
    case k:                                                                                 \
        if (k <= 3)                                                                         \
            k_energy_main<(k <= 3 ? k : 0)><<<nn, kRedBlock, 0, s>>>(                       \
                StateBuf{}, nullptr, 0, g, nullptr, StepConsts{}, 0, e, nullptr, 0, D,      \
                node_part, nn);                                                             \
        else                                                                                \
            k_energy_nodes<k><<<nn, kRedBlock, 0, s>>>(D, g.nodes, node_part);              \
        launch_pdl(k_energy_final<k>, dim3(1), dim3(kFinalBlock), 0, s, bead_part, nb_bead, \
                   (const unsigned long long*)node_part, nn, g.nodes, e, out6);             \
        break;
        HPF_ONLY(1) HPF_ONLY(2) HPF_ONLY(3) HPF_ONLY(4)
        HPF_ONLY(5) HPF_ONLY(6) HPF_ONLY(7) HPF_ONLY(8)
#undef HPF_ONLY
    }
}

}  // namespace hpf
