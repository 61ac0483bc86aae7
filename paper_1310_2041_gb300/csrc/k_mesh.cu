// k_mesh.cu -- density scatter (CIC, int64 fixed point) and the field stencil.
#include "hpf_internal.cuh"

namespace hpf {

// ------------------------------------------------------------------ A2 scatter
//
// One thread per bead adds its eight fixed-point CIC weights to D[T].  The
// weights are integers, so the mesh is the same for any summation order.
__global__ void __launch_bounds__(256) k_scatter(StateBuf st, const uint32_t* __restrict__ meta,
                                                 int n, MeshGeom g,
                                                 unsigned long long* __restrict__ D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float x = st.x[i], y = st.y[i], z = st.z[i];
    const uint32_t m = meta[i];
    const int T = (m >> kTypeShift) & kTypeMask;
    const AxisCoord ax = axis_coord(x, g.inv_h[0], g.mx, g.inv_m[0]);
    const AxisCoord ay = axis_coord(y, g.inv_h[1], g.my, g.inv_m[1]);
    const AxisCoord az = axis_coord(z, g.inv_h[2], g.mz, g.inv_m[2]);
    scatter_bead(D + (size_t)T * g.nodes, g, ax, ay, az);
}

void launch_scatter(StateBuf st, const uint32_t* meta, int n, MeshGeom g, unsigned long long* D,
                    cudaStream_t s) {
    if (n <= 0) return;
    k_scatter<<<(n + 255) / 256, 256, 0, s>>>(st, meta, n, g, D);
}

// ------------------------------------------------------------------ A3 field
//
// One thread per node.  Integer central differences of every species' count
// are exact; the potential gradient is their FP32 combination with the
// coefficients A_KK' c / (2h), A = kT chi + inv_kappa, c = 2^-39 / (rho0 h^3).
template <int S>
__device__ __forceinline__ void field_node(const long long* __restrict__ D, const MeshGeom& g,
                                           const FieldCoef& c, float4* __restrict__ G,
                                           unsigned long long* __restrict__ D_clear, int pnode) {
    // one node of the ghosted field array; ghost nodes repeat the periodic image
    const int px = pnode % g.gx;
    const int py = (pnode / g.gx) % (g.my + 1);
    const int pz = pnode / g.gxy;
    const int x = px == g.mx ? 0 : px, y = py == g.my ? 0 : py, z = pz == g.mz ? 0 : pz;
    const int node = (z * g.my + y) * g.mx + x;
    if (D_clear && px < g.mx && py < g.my && pz < g.mz) {
#pragma unroll
        for (int k = 0; k < S; ++k) D_clear[(size_t)k * g.nodes + node] = 0ull;
    }
    const int xp = node + ((x + 1 == g.mx) ? 1 - g.mx : 1);
    const int xm = node + ((x == 0) ? g.mx - 1 : -1);
    const int sy = g.mx, sz = g.mx * g.my;
    const int yp = node + ((y + 1 == g.my) ? (1 - g.my) * sy : sy);
    const int ym = node + ((y == 0) ? (g.my - 1) * sy : -sy);
    const int zp = node + ((z + 1 == g.mz) ? (1 - g.mz) * sz : sz);
    const int zm = node + ((z == 0) ? (g.mz - 1) * sz : -sz);
    float ddx[S], ddy[S], ddz[S], dc[S];
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const long long* Dk = D + (size_t)k * g.nodes;
        ddx[k] = (float)(__ldg(Dk + xp) - __ldg(Dk + xm));
        ddy[k] = (float)(__ldg(Dk + yp) - __ldg(Dk + ym));
        ddz[k] = (float)(__ldg(Dk + zp) - __ldg(Dk + zm));
        dc[k] = (float)__ldg(Dk + node);
    }
#pragma unroll
    for (int k = 0; k < S; ++k) {
        float gx = 0.f, gy = 0.f, gz = 0.f, v = c.v0;
#pragma unroll
        for (int kp = 0; kp < S; ++kp) {
            gx += c.gx[k][kp] * ddx[kp];
            gy += c.gy[k][kp] * ddy[kp];
            gz += c.gz[k][kp] * ddz[kp];
            v += c.v[k][kp] * dc[kp];
        }
        G[(size_t)k * g.gnodes + pnode] = make_float4(gx, gy, gz, v);
    }
}

template <int S>
__global__ void __launch_bounds__(256) k_field(const long long* __restrict__ D, MeshGeom g,
                                               FieldCoef c, float4* __restrict__ G,
                                               unsigned long long* __restrict__ D_clear) {
    const int pnode = blockIdx.x * blockDim.x + threadIdx.x;
    if (pnode >= g.gnodes) return;
    field_node<S>(D, g, c, G, D_clear, pnode);
}

// All replicas of a batch: each block belongs to one replica (block-uniform).
template <int S>
__global__ void __launch_bounds__(256) k_field_batch(const __grid_constant__ BatchFieldParams p) {
    int lo = 0, hi = p.R - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.rep[mid].blk_begin <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const BatchFieldRep& r = p.rep[lo];
    const int pnode = ((int)blockIdx.x - r.blk_begin) * blockDim.x + threadIdx.x;
    if (pnode >= r.g.gnodes) return;
    field_node<S>(r.D, r.g, p.coef[lo], r.G, r.D_clear, pnode);
}

void launch_field_batch(const BatchFieldParams& p, int S, cudaStream_t s) {
    if (p.blocks <= 0) return;
    switch (S) {
        case 1: k_field_batch<1><<<p.blocks, 256, 0, s>>>(p); break;
        case 2: k_field_batch<2><<<p.blocks, 256, 0, s>>>(p); break;
        case 3: k_field_batch<3><<<p.blocks, 256, 0, s>>>(p); break;
        case 4: k_field_batch<4><<<p.blocks, 256, 0, s>>>(p); break;
        case 5: k_field_batch<5><<<p.blocks, 256, 0, s>>>(p); break;
        case 6: k_field_batch<6><<<p.blocks, 256, 0, s>>>(p); break;
        case 7: k_field_batch<7><<<p.blocks, 256, 0, s>>>(p); break;
        default: k_field_batch<8><<<p.blocks, 256, 0, s>>>(p); break;
    }
}

// Ghosted field array -> dense [S][Mz][My][Mx] float4.
__global__ void k_unpad_field(const float4* __restrict__ G, MeshGeom g, int S,
                              float4* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)S * g.nodes) return;
    const int k = (int)(i / g.nodes), node = (int)(i % g.nodes);
    const int x = node % g.mx, y = (node / g.mx) % g.my, z = node / (g.mx * g.my);
    out[i] = G[(size_t)k * g.gnodes + (size_t)z * g.gxy + y * g.gx + x];
}

void launch_unpad_field(const float4* G, MeshGeom g, int S, float4* out, cudaStream_t s) {
    const long long n = (long long)S * g.nodes;
    k_unpad_field<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G, g, S, out);
}

void launch_field(const long long* D, MeshGeom g, const FieldCoef& coef, float4* G,
                  unsigned long long* D_clear, cudaStream_t s) {
    const int blocks = (g.gnodes + 255) / 256;
    switch (coef.S) {
        case 1: k_field<1><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 2: k_field<2><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 3: k_field<3><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 4: k_field<4><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 5: k_field<5><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 6: k_field<6><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        case 7: k_field<7><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
        default: k_field<8><<<blocks, 256, 0, s>>>(D, g, coef, G, D_clear); break;
    }
}

}  // namespace hpf
