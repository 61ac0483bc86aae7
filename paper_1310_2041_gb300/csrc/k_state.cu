// k_state.cu -- loading the bead state into storage order and copying it out.
#include "hpf_internal.cuh"

namespace hpf {

// Tag-order input -> storage arrays + meta word.  err[0] counts species out
// of range, err[1] non-finite coordinates.
__global__ void k_stage_state(const float* __restrict__ pos, const float* __restrict__ vel,
                              const int32_t* __restrict__ type, int n, int S, StateBuf st,
                              uint32_t* __restrict__ meta, int* __restrict__ err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float px = pos[3 * i], py = pos[3 * i + 1], pz = pos[3 * i + 2];
    const float ux = vel[3 * i], uy = vel[3 * i + 1], uz = vel[3 * i + 2];
    const int t = type[i];
    if (t < 0 || t >= S) atomicAdd(err + 0, 1);
    if (!(isfinite(px) && isfinite(py) && isfinite(pz) && isfinite(ux) && isfinite(uy) &&
          isfinite(uz)))
        atomicAdd(err + 1, 1);
    st.x[i] = px;
    st.y[i] = py;
    st.z[i] = pz;
    st.vx[i] = ux;
    st.vy[i] = uy;
    st.vz[i] = uz;
    meta[i] = (uint32_t)i | (((uint32_t)t & kTypeMask) << kTypeShift);
}

// Each bond must join consecutive tags; it sets bonded-to-next on the lower
// and bonded-to-previous on the upper bead.  err[2] counts malformed bonds,
// err[3] bonds given twice.
__global__ void k_mark_bonds(const int32_t* __restrict__ bonds, long long nb, int n,
                             uint32_t* __restrict__ meta, int* __restrict__ err) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int a = bonds[2 * b], c = bonds[2 * b + 1];
    const int lo = a < c ? a : c, hi = a < c ? c : a;
    if (lo < 0 || hi >= n || hi - lo != 1) {
        atomicAdd(err + 2, 1);
        return;
    }
    const uint32_t old = atomicOr(meta + lo, kBondNext);
    if (old & kBondNext) atomicAdd(err + 3, 1);
    atomicOr(meta + hi, kBondPrev);
}

// Storage order -> tag order, with a finiteness check of the state.
__global__ void k_unpermute(StateBuf st, const uint32_t* __restrict__ meta, int n,
                            float* __restrict__ pos_tag, float* __restrict__ vel_tag,
                            int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t tag = meta[i] & kTagMask;
    const float x = st.x[i], y = st.y[i], z = st.z[i];
    const float vx = st.vx[i], vy = st.vy[i], vz = st.vz[i];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) &&
          isfinite(vz)))
        atomicOr(flag, kFlagNonFinite);
    if (pos_tag) {
        pos_tag[3 * tag] = x;
        pos_tag[3 * tag + 1] = y;
        pos_tag[3 * tag + 2] = z;
    }
    if (vel_tag) {
        vel_tag[3 * tag] = vx;
        vel_tag[3 * tag + 1] = vy;
        vel_tag[3 * tag + 2] = vz;
    }
}

// New positions and velocities given in tag order, written in storage order
// (the inverse of k_unpermute); a non-finite value raises the device flag.
// With D, each bead's eight CIC weights of the new positions are also added
// to D[T] (the next field refresh and the observables need that density,
// which then costs no second pass over the beads).
__global__ void k_repermute(const float* __restrict__ pos_tag, const float* __restrict__ vel_tag,
                            const uint32_t* __restrict__ meta, int n, StateBuf st, MeshGeom g,
                            unsigned long long* __restrict__ D, int* __restrict__ flag) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t m = meta[i];
    const uint32_t tag = m & kTagMask;
    const float x = pos_tag[3 * tag], y = pos_tag[3 * tag + 1], z = pos_tag[3 * tag + 2];
    const float vx = vel_tag[3 * tag], vy = vel_tag[3 * tag + 1], vz = vel_tag[3 * tag + 2];
    if (!(isfinite(x) && isfinite(y) && isfinite(z) && isfinite(vx) && isfinite(vy) &&
          isfinite(vz)))
        atomicOr(flag, kFlagNonFinite);
    st.x[i] = x;
    st.y[i] = y;
    st.z[i] = z;
    st.vx[i] = vx;
    st.vy[i] = vy;
    st.vz[i] = vz;
    if (D) {
        const AxisCoord ax = axis_coord(x, g.inv_h[0], g.mx, g.inv_m[0]);
        const AxisCoord ay = axis_coord(y, g.inv_h[1], g.my, g.inv_m[1]);
        const AxisCoord az = axis_coord(z, g.inv_h[2], g.mz, g.inv_m[2]);
        scatter_bead(D + (size_t)((m >> kTypeShift) & kTypeMask) * g.nodes, g, ax, ay, az);
    }
}

__global__ void k_order(const uint32_t* __restrict__ meta, int n, int32_t* __restrict__ order) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[i] = (int32_t)(meta[i] & kTagMask);
}

void launch_order(const uint32_t* meta, int n, int32_t* order, cudaStream_t s) {
    if (n <= 0) return;
    k_order<<<(n + 255) / 256, 256, 0, s>>>(meta, n, order);
}

__global__ void k_advance_counter(long long* step, long long by) { *step += by; }

void launch_advance_counter(long long* step, long long by, cudaStream_t s) {
    k_advance_counter<<<1, 1, 0, s>>>(step, by);
}

__global__ void k_set_counter(long long* step, long long v) { *step = v; }

void launch_set_counter(long long* step, long long v, cudaStream_t s) {
    k_set_counter<<<1, 1, 0, s>>>(step, v);
}

void launch_stage_state(const float* pos, const float* vel, const int32_t* type, int n, int S,
                        StateBuf st, uint32_t* meta, int* err, cudaStream_t s) {
    if (n <= 0) return;
    k_stage_state<<<(n + 255) / 256, 256, 0, s>>>(pos, vel, type, n, S, st, meta, err);
}

void launch_mark_bonds(const int32_t* bonds, long long nb, int n, uint32_t* meta, int* err,
                       cudaStream_t s) {
    if (nb <= 0) return;
    k_mark_bonds<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(bonds, nb, n, meta, err);
}

void launch_repermute(const float* pos_tag, const float* vel_tag, const uint32_t* meta, int n,
                      StateBuf st, const MeshGeom& g, unsigned long long* D, int* flag,
                      cudaStream_t s) {
    if (n <= 0) return;
    k_repermute<<<(n + 255) / 256, 256, 0, s>>>(pos_tag, vel_tag, meta, n, st, g, D, flag);
}

void launch_unpermute(StateBuf st, const uint32_t* meta, int n, float* pos_tag, float* vel_tag,
                      int* flag, cudaStream_t s) {
    if (n <= 0) return;
    k_unpermute<<<(n + 255) / 256, 256, 0, s>>>(st, meta, n, pos_tag, vel_tag, flag);
}

}  // namespace hpf
