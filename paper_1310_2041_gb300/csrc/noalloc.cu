// noalloc.cu -- field forces for callers that must not allocate device memory.
//
// hpf_field_forces_noalloc computes the same field force as hpf_forces with
// HPF_FORCE_FIELD (scatter -> field stencil -> gather) without a context and
// without any allocation: its density and field meshes live in one
// file-scope static __device__ array that every GPU loading this library
// holds until the process exits.  Host code may not pass the array's name to
// a kernel (on the host it is only a stand-in for the device symbol), so the
// device address is looked up with cudaGetSymbolAddress once per device, with
// that device current, and cached.
#include <math.h>
#include <string.h>

#include <mutex>

#include "hpf_internal.cuh"

namespace hpf {
namespace {

constexpr int kMaxDevices = 64;

// Device scratch shared by every call on a device: [D | G], each part 256-byte
// aligned.
__device__ __align__(256) unsigned char g_noalloc_scratch[HPF_NOALLOC_SCRATCH_BYTES];

std::mutex g_addr_mutex;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scatter from caller-owned [n][3] positions (tag order).  Species outside
// [0, S) add nothing.
__global__ void k_na_scatter(const float* __restrict__ pos, const int32_t* __restrict__ type,
                             int n, int S, MeshGeom g, unsigned long long* __restrict__ D) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int T = type[i];
    if (T < 0 || T >= S) return;
    const AxisCoord ax = axis_coord(pos[3 * i], g.inv_h[0], g.mx, g.inv_m[0]);
    const AxisCoord ay = axis_coord(pos[3 * i + 1], g.inv_h[1], g.my, g.inv_m[1]);
    const AxisCoord az = axis_coord(pos[3 * i + 2], g.inv_h[2], g.mz, g.inv_m[2]);
    scatter_bead(D + (size_t)T * g.nodes, g, ax, ay, az);
}

// Gather the field force into caller-owned [n][3]; NaN for a species outside [0, S).
__global__ void k_na_gather(const float* __restrict__ pos, const int32_t* __restrict__ type,
                            int n, int S, MeshGeom g, const float4* __restrict__ G,
                            float* __restrict__ F) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int T = type[i];
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (T < 0 || T >= S) {
        fx = fy = fz = __int_as_float(0x7fc00000);
    } else {
        const AxisCoord ax = axis_gather(pos[3 * i], g.inv_h[0], (float)g.mx, g.inv_m[0]);
        const AxisCoord ay = axis_gather(pos[3 * i + 1], g.inv_h[1], (float)g.my, g.inv_m[1]);
        const AxisCoord az = axis_gather(pos[3 * i + 2], g.inv_h[2], (float)g.mz, g.inv_m[2]);
        gather_field(G + (size_t)T * g.gnodes, g, ax, ay, az, fx, fy, fz);
    }
    F[3 * i] = fx;
    F[3 * i + 1] = fy;
    F[3 * i + 2] = fz;
}

// Device memory of the current device (or managed memory): a buffer on
// another GPU would fault in the kernels instead of being refused here.
bool on_device(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

// Device address of the scratch on the current device (looked up once per device).
cudaError_t scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace hpf

using namespace hpf;

extern "C" size_t hpf_noalloc_scratch_bytes(const hpf_params* p) {
    if (!p || p->n_species < 1 || p->n_species > HPF_MAX_SPECIES) return 0;
    for (int a = 0; a < 3; ++a)
        if (p->mesh[a] < 2 || p->mesh[a] > 4096) return 0;
    const size_t nodes = (size_t)p->mesh[0] * p->mesh[1] * p->mesh[2];
    const size_t gnodes = (size_t)(p->mesh[0] + 1) * (p->mesh[1] + 1) * (p->mesh[2] + 1);
    const size_t d = align256(sizeof(unsigned long long) * nodes * p->n_species);
    return d + align256(sizeof(float4) * gnodes * p->n_species);
}

extern "C" hpf_status hpf_field_forces_noalloc(const hpf_params* p, const float* pos,
                                               const int32_t* type, int32_t n, float* F_out,
                                               void* stream) {
    if (!p || n < 0 || n > HPF_MAX_BEADS) return HPF_ERR_INVALID;
    // the same field parameters hpf_init accepts
    if (validate_field_params(p) != HPF_OK) return HPF_ERR_INVALID;
    const size_t need = hpf_noalloc_scratch_bytes(p);
    if (need > (size_t)HPF_NOALLOC_SCRATCH_BYTES) return HPF_ERR_SCRATCH;
    if (n > 0 && (!pos || !type || !F_out || !on_device(pos) || !on_device(type) ||
                  !on_device(F_out)))
        return HPF_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;

    // geometry and stencil coefficients, as hpf_init derives them
    MeshGeom g{};
    g.mx = p->mesh[0];
    g.my = p->mesh[1];
    g.mz = p->mesh[2];
    g.nodes = g.mx * g.my * g.mz;
    g.gx = g.mx + 1;
    g.gxy = (g.mx + 1) * (g.my + 1);
    g.gnodes = g.gxy * (g.mz + 1);
    double h[3], vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        g.inv_h[a] = (float)((double)p->mesh[a] / (double)p->box[a]);
        g.inv_m[a] = 1.0f / (float)p->mesh[a];
        h[a] = (double)p->box[a] / (double)p->mesh[a];
        vol *= h[a];
    }
    const double phi_c = ldexp(1.0, -3 * HPF_FRAC_BITS) / (p->rho0 * vol);
    FieldCoef f;
    memset(&f, 0, sizeof f);
    f.S = p->n_species;
    f.v0 = (float)(-p->inv_kappa);
    for (int k = 0; k < p->n_species; ++k)
        for (int j = 0; j < p->n_species; ++j) {
            const double A = p->kT * p->chi[k * HPF_MAX_SPECIES + j] + p->inv_kappa;
            f.gx[k][j] = (float)(A * phi_c / (2.0 * h[0]));
            f.gy[k][j] = (float)(A * phi_c / (2.0 * h[1]));
            f.gz[k][j] = (float)(A * phi_c / (2.0 * h[2]));
            f.v[k][j] = (float)(A * phi_c);
        }

    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    const size_t dbytes = sizeof(unsigned long long) * (size_t)g.nodes * f.S;
    unsigned long long* D = (unsigned long long*)base;
    float4* G = (float4*)((char*)base + align256(dbytes));

    // the scratch keeps the previous call's contents: clear the mesh first
    if (cudaMemsetAsync(D, 0, dbytes, s) != cudaSuccess) {
        cudaGetLastError();
        return HPF_ERR_CUDA;
    }
    if (n > 0) k_na_scatter<<<(n + 255) / 256, 256, 0, s>>>(pos, type, n, f.S, g, D);
    launch_field(reinterpret_cast<const long long*>(D), g, f, G, nullptr, s);
    if (n > 0) k_na_gather<<<(n + 255) / 256, 256, 0, s>>>(pos, type, n, f.S, g, G, F_out);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HPF_OK : HPF_ERR_CUDA;
}
