// nh_internal.cuh -- declarations of the Nose-Hoover NVT steps (k_nh.cu).
#pragma once

#include "hpf_internal.cuh"

namespace hpf {

// Nose-Hoover thermostat: device-resident state of one context.
struct NhDev {
    double xi, eta;       // at the middle of the last step
    double ke;            // kinetic energy of the last reduction (v^E, before the half steps)
    float s1, s2;         // velocity scales of the last two thermostat half steps
    unsigned int ticket;  // blocks done with the current reduction
};
struct NhConsts {
    double h;         // dt / 2
    double dof_kT;    // g kT, g = 3 (n - 1) kinetic degrees of freedom (3 for n = 1)
    double two_over_dof_kT;  // 2 / (g kT) (0 when g kT = 0)
    double inv_tau2;  // 1 / tau^2
    double mass;
};
struct NhParams {
    StateBuf in, out;     // state read (every bead's old values) and written
    const float* Fin[3];  // conservative force of the previous force evaluation
    float* Fout[3];       // written by force_kick launches
    const uint32_t* meta;
    int n;
    MeshGeom g;
    const float4* G;
    StepConsts c;
    NhConsts t;
    NhDev* nh;
    float2* part;     // [blocks] kinetic-energy partials (float-float)
    unsigned long long* D_next;  // deposit the final positions (kick_drift-only launches)
    int* flag;
    int kick_drift;  // v = s2 (s1 v) + dt/(2m) F; x += dt v
    int force_kick;  // F at the (new) positions; v += dt/(2m) F; K; thermostat half steps
};

int nh_blocks(int n);
void launch_nh_step(const NhParams& p, cudaStream_t s);

}  // namespace hpf
