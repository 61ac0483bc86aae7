/*
 * hpf_oracle.h -- plain CPU oracle of the hybrid particle-field MD step.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct reference the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it; the product path never does.
 * It shares no code with the CUDA library.
 *
 * Arithmetic: FP64 everywhere except the density mesh, which is accumulated
 * as 64-bit fixed-point integers (13 fractional bits per axis, so one bead
 * adds 2^39 in total).  Long double is used for the energy sums.
 *
 * Layouts (all row-major, C order):
 *   pos, vel, force : [n][3]
 *   D (density)     : int64 [S][Mz][My][Mx]     (x fastest)
 *   V (potential)   : double [S][Mz][My][Mx]
 *   G (grad V)      : double [S][Mz][My][Mx][3]
 *   BL / BN         : bond table in the paper's column-major form, entry
 *                     (i, k) at BL[k * n + i], BN[i] bonds of bead i
 *                     (section "MD methods and algorithms", Fig. 2)
 *
 * Parity status of each function is stated beside it.
 */
#ifndef HPF_ORACLE_H
#define HPF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_SPECIES 8
#define ORC_FRAC_BITS 13
#define ORC_MAX_BONDS 8

typedef struct {
    int32_t n_species;
    int32_t mesh[3];
    float box[3];
    double kT;
    double rho0;
    double inv_kappa;
    double chi[ORC_MAX_SPECIES * ORC_MAX_SPECIES]; /* [K][K'] in kT units */
    double bond_k;
    double bond_r0;
    double mass;
    double dt;
    double gamma;
    uint64_t seed;
    int32_t field_every;
    int32_t force_mode; /* 0: interpolated central-difference gradient (Algorithm 1);
                           1: exact derivative of the CIC field energy (pinning variant);
                           2: Algorithm 1's staggered differences blended at the
                              nearest vertex (orc_field_force_staggered) */
    double angle_k;     /* U = angle_k (cos theta - angle_cos0)^2 per bonded triplet */
    double angle_cos0;  /* (section "Bonded forces", the cosine form); 0: no angles;
                           with angle_form 1 U = angle_k (theta - angle_theta0)^2 */
    int32_t thermostat; /* 0: Langevin (gamma); 1: Nose-Hoover (section "MD methods and
                           algorithms" names it for NVT; orc_run_nh); 2: Andersen
                           (named there too; orc_run) */
    double nh_tau;      /* Nose-Hoover relaxation time tau (> 0) */
    double andersen_nu; /* Andersen collision frequency nu (>= 0) */
    double dihedral_k;  /* U = dihedral_k [1 + cos(dihedral_n phi - dihedral_delta)] per */
    int32_t dihedral_n; /* bonded quadruplet (section "Bonded forces"); 0: none */
    double dihedral_delta;
    int32_t angle_form;  /* 0: the cosine form; 1: the harmonic form in theta (radians) */
    double angle_theta0;
} orc_params;

int orc_num_threads(void);

/* Philox4x32-10 (Salmon et al., SC'11), counter ctr[4], key key[2]. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Three standard normals for bead `tag` at step `step` (Box-Muller). */
void orc_gauss3(uint64_t seed, uint32_t tag, int64_t step, double xi[3]);
/* Andersen collision of bead `tag` at step `step`: the uniform u of word 0 of
 * Philox4x32-10(counter = (tag, step lo, step hi, 1), key = seed), compared in
 * FP32 (both exact there): u < fl32(nu dt).  Returns 1 for a collision. */
int orc_andersen_collides(const orc_params* p, uint32_t tag, int64_t step);

/* Inverse mesh spacing per axis, fl32(M / L). */
float orc_inv_h(const orc_params* p, int axis);

/* Cloud-in-cell scatter into the fixed-point mesh (D is overwritten). */
void orc_scatter(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                 int64_t* D);
/* Nodal potential V_K and its central-difference gradient G. */
void orc_field(const orc_params* p, const int64_t* D, double* V, double* G);
/* Field force on each bead: trilinear interpolation of -G of its species. */
void orc_field_force(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                     const double* G, double* F);
/* Variant force: exact derivative of the CIC field energy for the potential V. */
void orc_field_force_exact(const orc_params* p, int64_t n, const double* pos, const int32_t* type,
                           const double* V, double* F);
/* Angle forces and energy: every pair (a, b) of bond partners of a bead j
 * forms the angle theta at j between x_a - x_j and x_b - x_j (pi for a
 * straight chain), with U = angle_k (cos theta - angle_cos0)^2, or with
 * angle_form 1 U = angle_k (theta - angle_theta0)^2. */
void orc_angle_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                     const int32_t* BN, double* F);
double orc_angle_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                        const int32_t* BN);
/* Build the BL / BN bond table from a list of bonded pairs; returns 0 or -1 on overflow. */
void orc_field_force_staggered(const orc_params* p, int64_t n, const double* pos,
                               const int32_t* type, const double* V, double* F);
/* Dihedrals (orc_dihedral_force / orc_dihedral_energy): every bonded
 * quadruplet (a, j, k, b), phi the angle between the planes (a, j, k) and
 * (j, k, b): with r_ij = x_a - x_j, r_kj = x_k - x_j, r_kl = x_k - x_b,
 * m = r_ij x r_kj, n = r_kj x r_kl, phi = atan2(|r_kj| (r_ij . n), m . n)
 * (trans +-pi, cis 0).  Parity: pinned (closed forms in phi, minus the
 * numerical energy derivative, zero net force and torque). */
void orc_dihedral_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                        const int32_t* BN, double* F);
double orc_dihedral_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                           const int32_t* BN);
int orc_bond_table(int64_t n, int64_t n_bonds, const int32_t* pairs, int32_t* BL, int32_t* BN);
/* Harmonic bond force per bead, each bond evaluated from both ends. */
void orc_bond_force(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                    const int32_t* BN, double* F);
/* Bond energy sum_bonds k (r - r0)^2 (each bond once). */
double orc_bond_energy(const orc_params* p, int64_t n, const double* pos, const int32_t* BL,
                       const int32_t* BN);
/* Field energy W of a density mesh. */
double orc_field_energy(const orc_params* p, const int64_t* D);

/* Energies at step `step` for the state (pos = x_n, vel = v_{n-1/2}) with the
 * field (V, G) in force: out = {kinetic, bond, field, total, |P|, T}. */
void orc_energy(const orc_params* p, int64_t n, const double* pos, const double* vel,
                const int32_t* type, const int32_t* BL, const int32_t* BN, const double* V,
                const double* G, int64_t step, double out[6]);

/* Advance n_steps steps from step0.  pos / vel are updated in place (vel holds
 * the half-step velocity).  If energies != NULL, energies[k*6 .. k*6+5] get
 * orc_energy() at step0 + k for k = 0 .. n_steps.  Returns 0, or -1 on bad input. */
int orc_run(const orc_params* p, int64_t n, double* pos, double* vel, const int32_t* type,
            int64_t n_bonds, const int32_t* pairs, int64_t step0, int32_t n_steps,
            double* energies);

/* Chain order used by the bead sort: key of each chain (first bead's cell in
 * brick-major order, bricks of `brick` cells per axis). */
/* Nose-Hoover NVT (section "MD methods and algorithms" names the thermostat;
 * the equations are Hoover's): dv/dt = F/m - xi v, dxi/dt = (2 K / (g kT) - 1) / tau^2,
 * deta/dt = xi, g = 3 (n - 1) kinetic degrees of freedom (3 for n = 1); the
 * extended energy E + g kT (tau^2 xi^2 / 2 + eta) is conserved.  State
 * (x_n, v_{n-1/2}, xi, eta) with xi, eta at the middle of step n - 1.  Each
 * step n: refresh the field if due; F_n; v^E = v + dt/(2m) F_n (the on-step
 * velocity before the thermostat); two thermostat half steps T(dt/2) (the end
 * of step n - 1 and the start of step n), each
 *   xi += (h/2) G(K); v *= exp(-xi h); K *= exp(-2 xi h); eta += xi h;
 *   xi += (h/2) G(K),      G(K) = (2 K / (g kT) - 1) / tau^2, h = dt/2;
 * then v <- v + dt/(2m) F_n; x <- x + dt v.  xe = (xi, eta) in and out.
 * energies (optional): [n_steps + 1][7] records at each step before its
 * update: kinetic (on-step, after the pending half step), bonded, field,
 * total, |P|, T, and the extended energy.  Returns 0, or -1 on bad input.
 * Parity: pinned (NVE limit, free-particle thermostat ODE, extended-energy
 * conservation, mean temperature). */
int orc_run_nh(const orc_params* p, int64_t n, double* pos, double* vel, const int32_t* type,
               int64_t n_bonds, const int32_t* pairs, int64_t step0, int32_t n_steps,
               double xe[2], double* energies);

int64_t orc_cell_key(const orc_params* p, const double* x, int32_t brick);

#ifdef __cplusplus
}
#endif
#endif
